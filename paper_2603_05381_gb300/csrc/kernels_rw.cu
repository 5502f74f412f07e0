// Second stage of B-BP4MF (Sec. "Belief-BP4MF (B-BP4MF)", Sec. "Correlated decoding"):
// the shared-memory decoding kernel in its reweighting mode.  Each block first runs
// Dijkstra from every unsatisfied check of its shot over the decoding graph whose edge
// weights come from the first stage's qubit posteriors, then BP4MF on the resulting
// priors.  Per-shot W, parity and the Dijkstra state live in a global scratch slot per
// resident block.
#include <cuda_runtime.h>

#include "decode_smem.cuh"
#include "device.cuh"

namespace bp4m {
namespace {

template <typename T, int CH, int G, bool REG>
cudaError_t rw_grid(int n_det, int num_sms, int* grid, int64_t* slot_bytes, size_t* smem_out) {
    constexpr int SMAX = CH * G, NT = CH * G * G;
    const size_t smem = smem_bytes_of<T, CH, G>();
    auto kern = decode_smem_kernel<T, CH, G, false, REG, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid = per_sm * num_sms;
    *slot_bytes = rw_slot_layout(SMAX, NT, n_det + 1);
    *smem_out = smem;
    return cudaSuccess;
}

template <typename T, int CH, int G, bool REG>
cudaError_t run_tier_rw(const DecodeArgs& a, int num_sms, cudaStream_t st, int64_t* query) {
    int grid = 0;
    int64_t slot = 0;
    size_t smem = 0;
    cudaError_t e = rw_grid<T, CH, G, REG>(a.tb.n_det, num_sms, &grid, &slot, &smem);
    if (e != cudaSuccess) return e;
    if (query) {
        query[0] = (int64_t)grid * slot;
        query[1] = slot;
        return cudaSuccess;
    }
    // every block indexes its own slot: the scratch must hold grid slots of this tier's size
    if (a.gscratch == nullptr || a.rw_slot_bytes != slot || (int64_t)grid * slot > a.gscratch_bytes)
        return cudaErrorInvalidValue;
    decode_smem_kernel<T, CH, G, false, REG, true><<<grid, CH * G * G, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t dispatch_rw(int precision, int tier, const DecodeArgs& a, int num_sms, cudaStream_t st,
                        int64_t* query) {
    if (precision == 0) {
        switch (tier) {
            case 1: return run_tier_rw<double, 16, 2, false>(a, num_sms, st, query);
            case 2: return run_tier_rw<double, 16, 4, false>(a, num_sms, st, query);
            case 3: return run_tier_rw<double, 28, 4, false>(a, num_sms, st, query);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (tier) {
        case 1: return run_tier_rw<float, 32, 1, kReg32[1]>(a, num_sms, st, query);
        case 2: return run_tier_rw<float, 32, 2, kReg32[2]>(a, num_sms, st, query);
        case 3: return run_tier_rw<float, 24, 4, kReg32[3]>(a, num_sms, st, query);
        case 4: return run_tier_rw<float, 28, 4, kReg32[4]>(a, num_sms, st, query);
        case 5: return run_tier_rw<float, 32, 4, kReg32[5]>(a, num_sms, st, query);
        case 6: return run_tier_rw<float, 36, 4, kReg32[6]>(a, num_sms, st, query);
        case 7: return run_tier_rw<float, 40, 4, kReg32[7]>(a, num_sms, st, query);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t rw_scratch_bytes(int precision, int tier, int n_det, int num_sms, int64_t* slot_bytes) {
    DecodeArgs a;
    a.tb.n_det = n_det;
    int64_t q[2] = {0, 0};
    if (dispatch_rw(precision, tier, a, num_sms, 0, q) != cudaSuccess) return 0;
    if (slot_bytes) *slot_bytes = q[1];
    return (size_t)q[0];
}

cudaError_t launch_decode_tier_rw(int precision, int tier, const DecodeArgs& a, int num_sms,
                                  cudaStream_t st) {
    return dispatch_rw(precision, tier, a, num_sms, st, nullptr);
}

}  // namespace bp4m
