// Sampling, syndrome extraction, defect classification and failure counting.
//
// Sampler: every (shot, unit) pair takes one 32-bit word of Philox4x32-10 (Salmon et al.,
// SC'11) with counter (shot low, shot high, unit >> 2, stream id) and key (seed low, seed
// high), word unit & 3.  Code capacity: unit = data qubit, X if u < t1, Y if u < t2, Z if
// u < t3 (t_k = floor(k p / 3 * 2^32)).  Circuit: unit = merged detector-graph edge, it
// fires iff u < floor(q_e * 2^32).  The syndrome is the XOR of the fired edges' endpoints
// and the true observable flip the XOR of their observable bits (the paper decodes X and Z
// errors separately, Sec. "MWPM on the surface code").
#include <cuda_runtime.h>

#include "device.cuh"

namespace bp4m {
namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4& r, int j) {
    return j == 0 ? r.x : j == 1 ? r.y : j == 2 ? r.z : r.w;
}

constexpr int kSampWarps = 8;

// One warp per shot; lanes take blocks of four units; fired edges XOR into a per-warp
// shared-memory syndrome.
__global__ void __launch_bounds__(kSampWarps * 32) sample_circuit_kernel(SampleArgs a) {
    extern __shared__ uint32_t smem_sw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = a.n_words[0];
    const int n_det = a.n_det[0];
    uint32_t* my = smem_sw + warp * nw;
    const int n_blocks = (a.n_units + 3) >> 2;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    for (int64_t shot = (int64_t)blockIdx.x * kSampWarps + warp; shot < a.shots;
         shot += (int64_t)gridDim.x * kSampWarps) {
        for (int w = lane; w < nw; w += 32) my[w] = 0u;
        __syncwarp();
        const uint64_t gs = a.first_shot + (uint64_t)shot;
        uint32_t obs = 0;
        for (int b = lane; b < n_blocks; b += 32) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)gs, (uint32_t)(gs >> 32),
                                                     (uint32_t)b, a.stream_id), k0, k1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int e = 4 * b + j;
                if (e < a.n_units && word_of(r, j) < __ldg(a.thr + e)) {
                    const uint32_t p = __ldg(a.uvo + e);
                    const int u = (int)(p & 0x7FFFu), v = (int)((p >> 15) & 0x7FFFu);
                    atomicXor(my + (u >> 5), 1u << (u & 31));
                    if (v < n_det) atomicXor(my + (v >> 5), 1u << (v & 31));
                    obs ^= p >> 31;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int off = 16; off; off >>= 1) obs ^= __shfl_xor_sync(0xffffffffu, obs, off);
        uint32_t* dst = a.synd + (size_t)shot * nw;
        for (int w = lane; w < nw; w += 32) dst[w] = my[w];
        if (lane == 0) a.obs[shot] = (uint8_t)obs;
        __syncwarp();
    }
}

constexpr int kCcThreads = 128;
constexpr int kCcMaxWords = 32;  // d <= 45

// One thread per shot; both Pauli types from the same draw.
__global__ void __launch_bounds__(kCcThreads) sample_cc_kernel(SampleArgs a) {
    __shared__ uint32_t sw[2][kCcMaxWords][kCcThreads];
    const int t = threadIdx.x;
    const int nw0 = a.n_words[0], nw1 = a.n_words[1];
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const uint32_t t1 = a.cc_thr[0], t2 = a.cc_thr[1], t3 = a.cc_thr[2];
    const int n0 = a.n_det[0], n1 = a.n_det[1];
    for (int64_t shot = (int64_t)blockIdx.x * kCcThreads + t; shot < a.shots;
         shot += (int64_t)gridDim.x * kCcThreads) {
        for (int w = 0; w < nw0; ++w) sw[0][w][t] = 0u;
        for (int w = 0; w < nw1; ++w) sw[1][w][t] = 0u;
        uint32_t obs0 = 0, obs1 = 0;
        const uint64_t gs = a.first_shot + (uint64_t)shot;
        const int n_blocks = (a.n_units + 3) >> 2;
        for (int b = 0; b < n_blocks; ++b) {
            const uint4 r = philox4x32_10(make_uint4((uint32_t)gs, (uint32_t)(gs >> 32),
                                                     (uint32_t)b, a.stream_id), k0, k1);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = 4 * b + j;
                if (q >= a.n_units) break;
                const uint32_t u = word_of(r, j);
                if (u < t2) {  // X or Y: flips the Z-checks (type 0)
                    const uint32_t p = __ldg(a.cc_uvo + q);
                    const int uu = (int)(p & 0x7FFFu), vv = (int)((p >> 15) & 0x7FFFu);
                    sw[0][uu >> 5][t] ^= 1u << (uu & 31);
                    if (vv < n0) sw[0][vv >> 5][t] ^= 1u << (vv & 31);
                    obs0 ^= p >> 31;
                }
                if (u >= t1 && u < t3) {  // Y or Z: flips the X-checks (type 1)
                    const uint32_t p = __ldg(a.cc_uvo + a.n_units + q);
                    const int uu = (int)(p & 0x7FFFu), vv = (int)((p >> 15) & 0x7FFFu);
                    sw[1][uu >> 5][t] ^= 1u << (uu & 31);
                    if (vv < n1) sw[1][vv >> 5][t] ^= 1u << (vv & 31);
                    obs1 ^= p >> 31;
                }
            }
        }
        uint32_t* d0 = a.synd + (size_t)shot * nw0;
        uint32_t* d1 = a.synd + (size_t)a.shots * nw0 + (size_t)shot * nw1;
        for (int w = 0; w < nw0; ++w) d0[w] = sw[0][w][t];
        for (int w = 0; w < nw1; ++w) d1[w] = sw[1][w][t];
        a.obs[shot] = (uint8_t)obs0;
        a.obs[a.shots + shot] = (uint8_t)obs1;
    }
}

constexpr int kClsThreads = 256;

__global__ void __launch_bounds__(kClsThreads) classify_kernel(
    const uint32_t* __restrict__ synd, int64_t shots, int n_words, TierPlan plan,
    int32_t* lists, int32_t* counts, int32_t* max_s, uint8_t* obs_pred, uint8_t* flags,
    int16_t* iters, int32_t* tr_defects, const uint8_t* skip, const uint8_t* skip_obs,
    const int16_t* skip_iters, int64_t list_stride, int32_t item_base) {
    int local_max = 0;
    for (int64_t shot = (int64_t)blockIdx.x * kClsThreads + threadIdx.x; shot < shots;
         shot += (int64_t)gridDim.x * kClsThreads) {
        const uint32_t* w = synd + (size_t)shot * n_words;
        int s = 0;
        for (int k = 0; k < n_words; ++k) s += __popc(__ldg(w + k));
        if (tr_defects) tr_defects[shot] = s;
        if (skip && skip[shot]) {
            if (obs_pred) obs_pred[shot] = skip_obs[shot];
            if (flags) flags[shot] = F_CONVERGED | F_FROM_QBP;
            if (iters) iters[shot] = skip_iters[shot];
            continue;
        }
        local_max = max(local_max, s);
        if (s == 0) {
            if (obs_pred) obs_pred[shot] = 0;
            if (flags) flags[shot] = F_CONVERGED;
            if (iters) iters[shot] = 0;
            continue;
        }
        int tier = kGlobalTier;
        for (int k = 1; k < kGlobalTier; ++k)
            if (s <= plan.smax[k]) {
                tier = k;
                break;
            }
        const int pos = atomicAdd(counts + tier, 1);
        lists[(size_t)tier * list_stride + pos] = item_base | (int32_t)shot;
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, off));
    if ((threadIdx.x & 31) == 0 && local_max > 0) atomicMax(max_s, local_max);
}

constexpr int kCntThreads = 256;

__global__ void __launch_bounds__(kCntThreads) count_kernel(
    const uint8_t* __restrict__ obs_true, const uint8_t* __restrict__ obs_pred,
    const uint8_t* __restrict__ flags, int64_t shots, int n_types, unsigned long long* ctr) {
    unsigned long long c[C_NUM] = {};
    for (int64_t shot = (int64_t)blockIdx.x * kCntThreads + threadIdx.x; shot < shots;
         shot += (int64_t)gridDim.x * kCntThreads) {
        c[C_SHOTS] += 1;
        bool any = false, all_conv = true;
        for (int ty = 0; ty < n_types; ++ty) {
            const size_t k = (size_t)ty * shots + shot;
            const bool fail = obs_true[k] != obs_pred[k];
            const uint8_t f = flags[k];
            any |= fail;
            all_conv &= (f & F_CONVERGED) != 0;
            c[C_FAIL_X + ty] += fail;
            c[C_UNCONV_X + ty] += !(f & F_CONVERGED);
            c[C_FORCED_X + ty] += (f & F_FROM_FORCED) ? 1 : 0;
            c[C_CONVFAIL_X + ty] += (fail && (f & F_CONVERGED)) ? 1 : 0;
        }
        c[C_FAIL_ANY] += any;
        c[C_UNCONV_ANY] += !all_conv;
        c[C_CONVFAIL_ANY] += (all_conv && any) ? 1 : 0;
    }
    for (int k = 0; k < C_NUM; ++k) {
        if (k >= C_ITERS && k != C_UNCONV_ANY && k != C_CONVFAIL_ANY) continue;
        unsigned long long v = c[k];
#pragma unroll
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr + k, v);
    }
}

// ---- MUFU throughput probe (measurement support; the roofline denominator of the
// shared-memory decode tiers).  Each thread runs kProbeChains independent chains of
// `steps` special-function operations; a block of 1024 threads (one per SM: the launch
// bounds and a large dynamic shared-memory request keep a second block off the SM) times
// its loop with the SM cycle counter.  Modes: 0 = ex2 (x <- 1 - ex2(x)/2, one FMA beside
// each ex2), 1 = lg2 (x <- lg2(x) + 2, one add beside each lg2), 2 = ex2 and lg2
// alternating (x <- lg2(ex2(x)), no other arithmetic).  The FMA/add pipe and the issue
// slots they take stay far below their own limits at these rates, so the MUFU unit bounds
// every mode.
constexpr int kProbeThreads = 1024;
constexpr int kProbeChains = 8;

__device__ __forceinline__ float probe_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float probe_lg2(float x) {
    float y;
    asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int MODE>
__global__ void __launch_bounds__(kProbeThreads, 1) mufu_probe_kernel(int steps, long long* cycles, float* sink) {
    float x[kProbeChains];
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) x[j] = (MODE == 1 ? 4.0f : 0.35f) + 1e-3f * j + 1e-7f * threadIdx.x;
    __syncthreads();
    const long long t0 = clock64();
    for (int s = 0; s < steps; ++s) {
#pragma unroll
        for (int j = 0; j < kProbeChains; ++j) {
            if (MODE == 0) x[j] = fmaf(probe_ex2(x[j]), -0.5f, 1.0f);
            if (MODE == 1) x[j] = probe_lg2(x[j]) + 2.0f;
            if (MODE == 2) x[j] = probe_lg2(probe_ex2(x[j]));
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < kProbeChains; ++j) acc += x[j];
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

int grid_for(int64_t items, int per_block, int cap) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

cudaError_t launch_sample_circuit(const SampleArgs& a, cudaStream_t st) {
    if (a.shots <= 0) return cudaSuccess;
    const size_t smem = (size_t)kSampWarps * a.n_words[0] * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(sample_circuit_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    sample_circuit_kernel<<<grid_for(a.shots, kSampWarps, 152 * 16), kSampWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sample_code_capacity(const SampleArgs& a, cudaStream_t st) {
    if (a.shots <= 0) return cudaSuccess;
    if (a.n_words[0] > kCcMaxWords || a.n_words[1] > kCcMaxWords) return cudaErrorInvalidValue;
    sample_cc_kernel<<<grid_for(a.shots, kCcThreads, 152 * 8), kCcThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_classify(const uint32_t* synd, int64_t shots, int n_words, const TierPlan& plan,
                            int32_t* lists, int32_t* counts, int32_t* max_s, uint8_t* obs_pred,
                            uint8_t* flags, int16_t* iters, int32_t* tr_defects, const uint8_t* skip,
                            const uint8_t* skip_obs, const int16_t* skip_iters, cudaStream_t st,
                            int64_t list_stride, int32_t item_base) {
    if (shots <= 0) return cudaSuccess;
    classify_kernel<<<grid_for(shots, kClsThreads, 152 * 8), kClsThreads, 0, st>>>(
        synd, shots, n_words, plan, lists, counts, max_s, obs_pred, flags, iters, tr_defects, skip,
        skip_obs, skip_iters, list_stride > 0 ? list_stride : shots, item_base);
    return cudaGetLastError();
}

cudaError_t launch_mufu_probe(int mode, int blocks, int steps, long long* cycles, float* sink, cudaStream_t st) {
    // 120 KB of dynamic shared memory (unused) so that no SM holds two probe blocks
    const int smem = 120 * 1024;
    auto launch = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        kern<<<blocks, kProbeThreads, smem, st>>>(steps, cycles, sink);
        return cudaGetLastError();
    };
    if (mode == 0) return launch(mufu_probe_kernel<0>);
    if (mode == 1) return launch(mufu_probe_kernel<1>);
    if (mode == 2) return launch(mufu_probe_kernel<2>);
    return cudaErrorInvalidValue;
}

int mufu_probe_ops_per_thread(int mode, int steps) { return kProbeChains * steps * (mode == 2 ? 2 : 1); }

cudaError_t launch_count(const uint8_t* obs_true, const uint8_t* obs_pred, const uint8_t* flags,
                         int64_t shots, int n_types, unsigned long long* ctr, cudaStream_t st) {
    if (shots <= 0) return cudaSuccess;
    count_kernel<<<grid_for(shots, kCntThreads, 152 * 4), kCntThreads, 0, st>>>(
        obs_true, obs_pred, flags, shots, n_types, ctr);
    return cudaGetLastError();
}

}  // namespace bp4m
