// Decoding with 16-bit message storage (IEEE half or bfloat16): the shared-memory kernel and
// the streaming kernel with MS = __half / __nv_bfloat16 and FP32 priors and arithmetic.
// Same tiers as FP32; shots above the widest streaming variant (1024 columns) use the FP32
// general global-memory kernel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "decode_smem.cuh"
#include "decode_stream.cuh"
#include "device.cuh"

namespace bp4m {
namespace {

template <typename MS>
cudaError_t dispatch_half(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep) {
    switch (tier) {
        case 1: return run_tier2<float, 32, 1, kReg32[1], MS>(a, num_sms, st, prep);
        case 2: return run_tier2<float, 32, 2, kReg32[2], MS>(a, num_sms, st, prep);
        case 3: return run_tier2<float, 24, 4, kReg32[3], MS>(a, num_sms, st, prep);
        case 4: return run_tier2<float, 28, 4, kReg32[4], MS>(a, num_sms, st, prep);
        // 128 rows: two blocks per SM without register-cached outputs (64 registers)
        case 5: return run_tier2<float, 32, 4, false, MS>(a, num_sms, st, prep);
        case 6: return run_tier2<float, 36, 4, kReg32[6], MS>(a, num_sms, st, prep);
        case 7: return run_tier2<float, 40, 4, kReg32[7], MS>(a, num_sms, st, prep);
        default: return cudaErrorInvalidValue;
    }
}

template <typename MS>
cudaError_t dispatch_stream_half(int ch, const DecodeArgs& a, int slots, cudaStream_t st) {
    switch (ch) {
        case 6: return run_stream<float, 6, MS>(a, slots, st);
        case 8: return run_stream<float, 8, MS>(a, slots, st);
        case 10: return run_stream<float, 10, MS>(a, slots, st);
        case 12: return run_stream<float, 12, MS>(a, slots, st);
        case 14: return run_stream<float, 14, MS>(a, slots, st);
        case 16: return run_stream<float, 16, MS>(a, slots, st);
        case 20: return run_stream<float, 20, MS>(a, slots, st);
        case 24: return run_stream<float, 24, MS>(a, slots, st);
        case 28: return run_stream<float, 28, MS>(a, slots, st);
        case 32: return run_stream<float, 32, MS>(a, slots, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_stream_half(int precision, int ch, const DecodeArgs& a, int slots, cudaStream_t st) {
    if (precision == 2) return dispatch_stream_half<__half>(ch, a, slots, st);
    if (precision == 3) return dispatch_stream_half<__nv_bfloat16>(ch, a, slots, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_decode_tier_half(int precision, int tier, const DecodeArgs& a, int num_sms, cudaStream_t st,
                                    bool prepare_only) {
    if (precision == 2) return dispatch_half<__half>(tier, a, num_sms, st, prepare_only);
    if (precision == 3) return dispatch_half<__nv_bfloat16>(tier, a, num_sms, st, prepare_only);
    return cudaErrorInvalidValue;
}

}  // namespace bp4m
