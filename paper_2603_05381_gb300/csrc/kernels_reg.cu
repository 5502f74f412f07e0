// Register-tile form of the FP32 shared-memory tiers of 128 and 144 rows (decode_reg.cuh):
// messages in registers, thread u holding a block pair of the message matrix and its mirror.
#include <cuda_runtime.h>

#include "decode_reg.cuh"
#include "device.cuh"

namespace bp4m {

bool reg_tier_available(int tier) { return tier == 5 || tier == 6; }

cudaError_t launch_decode_tier_reg(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prepare_only) {
    switch (tier) {
        case 5: return run_reg_tier2<32, 4>(a, num_sms, st, prepare_only);  // 128 rows, 544 threads
        case 6: return run_reg_tier2<24, 6>(a, num_sms, st, prepare_only);  // 144 rows, 320 threads
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bp4m
