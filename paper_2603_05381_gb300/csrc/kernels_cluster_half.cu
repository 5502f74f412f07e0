// Cluster form of the streaming tier with 16-bit message storage (precision 2 = IEEE half,
// 3 = bfloat16): one cluster size per width, the default of stream_cluster_default().
#include "decode_stream.cuh"

namespace bp4m {

namespace {

constexpr int cl_half(int ch) { return ch <= 10 ? 4 : ch <= 14 ? 8 : 16; }

template <typename MS, int CH>
cudaError_t launch_h(int cl, const DecodeArgs& a, int slots, cudaStream_t st) {
    if (cl != cl_half(CH)) return cudaErrorInvalidValue;
    return run_stream_cluster<float, CH, MS, cl_half(CH)>(a, slots, st);
}

template <typename MS, int CH>
int capacity_h(int cl) {
    if (cl != cl_half(CH)) return 0;
    return stream_cluster_capacity<float, CH, MS, cl_half(CH)>();
}

template <typename MS>
cudaError_t launch_ms(int ch, int cl, const DecodeArgs& a, int slots, cudaStream_t st) {
    switch (ch) {
        case 6: return launch_h<MS, 6>(cl, a, slots, st);
        case 8: return launch_h<MS, 8>(cl, a, slots, st);
        case 10: return launch_h<MS, 10>(cl, a, slots, st);
        case 12: return launch_h<MS, 12>(cl, a, slots, st);
        case 14: return launch_h<MS, 14>(cl, a, slots, st);
        case 16: return launch_h<MS, 16>(cl, a, slots, st);
        case 20: return launch_h<MS, 20>(cl, a, slots, st);
        case 24: return launch_h<MS, 24>(cl, a, slots, st);
        case 28: return launch_h<MS, 28>(cl, a, slots, st);
        case 32: return launch_h<MS, 32>(cl, a, slots, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename MS>
int capacity_ms(int ch, int cl) {
    switch (ch) {
        case 6: return capacity_h<MS, 6>(cl);
        case 8: return capacity_h<MS, 8>(cl);
        case 10: return capacity_h<MS, 10>(cl);
        case 12: return capacity_h<MS, 12>(cl);
        case 14: return capacity_h<MS, 14>(cl);
        case 16: return capacity_h<MS, 16>(cl);
        case 20: return capacity_h<MS, 20>(cl);
        case 24: return capacity_h<MS, 24>(cl);
        case 28: return capacity_h<MS, 28>(cl);
        case 32: return capacity_h<MS, 32>(cl);
        default: return 0;
    }
}

}  // namespace

int stream_cluster_capacity_half(int precision, int ch, int cl) {
    if (precision == 2) return capacity_ms<__half>(ch, cl);
    if (precision == 3) return capacity_ms<__nv_bfloat16>(ch, cl);
    return 0;
}

cudaError_t launch_stream_cluster_half(int precision, int ch, int cl, const DecodeArgs& a, int slots,
                                       cudaStream_t st) {
    if (precision == 2) return launch_ms<__half>(ch, cl, a, slots, st);
    if (precision == 3) return launch_ms<__nv_bfloat16>(ch, cl, a, slots, st);
    return cudaErrorInvalidValue;
}

}  // namespace bp4m
