// Cluster form of the streaming tier: instantiations for FP32 messages and the choice of the
// cluster size (kernels_cluster_half.cu holds the 16-bit message instantiations).
#include "decode_stream.cuh"

namespace bp4m {

namespace {

// Cluster sizes instantiated for FP32 messages, per width (CH columns per lane): two per
// width, so that the size can be chosen by measurement.
constexpr bool cl_f32(int ch, int cl) {
    return ch <= 8 ? (cl == 2 || cl == 4) : ch <= 12 ? (cl == 4 || cl == 8) : (cl == 8 || cl == 16);
}

template <int CH, int CL>
cudaError_t launch_f32(const DecodeArgs& a, int slots, cudaStream_t st) {
    if constexpr (cl_f32(CH, CL))
        return run_stream_cluster<float, CH, float, CL>(a, slots, st);
    else
        return cudaErrorInvalidValue;
}

template <int CH, int CL>
int capacity_f32() {
    if constexpr (cl_f32(CH, CL))
        return stream_cluster_capacity<float, CH, float, CL>();
    else
        return 0;
}

template <int CH>
cudaError_t launch_f32_cl(int cl, const DecodeArgs& a, int slots, cudaStream_t st) {
    switch (cl) {
        case 2: return launch_f32<CH, 2>(a, slots, st);
        case 4: return launch_f32<CH, 4>(a, slots, st);
        case 8: return launch_f32<CH, 8>(a, slots, st);
        case 16: return launch_f32<CH, 16>(a, slots, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int CH>
int capacity_f32_cl(int cl) {
    switch (cl) {
        case 2: return capacity_f32<CH, 2>();
        case 4: return capacity_f32<CH, 4>();
        case 8: return capacity_f32<CH, 8>();
        case 16: return capacity_f32<CH, 16>();
        default: return 0;
    }
}

}  // namespace

int stream_cluster_default(int ch) {
    // Slots of all clusters in flight (16 B per element and LD^2 elements each in FP32) of
    // at most ~90 MB, so that they stay in the 126 MB L2 beside the other data.
    return ch <= 10 ? 4 : ch <= 14 ? 8 : 16;
}

bool stream_cluster_instantiated(int precision, int ch, int cl) {
    if (precision == 1) return cl_f32(ch, cl);
    if (precision == 2 || precision == 3) return cl == stream_cluster_default(ch);
    return false;
}

int stream_cluster_capacity_of(int precision, int ch, int cl) {
    if (!stream_cluster_instantiated(precision, ch, cl)) return 0;
    if (precision != 1) return stream_cluster_capacity_half(precision, ch, cl);
    switch (ch) {
        case 6: return capacity_f32_cl<6>(cl);
        case 8: return capacity_f32_cl<8>(cl);
        case 10: return capacity_f32_cl<10>(cl);
        case 12: return capacity_f32_cl<12>(cl);
        case 14: return capacity_f32_cl<14>(cl);
        case 16: return capacity_f32_cl<16>(cl);
        case 20: return capacity_f32_cl<20>(cl);
        case 24: return capacity_f32_cl<24>(cl);
        case 28: return capacity_f32_cl<28>(cl);
        case 32: return capacity_f32_cl<32>(cl);
        default: return 0;
    }
}

int stream_cluster_size(int precision, int ch, int requested) {
    if (precision == 0 || requested == 1) return 1;
    const int def = stream_cluster_default(ch);
    const int want = requested > 1 ? requested : def;
    const int cands[3] = {want, def, def / 2};
    for (int cl : cands)
        if (cl > 1 && stream_cluster_capacity_of(precision, ch, cl) > 0) return cl;
    return 1;
}

cudaError_t launch_stream_cluster(int precision, int ch, int cl, const DecodeArgs& a, int slots, cudaStream_t st) {
    if (precision != 1) return launch_stream_cluster_half(precision, ch, cl, a, slots, st);
    switch (ch) {
        case 6: return launch_f32_cl<6>(cl, a, slots, st);
        case 8: return launch_f32_cl<8>(cl, a, slots, st);
        case 10: return launch_f32_cl<10>(cl, a, slots, st);
        case 12: return launch_f32_cl<12>(cl, a, slots, st);
        case 14: return launch_f32_cl<14>(cl, a, slots, st);
        case 16: return launch_f32_cl<16>(cl, a, slots, st);
        case 20: return launch_f32_cl<20>(cl, a, slots, st);
        case 24: return launch_f32_cl<24>(cl, a, slots, st);
        case 28: return launch_f32_cl<28>(cl, a, slots, st);
        case 32: return launch_f32_cl<32>(cl, a, slots, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bp4m
