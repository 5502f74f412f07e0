// First stage of B-BP4MF (Sec. "Belief-BP4MF (B-BP4MF)", Sec. "Correlated decoding"):
// quaternary BP on the code's Tanner graph under code-capacity depolarizing noise.
//
// Qubit v: prior p(I) = 1 - p, p(X) = p(Y) = p(Z) = p/3.  <E, c> = 1 iff Pauli E
// anticommutes with check c (X-checks see Z and Y, Z-checks see X and Y), z_c = syndrome.
// One scalar message per Tanner edge, flooding schedule, Delta = 0 before iteration 1:
//   qubit -> check  mu_vc    = ln( sum_{<E,c>=0} q(E) / sum_{<E,c>=1} q(E) ),
//                    q(E)     = p(E) prod_{c' != c} exp(-<E,c'> Delta_c'v)
//   check -> qubit  Delta_cv = (-1)^z_c 2 atanh( prod_{v' != v} tanh(mu_v'c / 2) )
//   posterior q_v(E) = p(E) prod_c exp(-<E,c> Delta_cv), decision argmax (ties I, X, Y, Z)
// A shot converges at the first iteration whose decision reproduces the syndrome; its
// output is the decision's observable flips.  Otherwise the per-qubit posteriors of an X
// component (X or Y) and of a Z component (Z or Y) go to the second stage.
#include <cuda_runtime.h>

#include <cmath>

#include "device.cuh"

namespace bp4m {
namespace {

constexpr int kQbpThreads = 256;

// anticommutation of I, X, Y, Z with an X-type (bit 0 of the mask) or Z-type check
__device__ __forceinline__ int anti(bool xcheck, int E) {
    return xcheck ? (E == 2 || E == 3) : (E == 1 || E == 2);
}

template <typename T>
__device__ __forceinline__ T lse2(T a, T b) {
    const T m = a > b ? a : b;
    if (m == -INFINITY) return m;
    return m + log(exp(a - m) + exp(b - m));
}

template <typename T>
__global__ void __launch_bounds__(kQbpThreads) qbp_kernel(QbpArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nc = a.n_checks, n = a.n_qubits;
    T* mu = reinterpret_cast<T*>(smem);             // [nc][4]
    T* dl = mu + 4 * nc;                            // [nc][4]
    unsigned char* zc = reinterpret_cast<unsigned char*>(dl + 4 * nc);  // [nc]
    unsigned char* dec = zc + nc;                   // [n]
    const T p = (T)a.p;
    const T lp[4] = {log(T(1) - p), log(p / T(3)), log(p / T(3)), log(p / T(3))};
    const T clampv = (T)a.clamp;
    const int tid = threadIdx.x;
    const int nw0 = a.n_words[0], nw1 = a.n_words[1];
    for (int64_t shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
        // X-checks are the detectors of type 1, Z-checks those of type 0
        const uint32_t* s1 = a.synd1 + (size_t)shot * nw1;
        const uint32_t* s0 = a.synd0 + (size_t)shot * nw0;
        for (int c = tid; c < nc; c += kQbpThreads) {
            const int d = c < a.n_xchecks ? c : c - a.n_xchecks;
            const uint32_t* w = c < a.n_xchecks ? s1 : s0;
            zc[c] = (w[d >> 5] >> (d & 31)) & 1u;
        }
        for (int e = tid; e < 4 * nc; e += kQbpThreads) dl[e] = T(0);
        __syncthreads();
        int conv = 0, it = 0;
        for (it = 1; it <= a.T; ++it) {
            // qubit -> check
            for (int e = tid; e < 4 * nc; e += kQbpThreads) {
                const int c = e >> 2;
                const int v = a.chk_q[e];
                if (v < 0) continue;
                T lq[4] = {lp[0], lp[1], lp[2], lp[3]};
                for (int j = 0; j < 4; ++j) {
                    const int e2 = a.q_edge[v * 4 + j];
                    if (e2 < 0 || e2 == e) continue;
                    const bool xc = (e2 >> 2) < a.n_xchecks;
                    const T dv = dl[e2];
                    for (int E = 1; E < 4; ++E)
                        if (anti(xc, E)) lq[E] -= dv;
                }
                const bool xc = c < a.n_xchecks;
                // commuting: I and (X for an X-check, Z for a Z-check); anticommuting: the rest
                const T num = lse2(lq[0], xc ? lq[1] : lq[3]);
                const T den = lse2(lq[2], xc ? lq[3] : lq[1]);
                mu[e] = num - den;
            }
            __syncthreads();
            // check -> qubit
            for (int e = tid; e < 4 * nc; e += kQbpThreads) {
                const int c = e >> 2, j0 = e & 3;
                if (a.chk_q[e] < 0) continue;
                T prod = T(1);
                for (int j = 0; j < 4; ++j)
                    if (j != j0 && a.chk_q[c * 4 + j] >= 0) prod *= tanh(mu[c * 4 + j] * T(0.5));
                prod = prod > T(1) - clampv ? T(1) - clampv : (prod < clampv - T(1) ? clampv - T(1) : prod);
                dl[e] = (zc[c] ? T(-2) : T(2)) * atanh(prod);
            }
            __syncthreads();
            // posterior and decision
            for (int v = tid; v < n; v += kQbpThreads) {
                T lq[4] = {lp[0], lp[1], lp[2], lp[3]};
                for (int j = 0; j < 4; ++j) {
                    const int e2 = a.q_edge[v * 4 + j];
                    if (e2 < 0) continue;
                    const bool xc = (e2 >> 2) < a.n_xchecks;
                    for (int E = 1; E < 4; ++E)
                        if (anti(xc, E)) lq[E] -= dl[e2];
                }
                int best = 0;
                for (int E = 1; E < 4; ++E)
                    if (lq[E] > lq[best]) best = E;
                dec[v] = (unsigned char)best;
            }
            __syncthreads();
            int ok = 1;
            for (int c = tid; c < nc; c += kQbpThreads) {
                const bool xc = c < a.n_xchecks;
                int par = 0;
                for (int j = 0; j < 4; ++j) {
                    const int v = a.chk_q[c * 4 + j];
                    if (v >= 0) par ^= anti(xc, dec[v]);
                }
                ok &= par == zc[c];
            }
            conv = __syncthreads_and(ok);
            if (conv) break;
        }
        if (conv) {
            int p0 = 0, p1 = 0;
            for (int v = tid; v < n; v += kQbpThreads) {
                const int E = dec[v];
                if ((E == 1 || E == 2) && a.in_zl[v]) p0 ^= 1;
                if ((E == 2 || E == 3) && a.in_xl[v]) p1 ^= 1;
            }
            const int o0 = __syncthreads_count(p0) & 1;
            const int o1 = __syncthreads_count(p1) & 1;
            if (tid == 0) {
                a.qconv[shot] = 1;
                a.qobs[shot] = (uint8_t)o0;
                a.qobs[a.shots + shot] = (uint8_t)o1;
                a.qiters[shot] = (int16_t)it;
            }
        } else {
            for (int v = tid; v < n; v += kQbpThreads) {
                T lq[4] = {lp[0], lp[1], lp[2], lp[3]};
                for (int j = 0; j < 4; ++j) {
                    const int e2 = a.q_edge[v * 4 + j];
                    if (e2 < 0) continue;
                    const bool xc = (e2 >> 2) < a.n_xchecks;
                    for (int E = 1; E < 4; ++E)
                        if (anti(xc, E)) lq[E] -= dl[e2];
                }
                T m = lq[0];
                for (int E = 1; E < 4; ++E) m = lq[E] > m ? lq[E] : m;
                T q[4], tot = T(0);
                for (int E = 0; E < 4; ++E) {
                    q[E] = exp(lq[E] - m);
                    tot += q[E];
                }
                a.post[(size_t)shot * n + v] = (double)((q[1] + q[2]) / tot);
                a.post[(size_t)(a.shots + shot) * n + v] = (double)((q[2] + q[3]) / tot);
            }
            if (tid == 0) {
                a.qconv[shot] = 0;
                a.qiters[shot] = (int16_t)a.T;
            }
        }
        __syncthreads();
    }
}

// Second-stage preparation.  The paper does not say how an edge whose posterior P exceeds
// 1/2 (weight ln((1-P)/P) < 0, no shortest paths) enters Dijkstra's algorithm; as matching
// decoders with negative weights do, such an edge is taken as present: its endpoints flip in
// a copy of the syndrome, its observable bit goes into a base parity added to the decoded
// one, and it enters the graph with probability 1 - P.  One warp per (type, shot).
constexpr int kFlipWarps = 8;

__global__ void __launch_bounds__(kFlipWarps * 32) rw_flip_kernel(RwFlipArgs a, int max_words) {
    extern __shared__ uint32_t fw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* my = fw + warp * max_words;
    for (int64_t item = (int64_t)blockIdx.x * kFlipWarps + warp; item < 2 * a.shots;
         item += (int64_t)gridDim.x * kFlipWarps) {
        const int ty = item >= a.shots ? 1 : 0;
        const int64_t shot = item - (ty ? a.shots : 0);
        const int nw = a.n_words[ty], nd = a.n_det[ty];
        const uint32_t* src = a.synd[ty] + (size_t)shot * nw;
        for (int w = lane; w < nw; w += 32) my[w] = src[w];
        __syncwarp();
        const double* post = a.post + ((size_t)ty * a.shots + shot) * a.n_units;
        const uint32_t* uvo = a.cc_uvo + (size_t)ty * a.n_units;
        unsigned ob = 0;
        for (int q = lane; q < a.n_units; q += 32) {
            if (post[q] > 0.5) {
                const uint32_t pk = __ldg(uvo + q);
                const int u = (int)(pk & 0x7FFFu), v = (int)((pk >> 15) & 0x7FFFu);
                atomicXor(my + (u >> 5), 1u << (u & 31));
                if (v < nd) atomicXor(my + (v >> 5), 1u << (v & 31));
                ob ^= pk >> 31;
            }
        }
        ob = __reduce_xor_sync(0xffffffffu, ob);
        __syncwarp();
        uint32_t* dst = a.out[ty] + (size_t)shot * nw;
        for (int w = lane; w < nw; w += 32) dst[w] = my[w];
        if (lane == 0) a.base[(size_t)ty * a.shots + shot] = (uint8_t)(ob & 1u);
        __syncwarp();
    }
}

__global__ void rw_base_kernel(uint8_t* obs_pred, const uint8_t* skip, const uint8_t* base, int64_t shots) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 2 * shots; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t shot = k < shots ? k : k - shots;
        if (!skip[shot]) obs_pred[k] ^= base[k];
    }
}

}  // namespace

cudaError_t launch_rw_flip(const RwFlipArgs& a, int num_sms, cudaStream_t st) {
    if (a.shots <= 0) return cudaSuccess;
    const int max_words = a.n_words[0] > a.n_words[1] ? a.n_words[0] : a.n_words[1];
    const size_t smem = (size_t)kFlipWarps * max_words * sizeof(uint32_t);
    if (smem > 48 * 1024) return cudaErrorInvalidValue;
    int64_t g = (2 * a.shots + kFlipWarps - 1) / kFlipWarps;
    if (g > (int64_t)num_sms * 16) g = (int64_t)num_sms * 16;
    rw_flip_kernel<<<(int)g, kFlipWarps * 32, smem, st>>>(a, max_words);
    return cudaGetLastError();
}

cudaError_t launch_rw_base(uint8_t* obs_pred, const uint8_t* skip, const uint8_t* base, int64_t shots,
                           cudaStream_t st) {
    if (shots <= 0) return cudaSuccess;
    int64_t g = (2 * shots + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    rw_base_kernel<<<(int)g, 256, 0, st>>>(obs_pred, skip, base, shots);
    return cudaGetLastError();
}

cudaError_t launch_qbp(int precision, const QbpArgs& a, int num_sms, cudaStream_t st) {
    if (a.shots <= 0) return cudaSuccess;
    const size_t esz = precision == 0 ? sizeof(double) : sizeof(float);
    const size_t smem = 8 * (size_t)a.n_checks * esz + a.n_checks + a.n_qubits + 16;
    int grid = (int)(a.shots < (int64_t)num_sms * 8 ? a.shots : (int64_t)num_sms * 8);
    if (precision == 0)
        qbp_kernel<double><<<grid, kQbpThreads, smem, st>>>(a);
    else
        qbp_kernel<float><<<grid, kQbpThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace bp4m
