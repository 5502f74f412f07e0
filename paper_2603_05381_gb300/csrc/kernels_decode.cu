// BP4M / BP4MF decoding of one shot per thread block.
//
// Per shot with s unsatisfied detectors (Sec. "Bipartite Graph Representation"): factor c_i
// per detector, variable v_ij per pair and v_ii to the boundary; prior LLR l_ij gathered
// from the per-graph table.  Log-domain sum-product with the flooding schedule (Sec.
// "Belief Propagation"):
//   Q[i][k]  = l_ik + M[k][i] / alpha (k != i),  Q[i][i] = l_ii
//   M'[i][j] = -max*_{k != j} Q[i][k],           max*(x) = ln sum exp(x)
//   lambda_ij = l_ij + (M'[i][j] + M'[j][i]),    lambda_ii = l_ii + M'[i][i]
// The leave-one-out max* of a row uses its largest entry m1 (at k = a), second largest m2
// and S = sum_{k != a} exp(Q_k - m2) >= 1:
//   j == a:  max*_{k != a} = m2 + ln S
//   j != a:  max*_{k != j} = m1 + ln(1 + exp(m2 - m1) (S - exp(Q_j - m2)))
// which is exact algebra, has no cancellation beyond S - exp(Q_j - m2) >= 0, and costs one
// exp and one log per message.  Marginalization keeps v iff lambda_v > 0; convergence =
// every factor keeps exactly one variable (Sec. "Checking convergence").  Forced
// convergence (Sec. "Forced convergence") is the greedy matching in the order
// (lambda desc, i asc, j asc); it is computed here by rounds of locally dominant
// choices (a variable that is the best remaining one at both of its factors is accepted),
// which yields exactly the same matching as the sequential greedy scan.
//
// Layout (shared-memory tiers): Mt[i][k] = M[k][i], the message arriving at factor i from
// the factor k side; Lm[i][k] = l_ik.  Row i is processed by G threads, thread g taking
// columns k = g + G*c.  The update is in place: every thread caches its row in registers,
// the block synchronises, then each thread writes its outputs M'[i][k] into Mt[k][i].
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "device.cuh"

namespace bp4m {
namespace {

template <typename T>
struct Num;

template <>
struct Num<float> {
    static __device__ __forceinline__ float ninf() { return __int_as_float(0xff800000); }
    static __device__ __forceinline__ float pinf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float lg(float x) { return __logf(x); }
    static __device__ __forceinline__ float lg1p(float x) { return __logf(1.0f + x); }
    static __device__ __forceinline__ const float* L(const DevTables& t) { return t.L32; }
};

template <>
struct Num<double> {
    static __device__ __forceinline__ double ninf() { return __longlong_as_double(0xfff0000000000000ull); }
    static __device__ __forceinline__ double pinf() { return __longlong_as_double(0x7ff0000000000000ull); }
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double lg(double x) { return log(x); }
    static __device__ __forceinline__ double lg1p(double x) { return log1p(x); }
    static __device__ __forceinline__ const double* L(const DevTables& t) { return t.L64; }
};

constexpr unsigned kFull = 0xffffffffu;

// Warp 0 turns the shot's bit-packed syndrome into the sorted detector list.
__device__ __forceinline__ int compact_defects(const uint32_t* __restrict__ sw, int nw, int* dets,
                                               int cap, int lane) {
    int base = 0;
    for (int w0 = 0; w0 < nw; w0 += 32) {
        uint32_t word = (w0 + lane < nw) ? __ldg(sw + w0 + lane) : 0u;
        const int c = __popc(word);
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += y;
        }
        int pos = base + incl - c;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            if (pos < cap) dets[pos] = (w0 + lane) * 32 + b;
            ++pos;
        }
        base += __shfl_sync(kFull, incl, 31);
    }
    return base;
}

// Blocks per SM requested from the compiler: enough to keep registers at or below 128.
constexpr int min_blocks(int nt) { return 65536 / (nt * 128) > 1 ? 65536 / (nt * 128) : 1; }

template <typename T, int CH, int G, bool REG_OUT>
__global__ void __launch_bounds__(CH * G * G, min_blocks(CH * G * G)) decode_smem_kernel(const DecodeArgs a) {
    constexpr int SMAX = CH * G;
    constexpr int NT = SMAX * G;
    constexpr int R = 32 / G;
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    extern __shared__ __align__(16) unsigned char smem[];
    const int pitch = a.pitch;
    T* Mt = reinterpret_cast<T*>(smem);
    T* Lm = Mt + (size_t)SMAX * pitch;
    double* rowacc = reinterpret_cast<double*>(Lm + (size_t)SMAX * pitch);
    int* dets = reinterpret_cast<int*>(rowacc + SMAX);
    int* choice = dets + SMAX;
    short* bestp = reinterpret_cast<short*>(choice + SMAX);
    unsigned char* matched = reinterpret_cast<unsigned char*>(bestp + SMAX);
    __shared__ int sh_item, sh_s, sh_best_par, sh_best_forced, sh_improve, sh_use_best;
    __shared__ double sh_best_w;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i = warp * R + (lane % R);
    const int g = lane / R;
    const int n = a.tb.n_det;
    const T* __restrict__ Ltab = Num<T>::L(a.tb);
    const int count = *a.count;
    const bool plain = a.alpha == 1.0;
    const T ainv = (T)(1.0 / a.alpha);
    const bool full = (a.decoder == 1) || !a.early_exit;
    const bool want_w = full;
    T* trl = reinterpret_cast<T*>(a.tr_lambda);
    unsigned long long acc_it = 0, acc_msg = 0, acc_def = 0;

    for (;;) {
        if (tid == 0) sh_item = atomicAdd(a.next, 1);
        __syncthreads();
        const int item = sh_item;
        if (item >= count) break;
        const int64_t shot = a.list[item];
        if (warp == 0) {
            const int s0 = compact_defects(a.synd + (size_t)shot * a.tb.n_words, a.tb.n_words,
                                           dets, SMAX, lane);
            if (lane == 0) sh_s = s0;
        }
        __syncthreads();
        const int s = sh_s;
        if (s > SMAX || s < 1) {
            if (tid == 0 && a.ctr) atomicAdd(a.ctr + C_ERRORS, 1ull);
            continue;
        }
        const bool tr_on = (trl != nullptr || a.tr_partner != nullptr) && s <= a.s_cap;
        if (s == 1) {
            // a single factor with a single variable: the leave-one-out set is empty, the
            // message is +inf and v_00 is kept at iteration 1
            if (tid == 0) {
                const int d0 = dets[0];
                if (a.obs_pred) a.obs_pred[shot] = a.tb.P[(size_t)d0 * n + d0];
                if (a.flags) a.flags[shot] = F_CONVERGED;
                if (a.iters) a.iters[shot] = 1;
                if (tr_on && trl) trl[(size_t)shot * a.s_cap * a.s_cap] = Num<T>::pinf();
                if (tr_on && a.tr_partner) {
                    a.tr_partner[(size_t)shot * a.s_cap] = 0;
                    for (int k = 1; k < a.s_cap; ++k) a.tr_partner[(size_t)shot * a.s_cap + k] = -1;
                }
                acc_it += 1;
                acc_msg += 1;
                acc_def += 1;
            }
            continue;
        }
        for (int r = warp; r < s; r += NT / 32) {
            const T* trow = Ltab + (size_t)dets[r] * n;
            for (int k = lane; k < s; k += 32) {
                Lm[r * pitch + k] = __ldg(trow + dets[k]);
                Mt[r * pitch + k] = T(0);
            }
        }
        if (tid < SMAX) {
            matched[tid] = 0;
            bestp[tid] = -1;
        }
        if (tid == 0) {
            sh_best_w = Num<double>::pinf();
            sh_best_par = 0;
            sh_best_forced = 0;
            sh_use_best = 0;
        }
        __syncthreads();

        const bool act = i < s;
        const int rowbase = i * pitch;
        T q[CH];
        T mo[REG_OUT ? CH : 1];
        int t = 0;
        bool any_conv = false, forced_ran = false;
        int out_par = 0, out_forced = 0, out_from_best = 0;
        int partner = -1;  // the output candidate's partner of row i (g == 0 lanes)

        for (;;) {
            // ---- read phase: Q for the next update and, for t > 0, lambda^t decisions
            int cnt = 0, chosen = -1;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int k = g + G * c;
                T qv = Num<T>::ninf();
                if (act && k < s) {
                    const T l = Lm[rowbase + k];
                    const T x = Mt[rowbase + k];
                    qv = (k == i) ? l : (plain ? l + x : l + x * ainv);
                    if (t > 0) {
                        const T own = REG_OUT ? mo[c] : Mt[k * pitch + i];
                        const T lam = (k == i) ? l + own : l + (own + x);
                        if (lam > T(0)) {
                            ++cnt;
                            chosen = k;
                        }
                        if (tr_on && trl) trl[((size_t)shot * a.s_cap + i) * a.s_cap + k] = lam;
                    }
                }
                q[c] = qv;
            }
#pragma unroll
            for (int off = R; off < 32; off <<= 1) {
                cnt += __shfl_xor_sync(kFull, cnt, off);
                chosen = max(chosen, __shfl_xor_sync(kFull, chosen, off));
            }
            const int conv = __syncthreads_and(t > 0 && (!act || cnt == 1));

            if (t > 0) {
                bool have_cand = false, cand_forced = false;
                int cand_p = -1;
                if (conv) {
                    any_conv = true;
                    have_cand = true;
                    cand_p = chosen;
                } else if (a.decoder == 1 || t == a.T) {
                    // ---- forced convergence on lambda^t by locally dominant rounds
                    forced_ran = true;
                    if (act && g == 0) matched[i] = 0;
                    __syncthreads();
                    for (int round = 0; round < s; ++round) {
                        const bool open = act && !matched[i];
                        T bl = Num<T>::ninf();
                        int bk = -1;
                        if (open) {
#pragma unroll
                            for (int c = 0; c < CH; ++c) {
                                const int k = g + G * c;
                                if (k < s && (k == i || !matched[k])) {
                                    const T l = Lm[rowbase + k];
                                    const T x = Mt[rowbase + k];
                                    const T own = REG_OUT ? mo[c] : Mt[k * pitch + i];
                                    const T lam = (k == i) ? l + own : l + (own + x);
                                    if (bk < 0 || lam > bl) {
                                        bl = lam;
                                        bk = k;
                                    }
                                }
                            }
                        }
#pragma unroll
                        for (int off = R; off < 32; off <<= 1) {
                            const T ol = __shfl_xor_sync(kFull, bl, off);
                            const int ok = __shfl_xor_sync(kFull, bk, off);
                            if (ok >= 0 && (bk < 0 || ol > bl || (ol == bl && ok < bk))) {
                                bl = ol;
                                bk = ok;
                            }
                        }
                        if (open && g == 0) choice[i] = bk >= 0 ? bk : i;
                        __syncthreads();
                        bool newm = false;
                        if (open && g == 0) {
                            const int pk = choice[i];
                            newm = (pk == i) || (choice[pk] == i);
                        }
                        __syncthreads();
                        if (newm) matched[i] = 1;
                        const int left = __syncthreads_count(open && g == 0 && !newm);
                        if (left == 0) break;
                    }
                    have_cand = true;
                    cand_forced = true;
                    if (act && g == 0) cand_p = choice[i];
                }
                if (have_cand) {
                    // ---- candidate parity (and weight when candidates are compared)
                    int pc = 0;
                    if (act && g == 0) {
                        const int k = cand_p;
                        double w = 0.0;
                        if (k >= i) {
                            const size_t off = (size_t)dets[i] * n + dets[k];
                            pc = a.tb.P[off];
                            if (want_w) w = a.tb.W64[off];
                        }
                        rowacc[i] = w;
                    }
                    const int par = __syncthreads_count(pc) & 1;
                    bool finish = false;
                    if (!full) {
                        // BP4M early exit: first converged iteration, or forced at T
                        out_par = par;
                        out_forced = cand_forced;
                        partner = cand_p;
                        finish = true;
                    } else {
                        if (tid == 0) {
                            double w = 0.0;
                            for (int r = 0; r < s; ++r) w += rowacc[r];
                            sh_improve = 0;
                            sh_use_best = 0;
                            if (a.decoder == 1 || !cand_forced) {
                                if (w < sh_best_w) {
                                    sh_best_w = w;
                                    sh_best_par = par;
                                    sh_best_forced = cand_forced;
                                    sh_improve = 1;
                                }
                            } else {
                                // BP4M full-T: forced candidate of iteration T against the
                                // lightest converged one (ties: the converged one)
                                sh_use_best = sh_best_w <= w;
                            }
                        }
                        __syncthreads();
                        if (sh_improve && act && g == 0) bestp[i] = (short)cand_p;
                        if (t == a.T || (a.decoder == 0 && cand_forced)) {
                            finish = true;
                            if (a.decoder == 0 && cand_forced && !sh_use_best) {
                                out_par = par;
                                out_forced = 1;
                                partner = cand_p;
                            } else {
                                out_par = sh_best_par;
                                out_forced = sh_best_forced;
                                out_from_best = 1;
                            }
                        }
                        __syncthreads();
                    }
                    if (finish) break;
                }
            }

            // ---- compute phase: leave-one-out max* of every row, written in place
            T m1 = Num<T>::ninf(), m2 = Num<T>::ninf();
            int am = 0x7fffffff;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int k = g + G * c;
                if (act && k < s) {
                    const T v = q[c];
                    if (v > m1) {
                        m2 = m1;
                        m1 = v;
                        am = k;
                    } else if (v > m2) {
                        m2 = v;
                    }
                }
            }
#pragma unroll
            for (int off = R; off < 32; off <<= 1) {
                const T o1 = __shfl_xor_sync(kFull, m1, off);
                const int oa = __shfl_xor_sync(kFull, am, off);
                const T o2 = __shfl_xor_sync(kFull, m2, off);
                if (o1 > m1 || (o1 == m1 && oa < am)) {
                    m2 = m1 > o2 ? m1 : o2;
                    m1 = o1;
                    am = oa;
                } else {
                    m2 = m2 > o1 ? m2 : o1;
                }
            }
            T S = T(0);
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const int k = g + G * c;
                if (act && k < s && k != am) {
                    const T u = Num<T>::ex(q[c] - m2);
                    q[c] = u;
                    S += u;
                }
            }
#pragma unroll
            for (int off = R; off < 32; off <<= 1) S += __shfl_xor_sync(kFull, S, off);
            if (act) {
                const T cf = Num<T>::ex(m2 - m1);
                const T lS = Num<T>::lg(S);
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    const int k = g + G * c;
                    if (k < s) {
                        const T out = (k == am) ? -(m2 + lS) : -(m1 + Num<T>::lg1p(cf * (S - q[c])));
                        Mt[k * pitch + i] = out;
                        if (REG_OUT) mo[c] = out;
                    }
                }
            }
            __syncthreads();
            ++t;
        }

        // ---- outputs of the shot
        if (tr_on && a.tr_partner) {
            if (act && g == 0) {
                const int pk = out_from_best ? (int)bestp[i] : partner;
                a.tr_partner[(size_t)shot * a.s_cap + i] = (int16_t)pk;
            }
            for (int k = s + tid; k < a.s_cap; k += NT) a.tr_partner[(size_t)shot * a.s_cap + k] = -1;
        }
        if (tid == 0) {
            if (a.obs_pred) a.obs_pred[shot] = (uint8_t)out_par;
            if (a.flags)
                a.flags[shot] = (uint8_t)((any_conv ? F_CONVERGED : 0) | (forced_ran ? F_FORCED_RAN : 0) |
                                          (out_forced ? F_FROM_FORCED : 0));
            if (a.iters) a.iters[shot] = (int16_t)t;
            acc_it += (unsigned long long)t;
            acc_msg += (unsigned long long)s * s * t;
            acc_def += (unsigned long long)s;
        }
        __syncthreads();
    }
    if (tid == 0 && a.ctr) {
        atomicAdd(a.ctr + C_ITERS, acc_it);
        atomicAdd(a.ctr + C_MSGS, acc_msg);
        atomicAdd(a.ctr + C_DEFECTS, acc_def);
    }
}

// ------------------------------------------------------------------ global-memory tier
//
// Same iteration as above for shots too large for shared memory.  Messages are double
// buffered in a per-block global scratch slot (Mt layout, leading dimension s) and every
// thread walks whole rows in three passes (max, sum, write).
constexpr int kGlobThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kGlobThreads) decode_global_kernel(const DecodeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int gsmax = a.gsmax;
    double* rowacc = reinterpret_cast<double*>(smem);
    int* dets = reinterpret_cast<int*>(rowacc + gsmax);
    int* choice = dets + gsmax;
    short* bestp = reinterpret_cast<short*>(choice + gsmax);
    unsigned char* matched = reinterpret_cast<unsigned char*>(bestp + gsmax);
    __shared__ int sh_item, sh_s, sh_best_par, sh_best_forced, sh_improve, sh_use_best;
    __shared__ double sh_best_w;
    T* slot = reinterpret_cast<T*>(a.gscratch) + (size_t)blockIdx.x * 3 * a.gslot_elems;
    T* Lg = slot;
    T* Ma = slot + a.gslot_elems;
    T* Mb = slot + 2 * a.gslot_elems;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = a.tb.n_det;
    const T* __restrict__ Ltab = Num<T>::L(a.tb);
    const int count = *a.count;
    const bool plain = a.alpha == 1.0;
    const T ainv = (T)(1.0 / a.alpha);
    const bool full = (a.decoder == 1) || !a.early_exit;
    T* trl = reinterpret_cast<T*>(a.tr_lambda);
    unsigned long long acc_it = 0, acc_msg = 0, acc_def = 0;

    for (;;) {
        if (tid == 0) sh_item = atomicAdd(a.next, 1);
        __syncthreads();
        const int item = sh_item;
        if (item >= count) break;
        const int64_t shot = a.list[item];
        if (warp == 0) {
            const int s0 = compact_defects(a.synd + (size_t)shot * a.tb.n_words, a.tb.n_words,
                                           dets, gsmax, lane);
            if (lane == 0) sh_s = s0;
        }
        __syncthreads();
        const int s = sh_s;
        if (s > gsmax || s < 2) {
            if (tid == 0 && a.ctr) atomicAdd(a.ctr + C_ERRORS, 1ull);
            continue;
        }
        const bool tr_on = (trl != nullptr || a.tr_partner != nullptr) && s <= a.s_cap;
        for (int r = warp; r < s; r += kGlobThreads / 32) {
            const T* trow = Ltab + (size_t)dets[r] * n;
            for (int k = lane; k < s; k += 32) {
                Lg[(size_t)r * s + k] = __ldg(trow + dets[k]);
                Ma[(size_t)r * s + k] = T(0);
            }
        }
        for (int r = tid; r < s; r += kGlobThreads) {
            matched[r] = 0;
            bestp[r] = -1;
        }
        if (tid == 0) {
            sh_best_w = Num<double>::pinf();
            sh_best_par = 0;
            sh_best_forced = 0;
            sh_use_best = 0;
        }
        __syncthreads();
        T* Mc = Ma;  // Mc[i][k] = M[k][i] of the current iteration
        T* Mn = Mb;
        int t = 0;
        bool any_conv = false, forced_ran = false;
        int out_par = 0, out_forced = 0, out_from_best = 0;

        for (;;) {
            if (t > 0) {
                // ---- decisions of lambda^t
                int ok_all = 1;
                for (int r = tid; r < s; r += kGlobThreads) {
                    int cnt = 0, chosen = -1;
                    for (int k = 0; k < s; ++k) {
                        const T l = Lg[(size_t)r * s + k];
                        const T own = Mc[(size_t)k * s + r];
                        const T lam = (k == r) ? l + own : l + (own + Mc[(size_t)r * s + k]);
                        if (lam > T(0)) {
                            ++cnt;
                            chosen = k;
                        }
                        if (tr_on && trl) trl[((size_t)shot * a.s_cap + r) * a.s_cap + k] = lam;
                    }
                    choice[r] = chosen;
                    ok_all &= (cnt == 1);
                }
                const int conv = __syncthreads_and(ok_all);
                bool have_cand = false, cand_forced = false;
                if (conv) {
                    any_conv = true;
                    have_cand = true;
                } else if (a.decoder == 1 || t == a.T) {
                    forced_ran = true;
                    for (int r = tid; r < s; r += kGlobThreads) matched[r] = 0;
                    __syncthreads();
                    for (int round = 0; round < s; ++round) {
                        for (int r = tid; r < s; r += kGlobThreads) {
                            if (matched[r]) continue;
                            T bl = Num<T>::ninf();
                            int bk = -1;
                            for (int k = 0; k < s; ++k) {
                                if (k != r && matched[k]) continue;
                                const T l = Lg[(size_t)r * s + k];
                                const T own = Mc[(size_t)k * s + r];
                                const T lam = (k == r) ? l + own : l + (own + Mc[(size_t)r * s + k]);
                                if (bk < 0 || lam > bl) {
                                    bl = lam;
                                    bk = k;
                                }
                            }
                            choice[r] = bk >= 0 ? bk : r;
                        }
                        __syncthreads();
                        int left = 0;
                        for (int r = tid; r < s; r += kGlobThreads) {
                            if (matched[r]) continue;
                            const int pk = choice[r];
                            const bool newm = (pk == r) || (choice[pk] == r);
                            // matched[] is only read in the search phase above
                            rowacc[r] = newm ? 1.0 : 0.0;
                            left += !newm;
                        }
                        __syncthreads();
                        for (int r = tid; r < s; r += kGlobThreads)
                            if (!matched[r] && rowacc[r] != 0.0) matched[r] = 1;
                        if (__syncthreads_count(left) == 0) break;
                    }
                    have_cand = true;
                    cand_forced = true;
                }
                if (have_cand) {
                    int pc = 0;
                    for (int r = tid; r < s; r += kGlobThreads) {
                        const int k = choice[r];
                        double w = 0.0;
                        if (k >= r) {
                            const size_t off = (size_t)dets[r] * n + dets[k];
                            pc ^= a.tb.P[off];
                            if (full) w = a.tb.W64[off];
                        }
                        rowacc[r] = w;
                    }
                    const int par = __syncthreads_count(pc) & 1;
                    bool finish = false;
                    if (!full) {
                        out_par = par;
                        out_forced = cand_forced;
                        finish = true;
                    } else {
                        if (tid == 0) {
                            double w = 0.0;
                            for (int r = 0; r < s; ++r) w += rowacc[r];
                            sh_improve = 0;
                            sh_use_best = 0;
                            if (a.decoder == 1 || !cand_forced) {
                                if (w < sh_best_w) {
                                    sh_best_w = w;
                                    sh_best_par = par;
                                    sh_best_forced = cand_forced;
                                    sh_improve = 1;
                                }
                            } else {
                                sh_use_best = sh_best_w <= w;
                            }
                        }
                        __syncthreads();
                        if (sh_improve)
                            for (int r = tid; r < s; r += kGlobThreads) bestp[r] = (short)choice[r];
                        if (t == a.T || (a.decoder == 0 && cand_forced)) {
                            finish = true;
                            if (a.decoder == 0 && cand_forced && !sh_use_best) {
                                out_par = par;
                                out_forced = 1;
                            } else {
                                out_par = sh_best_par;
                                out_forced = sh_best_forced;
                                out_from_best = 1;
                            }
                        }
                        __syncthreads();
                    }
                    if (finish) break;
                }
                __syncthreads();
            }
            // ---- factor update into the other buffer
            for (int r = tid; r < s; r += kGlobThreads) {
                const T* lrow = Lg + (size_t)r * s;
                const T* mrow = Mc + (size_t)r * s;
                T m1 = Num<T>::ninf(), m2 = Num<T>::ninf();
                int am = 0;
                for (int k = 0; k < s; ++k) {
                    const T v = (k == r) ? lrow[k] : (plain ? lrow[k] + mrow[k] : lrow[k] + mrow[k] * ainv);
                    if (v > m1) {
                        m2 = m1;
                        m1 = v;
                        am = k;
                    } else if (v > m2) {
                        m2 = v;
                    }
                }
                T S = T(0);
                for (int k = 0; k < s; ++k) {
                    if (k == am) continue;
                    const T v = (k == r) ? lrow[k] : (plain ? lrow[k] + mrow[k] : lrow[k] + mrow[k] * ainv);
                    S += Num<T>::ex(v - m2);
                }
                const T cf = Num<T>::ex(m2 - m1);
                const T lS = Num<T>::lg(S);
                for (int k = 0; k < s; ++k) {
                    T out;
                    if (k == am) {
                        out = -(m2 + lS);
                    } else {
                        const T v = (k == r) ? lrow[k] : (plain ? lrow[k] + mrow[k] : lrow[k] + mrow[k] * ainv);
                        out = -(m1 + Num<T>::lg1p(cf * (S - Num<T>::ex(v - m2))));
                    }
                    Mn[(size_t)k * s + r] = out;
                }
            }
            __syncthreads();
            T* tmp = Mc;
            Mc = Mn;
            Mn = tmp;
            ++t;
        }
        if (tr_on && a.tr_partner) {
            for (int r = tid; r < a.s_cap; r += kGlobThreads) {
                int pk = -1;
                if (r < s) pk = out_from_best ? (int)bestp[r] : choice[r];
                a.tr_partner[(size_t)shot * a.s_cap + r] = (int16_t)pk;
            }
        }
        if (tid == 0) {
            if (a.obs_pred) a.obs_pred[shot] = (uint8_t)out_par;
            if (a.flags)
                a.flags[shot] = (uint8_t)((any_conv ? F_CONVERGED : 0) | (forced_ran ? F_FORCED_RAN : 0) |
                                          (out_forced ? F_FROM_FORCED : 0));
            if (a.iters) a.iters[shot] = (int16_t)t;
            acc_it += (unsigned long long)t;
            acc_msg += (unsigned long long)s * s * t;
            acc_def += (unsigned long long)s;
        }
        __syncthreads();
    }
    if (tid == 0 && a.ctr) {
        atomicAdd(a.ctr + C_ITERS, acc_it);
        atomicAdd(a.ctr + C_MSGS, acc_msg);
        atomicAdd(a.ctr + C_DEFECTS, acc_def);
    }
}

// ------------------------------------------------------------------ tier table

struct TierCfg {
    int smax;
    int ch, g;
    bool reg_out;
};

// FP32: 32/64/128/160 rows in shared memory; FP64: 32/64/112.
constexpr TierCfg kCfg32[5] = {{0, 0, 0, false}, {32, 32, 1, true}, {64, 32, 2, true},
                               {128, 32, 4, true}, {160, 40, 4, false}};
constexpr TierCfg kCfg64[5] = {{0, 0, 0, false}, {32, 16, 2, false}, {64, 16, 4, false},
                               {112, 14, 8, false}, {112, 14, 8, false}};

int pitch_for(int smax, int g) {
    int p = smax;
    while (p % 32 != g % 32) ++p;
    return p;
}

template <typename T, int CH, int G, bool REG>
size_t smem_bytes_of(int* pitch) {
    constexpr int SMAX = CH * G;
    const int p = pitch_for(SMAX, G);
    if (pitch) *pitch = p;
    return (size_t)2 * SMAX * p * sizeof(T) + (size_t)SMAX * (sizeof(double) + 2 * sizeof(int) +
                                                              sizeof(short) + 1) + 16;
}

template <typename T, int CH, int G, bool REG>
cudaError_t run_tier(const DecodeArgs& a0, int num_sms, cudaStream_t st, bool prepare_only) {
    int pitch = 0;
    const size_t smem = smem_bytes_of<T, CH, G, REG>(&pitch);
    auto kern = decode_smem_kernel<T, CH, G, REG>;
    if (prepare_only)
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CH * G * G, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    DecodeArgs a = a0;
    a.pitch = pitch;
    kern<<<per_sm * num_sms, CH * G * G, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_tier(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep);

template <>
cudaError_t dispatch_tier<float>(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep) {
    switch (tier) {
        case 1: return run_tier<float, 32, 1, true>(a, num_sms, st, prep);
        case 2: return run_tier<float, 32, 2, true>(a, num_sms, st, prep);
        case 3: return run_tier<float, 32, 4, true>(a, num_sms, st, prep);
        case 4: return run_tier<float, 40, 4, false>(a, num_sms, st, prep);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t dispatch_tier<double>(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep) {
    switch (tier) {
        case 1: return run_tier<double, 16, 2, false>(a, num_sms, st, prep);
        case 2: return run_tier<double, 16, 4, false>(a, num_sms, st, prep);
        case 3: return run_tier<double, 14, 8, false>(a, num_sms, st, prep);
        case 4: return cudaSuccess;  // same bound as tier 3: never populated
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

TierPlan tier_plan(int precision) {
    TierPlan p{};
    const TierCfg* c = precision == 0 ? kCfg64 : kCfg32;
    for (int k = 0; k < kTiers; ++k) p.smax[k] = k < 5 ? c[k].smax : 0x7fffffff;
    p.smax[kGlobalTier] = 0x7fffffff;
    return p;
}

size_t tier_smem_bytes(int precision, int tier, int* pitch_out) {
    if (precision == 0) {
        switch (tier) {
            case 1: return smem_bytes_of<double, 16, 2, false>(pitch_out);
            case 2: return smem_bytes_of<double, 16, 4, false>(pitch_out);
            case 3: case 4: return smem_bytes_of<double, 14, 8, false>(pitch_out);
        }
    } else {
        switch (tier) {
            case 1: return smem_bytes_of<float, 32, 1, true>(pitch_out);
            case 2: return smem_bytes_of<float, 32, 2, true>(pitch_out);
            case 3: return smem_bytes_of<float, 32, 4, true>(pitch_out);
            case 4: return smem_bytes_of<float, 40, 4, false>(pitch_out);
        }
    }
    return 0;
}

cudaError_t prepare_decode_kernels(int precision) {
    DecodeArgs dummy;
    for (int tier = 1; tier <= 4; ++tier) {
        cudaError_t e = precision == 0 ? dispatch_tier<double>(tier, dummy, 0, 0, true)
                                       : dispatch_tier<float>(tier, dummy, 0, 0, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_decode_tier(int precision, int tier, const DecodeArgs& a, int num_sms,
                               cudaStream_t st) {
    return precision == 0 ? dispatch_tier<double>(tier, a, num_sms, st, false)
                          : dispatch_tier<float>(tier, a, num_sms, st, false);
}

cudaError_t launch_decode_global(int precision, const DecodeArgs& a, int slots, cudaStream_t st) {
    if (slots <= 0) return cudaSuccess;
    const size_t smem = (size_t)a.gsmax * (sizeof(double) + 2 * sizeof(int) + sizeof(short) + 1) + 16;
    cudaError_t e;
    if (precision == 0) {
        e = cudaFuncSetAttribute(decode_global_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        decode_global_kernel<double><<<slots, kGlobThreads, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(decode_global_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        decode_global_kernel<float><<<slots, kGlobThreads, smem, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace bp4m
