#pragma once
// Register-tile form of the FP32 shared-memory decode tiers (BP4M / BP4MF, Sec. "Belief
// Propagation", "Checking convergence", "Forced convergence"): the same message updates,
// decisions and outputs as decode_smem_kernel, with the messages held in registers.
//
// Layout.  The s x s message matrix of a shot (rows and columns padded to NB x B) is cut
// into NB x NB blocks of B x B.  Off-diagonal thread u owns the block pair {P, Q}, P < Q:
// the tile of messages M[i][k] (i in block P, k in block Q) and its mirror M[k][i], plus the
// priors l_ik = l_ki they share; diagonal thread D owns block (D, D).  A message and the
// message that meets it on the same variable v_ik therefore sit in the same thread, so the
// next incoming value Q_ik = l_ik + M[k][i] / alpha and the posterior
// lambda_ik = l_ik + (M[i][k] + M[k][i]) are formed in registers right after the update that
// produced them; no message crosses threads.  Only per-row statistics do: every thread
// writes one partial per row of its tiles (largest and second largest Q, kept-variable
// count; then the exponential sum) into shared memory, and two threads per row combine a
// row's partials.
//
// Leave-one-out max* in one formula for every column (base-2 units; m1 >= m2 the row's two
// largest Q, a the column of m1; c = 2^(m2 - m1)):
//   u_k = 2^max(x, 2^126 x), x = Q_k - m2       (u_k = 2^x <= 1 for k != a; u_a > 2^(m1-m2+1)
//                                                unless m1 == m2, where u_a = 1)
//   S' = sum_k min(u_k, 1) - 1 = sum_{k != a} 2^(Q_k - m2)  (>= 1: the column of m2 gives 1)
//   M'[i][k] = min(-(m1 + lg2(1 + c (S' - u_k))), -(m2 + lg2 S'))
// For k != a the first term is the exact -max*_{j != k} Q_j and is the smaller one (the set
// without k still holds the maximum).  For k = a the argument 1 + c (S' - u_a) lies below
// c S' (or is negative or not a number), so the first term exceeds the second, which is the
// exact -max*_{j != a} Q_j.  With exact ties (m1 == m2) every tied column has u = 1 and both
// terms agree.  One ex2 and one lg2 per message, as in the row form.
//
// Kept count and kept column of a row in one exactly summed float: a kept variable v_ik adds
// 1 + (k + 1) 2^-12 to row i; the row keeps exactly one variable iff its sum lies in [1, 2),
// and then (sum - 1) 2^12 - 1 is the column.  The per-shot decisions (candidates, forced
// convergence on the posteriors of the last iteration, kept in shared memory when needed)
// follow decode_smem_kernel step by step.
#include "decode_smem.cuh"

namespace bp4m {
namespace {

template <int NB>
struct RegShape {
    static constexpr int NOFF = NB * (NB - 1) / 2;  // off-diagonal block pairs
    static constexpr int WOFF = (NOFF + 31) / 32;   // their warps
    static constexpr int WDIAG = (NB + 31) / 32;    // warps of the diagonal blocks
    static constexpr int NT = 32 * (WOFF + WDIAG);
};

// Block pair of off-diagonal unit u, enumerated by the larger block: u = Q (Q - 1) / 2 + P,
// P < Q, so that the units of the first nb blocks are u < nb (nb - 1) / 2.
__host__ __device__ inline void reg_unit_pair(int u, int& P, int& Q) {
    int q = 1;
    while ((q + 1) * q / 2 <= u) ++q;
    Q = q;
    P = u - q * (q - 1) / 2;
}

// 1.0f if lam > 0, else 0.0f (NaN gives 0)
__device__ __forceinline__ float gt0f(float lam) {
    float r;
    asm("set.gt.f32.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(lam));
    return r;
}

// (largest, second largest) of the values so far and two more
__device__ __forceinline__ void top2_add(float& m1, float& m2, float v, float w) {
    const float hi = fmaxf(v, w), lo = fminf(v, w);
    m2 = max3f(m2, lo, fminf(m1, hi));
    m1 = fmaxf(m1, hi);
}

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 lg2x2(float2 y) { return mk2(B2<float>::lg2(y.x), B2<float>::lg2(y.y)); }

// 2^max(x, 2^126 x) for both halves (see the header comment)
__device__ __forceinline__ float2 ex2_marked(float2 x) {
    const float2 z = __fmul2_rn(x, mk2(0x1p126f, 0x1p126f));
    return mk2(B2<float>::ex2(fmaxf(x.x, z.x)), B2<float>::ex2(fmaxf(x.y, z.y)));
}

// Per-row constants of the output formula
struct RowK {
    float ncf, A, nm1, SP;
};
__device__ __forceinline__ RowK row_consts(float2 mm, float S) {
    RowK k;
    const float cf = B2<float>::ex2(mm.y - mm.x);
    const float S1 = S - 1.f;
    k.ncf = -cf;
    k.A = __fmaf_rn(cf, S1, 1.f);
    k.nm1 = -mm.x;
    k.SP = -mm.y - B2<float>::lg2(S1);
    return k;
}

// Kept-variable weight of column k
__device__ __forceinline__ float kept_w(int k) { return 1.f + (float)(k + 1) * (1.f / 4096.f); }

// Dynamic shared memory of the register-tile form
template <int NB, int B>
struct RegSmem {
    static constexpr int SMAX = NB * B;
    static constexpr int PP = SMAX + 1;  // pitch of the partial planes [NB][PP]
    static constexpr int LP = SMAX + 1;  // pitch of the posterior matrix
    static constexpr size_t o_rowd = 0;                                        // double [SMAX]
    static constexpr size_t o_pm = o_rowd + (size_t)SMAX * 8;                  // float2 [NB][PP]
    static constexpr size_t o_pa = o_pm + (size_t)NB * PP * 8;                 // float [NB][PP]
    static constexpr size_t o_ps = o_pa + (size_t)NB * PP * 4;                 // float [NB][PP]
    static constexpr size_t o_rst = (o_ps + (size_t)NB * PP * 4 + 7) / 8 * 8;  // float2 [SMAX]
    static constexpr size_t o_rS = o_rst + (size_t)SMAX * 8;                   // float [SMAX]
    static constexpr size_t o_racc = o_rS + (size_t)SMAX * 4;                  // float [SMAX]
    static constexpr size_t o_rk = (o_racc + (size_t)SMAX * 4 + 15) / 16 * 16;  // float4 [2][SMAX / 2]
    static constexpr size_t o_lam = o_rk + (size_t)SMAX * 16;                  // float [SMAX][LP]
    static constexpr size_t o_dets = o_lam + (size_t)SMAX * LP * 4;            // int [SMAX]
    static constexpr size_t o_choice = o_dets + (size_t)SMAX * 4;              // int [SMAX]
    static constexpr size_t o_bestp = o_choice + (size_t)SMAX * 4;             // short [SMAX]
    static constexpr size_t o_order = o_bestp + (size_t)SMAX * 2;              // short [SMAX]
    static constexpr size_t o_matched = o_order + (size_t)SMAX * 2;            // uchar [SMAX]
    static constexpr size_t o_flag = o_matched + (size_t)SMAX;                 // uchar [SMAX]
    static constexpr size_t bytes = o_flag + (size_t)SMAX + 16;
};

template <int NB, int B, bool TRACE>
__global__ void __launch_bounds__(RegShape<NB>::NT, 1) decode_reg_kernel(const DecodeArgs a) {
    static_assert(B % 2 == 0, "tiles are held as column pairs");
    using SH = RegShape<NB>;
    using SM = RegSmem<NB, B>;
    constexpr int SMAX = NB * B, BP = B / 2, NT = SH::NT, NW = NT / 32, PP = SM::PP, LP = SM::LP;
    static_assert(2 * SMAX <= NT && (2 * SMAX) % 32 == 0, "two combining threads per row, whole warps");
    extern __shared__ __align__(16) unsigned char smem[];
    double* rowd = reinterpret_cast<double*>(smem + SM::o_rowd);
    float2* pm = reinterpret_cast<float2*>(smem + SM::o_pm);
    float* pa = reinterpret_cast<float*>(smem + SM::o_pa);
    float* ps = reinterpret_cast<float*>(smem + SM::o_ps);
    float2* rst = reinterpret_cast<float2*>(smem + SM::o_rst);
    float* racc = reinterpret_cast<float*>(smem + SM::o_racc);
    // output constants of the row pair (2j, 2j + 1): rkA[j] = (-c, -c', A, A'),
    // rkB[j] = (-m1, -m1', SP, SP') (see row_consts)
    float4* rkA = reinterpret_cast<float4*>(smem + SM::o_rk);
    float4* rkB = rkA + SMAX / 2;
    float* Lam = reinterpret_cast<float*>(smem + SM::o_lam);
    int* dets = reinterpret_cast<int*>(smem + SM::o_dets);
    int* choice = reinterpret_cast<int*>(smem + SM::o_choice);
    short* bestp = reinterpret_cast<short*>(smem + SM::o_bestp);
    short* order = reinterpret_cast<short*>(smem + SM::o_order);
    unsigned char* matched = smem + SM::o_matched;
    unsigned char* flagb = smem + SM::o_flag;
    __shared__ int sh_item, sh_s, sh_best_par, sh_best_forced, sh_improve, sh_use_best;
    __shared__ double sh_best_w;
    __shared__ unsigned long long sh_acc[6];
    unsigned long long &acc_it = sh_acc[0], &acc_msg = sh_acc[1], &acc_def = sh_acc[2], &acc_shots = sh_acc[3],
                       &acc_fc = sh_acc[4], &acc_fcr = sh_acc[5];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool offd = warp < SH::WOFF;  // uniform per warp
    // this thread's blocks; a thread past the last unit gets NB (never active)
    int P = NB, Q = NB;
    if (offd) {
        if (tid < SH::NOFF) reg_unit_pair(tid, P, Q);
    } else if (tid - 32 * SH::WOFF < NB) {
        P = Q = tid - 32 * SH::WOFF;
    }
    const int count = *a.count;
    const float ainv = (float)(1.0 / a.alpha);
    const float2 ainv2 = mk2(ainv, ainv);
    const bool full = (a.decoder == 1) || !a.early_exit;
    float* trl = reinterpret_cast<float*>(a.tr_lambda);
    const float ninf = Num<float>::ninf();
    if (tid == 0)
        for (int k = 0; k < 6; ++k) sh_acc[k] = 0;

    // diagonal threads use L and X only (rows D B + r, columns D B + 2 cp, + 1)
    float2 L[B][BP], X[B][BP], Y[B][BP];

    for (;;) {
        if (tid == 0) sh_item = atomicAdd(a.next, 1);
        __syncthreads();
        const int item = sh_item;
        if (item >= count) break;
        const ItemCtx ic = resolve_item(a, a.list[item]);
        const int64_t shot = ic.shot;
        const int n = ic.tb.n_det;
        const float* __restrict__ Ltab = ic.tb.L32;
        if (warp == 0) {
            const int s0 = compact_defects(ic.synd + (size_t)shot * ic.tb.n_words, ic.tb.n_words, dets, SMAX, lane);
            if (lane == 0) sh_s = s0;
        }
        __syncthreads();
        const int s = sh_s;
        if (s > SMAX || s < 1) {
            if (tid == 0 && a.ctr) atomicAdd(a.ctr + C_ERRORS, 1ull);
            continue;
        }
        const bool tr_on = TRACE && s <= a.s_cap;
        if (s == 1) {
            // a single factor with a single variable: the leave-one-out set is empty, the
            // message is +inf and v_00 is kept in every iteration
            if (tid == 0) {
                const int its = full ? a.T : 1;
                const int d0 = dets[0];
                if (ic.obs_pred) ic.obs_pred[shot] = ic.tb.P[(size_t)d0 * n + d0];
                if (ic.flags) ic.flags[shot] = F_CONVERGED;
                if (ic.iters) ic.iters[shot] = (int16_t)its;
                if (tr_on && trl) trl[(size_t)shot * a.s_cap * a.s_cap] = Num<float>::pinf();
                if (tr_on && a.tr_partner) {
                    a.tr_partner[(size_t)shot * a.s_cap] = 0;
                    for (int k = 1; k < a.s_cap; ++k) a.tr_partner[(size_t)shot * a.s_cap + k] = -1;
                }
                acc_it += (unsigned long long)its;
                acc_msg += (unsigned long long)its;
                acc_def += 1;
                acc_shots += 1;
            }
            continue;
        }
        // blocks that hold the shot's rows; a thread works iff its larger block is one of them
        const int nbv = (s + B - 1) / B;
        const bool act = Q < nbv;
        const int i0 = P * B, k0 = Q * B;  // first row of block P, first column of block Q
        for (int r = tid; r < SMAX; r += NT) {
            matched[r] = r >= s;
            bestp[r] = -1;
        }
        if (tid == 0) {
            sh_best_w = Num<double>::pinf();
            sh_best_par = 0;
            sh_best_forced = 0;
            sh_use_best = 0;
        }
        // ---- priors (log2 units, -inf past s) and Q of the first update (M = 0: Q = l); the
        // rows' partial maxima
        auto prior = [&](int i, int k) -> float {
            return (i < s && k < s) ? __ldg(Ltab + (size_t)dets[i] * n + dets[k]) * (float)kLog2e : ninf;
        };
        if (act) {
#pragma unroll
            for (int r = 0; r < B; ++r)
#pragma unroll
                for (int cp = 0; cp < BP; ++cp) {
                    L[r][cp] = mk2(prior(i0 + r, k0 + 2 * cp), prior(i0 + r, k0 + 2 * cp + 1));
                    X[r][cp] = L[r][cp];
                    Y[r][cp] = L[r][cp];
                }
#pragma unroll
            for (int r = 0; r < B; ++r) {
                float m1 = ninf, m2 = ninf;
#pragma unroll
                for (int cp = 0; cp < BP; ++cp) top2_add(m1, m2, X[r][cp].x, X[r][cp].y);
                pm[Q * PP + i0 + r] = mk2(m1, m2);
                pa[Q * PP + i0 + r] = 0.f;
            }
            if (offd) {
#pragma unroll
                for (int c = 0; c < B; ++c) {
                    float m1 = ninf, m2 = ninf;
#pragma unroll
                    for (int rp = 0; rp < BP; ++rp) {
                        const float v = (c & 1) ? Y[2 * rp][c >> 1].y : Y[2 * rp][c >> 1].x;
                        const float w = (c & 1) ? Y[2 * rp + 1][c >> 1].y : Y[2 * rp + 1][c >> 1].x;
                        top2_add(m1, m2, v, w);
                    }
                    pm[P * PP + k0 + c] = mk2(m1, m2);
                    pa[P * PP + k0 + c] = 0.f;
                }
            }
        }

        int t = 0;
        bool any_conv = false, forced_ran = false;
        int out_par = 0, out_forced = 0, out_from_best = 0;
        for (;;) {
            __syncthreads();  // partials of Q^(t+1) and of the kept counts of lambda^t are written
            // ---- row statistics: two threads per row combine the row's partials
            bool ok = true;
            if (tid < 2 * SMAX) {
                const int row = tid >> 1, half = tid & 1;
                float m1 = ninf, m2 = ninf, acc = 0.f;
                if (row < s) {
                    // four partials in flight per step (independent loads), combined in order
                    for (int cb0 = half; cb0 < nbv; cb0 += 8) {
                        float2 o[4];
                        float oa[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int cb = cb0 + 2 * j;
                            o[j] = cb < nbv ? pm[cb * PP + row] : mk2(ninf, ninf);
                            oa[j] = cb < nbv ? pa[cb * PP + row] : 0.f;
                        }
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            m2 = max3f(m2, o[j].y, fminf(m1, o[j].x));
                            m1 = fmaxf(m1, o[j].x);
                            acc += oa[j];
                        }
                    }
                }
                const float o1 = __shfl_xor_sync(kFull, m1, 1), o2 = __shfl_xor_sync(kFull, m2, 1);
                const float oa = __shfl_xor_sync(kFull, acc, 1);
                m2 = max3f(m2, o2, fminf(m1, o1));
                m1 = fmaxf(m1, o1);
                acc += oa;
                if (half == 0) {
                    // rows past s get constants that keep their (unused) messages finite
                    rst[row] = row < s ? mk2(m1, m2) : mk2(0.f, 0.f);
                    racc[row] = acc;
                }
                ok = row >= s || (acc >= 1.f && acc < 2.f);
            }
            const int conv = __syncthreads_and(t > 0 && ok);

            if (t > 0) {
                bool have_cand = false, cand_forced = false;
                if (conv) {
                    // every row keeps exactly one variable: its column from the row's sum
                    any_conv = true;
                    have_cand = true;
                    for (int r = tid; r < s; r += NT) {
                        const int k = (int)rintf((racc[r] - 1.f) * 4096.f) - 1;
                        choice[r] = (k >= 0 && k < s) ? k : r;  // always in range (exact by construction)
                    }
                    __syncthreads();
                } else if (a.decoder == 1 || t == a.T) {
                    // ---- forced convergence on lambda^t (in Lam) by locally dominant rounds
                    forced_ran = true;
                    for (int r = tid; r < s; r += NT) matched[r] = 0;
                    __syncthreads();
                    if (a.forced_static) {
                        // the paper's static partition: row r's block is v_rk, k >= r; its
                        // maximum (ties: smaller k) represents factor r; representatives are
                        // ranked by posterior (ties: smaller r) and processed in that order
                        for (int r = warp; r < s; r += NW) {
                            float bl = ninf;
                            int bk = 0x7fffffff;
                            for (int k = r + lane; k < s; k += 32) {
                                const float lam = Lam[r * LP + k];
                                if (bk == 0x7fffffff || lam > bl) {
                                    bl = lam;
                                    bk = k;
                                }
                            }
#pragma unroll
                            for (int off = 16; off; off >>= 1) {
                                const float ol = __shfl_xor_sync(kFull, bl, off);
                                const int okk = __shfl_xor_sync(kFull, bk, off);
                                if (okk != 0x7fffffff && (bk == 0x7fffffff || ol > bl || (ol == bl && okk < bk))) {
                                    bl = ol;
                                    bk = okk;
                                }
                            }
                            if (lane == 0) {
                                choice[r] = bk != 0x7fffffff ? bk : r;
                                rowd[r] = (double)bl;
                            }
                        }
                        __syncthreads();
                        for (int r = tid; r < s; r += NT) {
                            const double v = rowd[r];
                            int rank = 0;
                            for (int j = 0; j < s; ++j) {
                                const double u = rowd[j];
                                rank += (u > v || (u == v && j < r)) ? 1 : 0;
                            }
                            order[rank] = (short)r;
                        }
                        __syncthreads();
                        if (tid == 0) {
                            // a factor whose representative's other factor is taken goes to
                            // the boundary (a case the paper does not treat)
                            for (int q = 0; q < s; ++q) {
                                const int rr = order[q];
                                if (matched[rr]) continue;
                                const int k = choice[rr];
                                matched[rr] = 1;
                                if (k == rr || matched[k]) {
                                    choice[rr] = rr;
                                } else {
                                    matched[k] = 1;
                                    choice[k] = rr;
                                }
                            }
                            acc_fcr += 1;
                        }
                        __syncthreads();
                    }
                    for (int round = 0; round < s && !a.forced_static; ++round) {
                        for (int r = warp; r < s; r += NW) {
                            if (matched[r]) continue;  // uniform per warp
                            float bl = ninf;
                            int bk = 0x7fffffff;
                            for (int k = lane; k < s; k += 32) {
                                if (k == r || !matched[k]) {
                                    const float lam = Lam[r * LP + k];
                                    if (bk == 0x7fffffff || lam > bl) {
                                        bl = lam;
                                        bk = k;
                                    }
                                }
                            }
#pragma unroll
                            for (int off = 16; off; off >>= 1) {
                                const float ol = __shfl_xor_sync(kFull, bl, off);
                                const int okk = __shfl_xor_sync(kFull, bk, off);
                                if (okk != 0x7fffffff && (bk == 0x7fffffff || ol > bl || (ol == bl && okk < bk))) {
                                    bl = ol;
                                    bk = okk;
                                }
                            }
                            if (lane == 0) choice[r] = bk != 0x7fffffff ? bk : r;
                        }
                        __syncthreads();
                        int left = 0;
                        for (int r = tid; r < s; r += NT) {
                            if (matched[r]) continue;
                            const int pk = choice[r];
                            const bool newm = (pk == r) || (choice[pk] == r);
                            flagb[r] = newm ? 1 : 0;
                            left += !newm;
                        }
                        __syncthreads();
                        for (int r = tid; r < s; r += NT)
                            if (!matched[r] && flagb[r]) matched[r] = 1;
                        if (tid == 0) acc_fcr += 1;
                        const int left_all = __syncthreads_count(left);
                        if (left_all == 0) break;
                    }
                    if (tid == 0) acc_fc += 1;
                    have_cand = true;
                    cand_forced = true;
                }
                if (have_cand) {
                    // ---- candidate parity (and weight when candidates are compared)
                    int pc = 0;
                    for (int r = tid; r < s; r += NT) {
                        const int k = choice[r];
                        double w = 0.0;
                        if (k >= r) {
                            const size_t off = (size_t)dets[r] * n + dets[k];
                            pc ^= ic.tb.P[off];
                            if (full) w = ic.tb.W64[off];
                        }
                        rowd[r] = w;
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
                            for (int r = 0; r < s; ++r) w += rowd[r];
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
                            for (int r = tid; r < s; r += NT) bestp[r] = (short)choice[r];
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
            }

            // ---- exponentials of the update: u = 2^max(x, 2^126 x), x = Q - m2; partial sums
            // of min(u, 1) per row
            if (act) {
#pragma unroll
                for (int r = 0; r < B; ++r) {
                    const float nm2 = -rst[i0 + r].y;
                    float2 sm = mk2(0.f, 0.f);
#pragma unroll
                    for (int cp = 0; cp < BP; ++cp) {
                        const float2 u = ex2_marked(__fadd2_rn(X[r][cp], mk2(nm2, nm2)));
                        X[r][cp] = u;
                        sm = __fadd2_rn(sm, mk2(fminf(u.x, 1.f), fminf(u.y, 1.f)));
                    }
                    ps[Q * PP + i0 + r] = sm.x + sm.y;
                }
                if (offd) {
#pragma unroll
                    for (int cp = 0; cp < BP; ++cp) {
                        const float2 nm2 = mk2(-rst[k0 + 2 * cp].y, -rst[k0 + 2 * cp + 1].y);
                        float2 sm = mk2(0.f, 0.f);
#pragma unroll
                        for (int r = 0; r < B; ++r) {
                            const float2 u = ex2_marked(__fadd2_rn(Y[r][cp], nm2));
                            Y[r][cp] = u;
                            sm = __fadd2_rn(sm, mk2(fminf(u.x, 1.f), fminf(u.y, 1.f)));
                        }
                        ps[P * PP + k0 + 2 * cp] = sm.x;
                        ps[P * PP + k0 + 2 * cp + 1] = sm.y;
                    }
                }
            }
            __syncthreads();
            if (tid < 2 * SMAX) {
                const int row = tid >> 1, half = tid & 1;
                float S = 0.f;
                if (row < s)
                    for (int cb0 = half; cb0 < nbv; cb0 += 8) {
                        float o[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) o[j] = cb0 + 2 * j < nbv ? ps[(cb0 + 2 * j) * PP + row] : 0.f;
#pragma unroll
                        for (int j = 0; j < 4; ++j) S += o[j];
                    }
                S += __shfl_xor_sync(kFull, S, 1);
                if (half == 0) {
                    // the row's output constants (rows past s: finite values for unused messages)
                    const RowK k = row < s ? row_consts(rst[row], S) : row_consts(mk2(0.f, 0.f), 2.f);
                    float* ra = reinterpret_cast<float*>(rkA + (row >> 1)) + (row & 1);
                    float* rb = reinterpret_cast<float*>(rkB + (row >> 1)) + (row & 1);
                    ra[0] = k.ncf;
                    ra[2] = k.A;
                    rb[0] = k.nm1;
                    rb[2] = k.SP;
                }
            }
            __syncthreads();

            // ---- outputs M^(t+1), then in the same registers lambda^(t+1), its kept counts and
            // Q^(t+2) with the rows' partial maxima
            if (act) {
                const bool need_lam = a.decoder == 1 || t + 1 == a.T;
                const bool tr_it = tr_on && trl != nullptr;
                if (offd) {
                    float sY1[B], sY2[B];
                    float2 accY[BP];
#pragma unroll
                    for (int c = 0; c < B; ++c) sY1[c] = sY2[c] = ninf;
#pragma unroll
                    for (int cp = 0; cp < BP; ++cp) accY[cp] = mk2(0.f, 0.f);
                    const float2 neg1 = mk2(-1.f, -1.f);
#pragma unroll
                    for (int rp = 0; rp < BP; ++rp) {
                        float sM1[2], sM2[2];
                        float2 accM[2];
                        // main rows i0 + 2 rp, i0 + 2 rp + 1 (one row pair record)
                        const float4 ma = rkA[(i0 >> 1) + rp], mb = rkB[(i0 >> 1) + rp];
                        const float2 mncf[2] = {mk2(ma.x, ma.x), mk2(ma.y, ma.y)};
                        const float2 mA[2] = {mk2(ma.z, ma.z), mk2(ma.w, ma.w)};
                        const float2 mnm1[2] = {mk2(mb.x, mb.x), mk2(mb.y, mb.y)};
                        const float mSP[2] = {mb.z, mb.w};
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            sM1[h] = sM2[h] = ninf;
                            accM[h] = mk2(0.f, 0.f);
                        }
#pragma unroll
                        for (int cp = 0; cp < BP; ++cp) {
                            const float2 wq = mk2(kept_w(k0 + 2 * cp), kept_w(k0 + 2 * cp + 1));
                            // mirror rows k0 + 2 cp, k0 + 2 cp + 1 (one row pair record)
                            const float4 ya = rkA[(k0 >> 1) + cp], yb = rkB[(k0 >> 1) + cp];
                            const float2 yncf = mk2(ya.x, ya.y), yA = mk2(ya.z, ya.w), ynm1 = mk2(yb.x, yb.y);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int r = 2 * rp + h;
                                // M'[i][k] (main pair) and M'[k][i] (mirror pair)
                                const float2 y = __ffma2_rn(mncf[h], X[r][cp], mA[h]);
                                float2 oM = __ffma2_rn(lg2x2(y), neg1, mnm1[h]);
                                oM = mk2(fminf(oM.x, mSP[h]), fminf(oM.y, mSP[h]));
                                const float2 yy = __ffma2_rn(yncf, Y[r][cp], yA);
                                float2 oY = __ffma2_rn(lg2x2(yy), neg1, ynm1);
                                oY = mk2(fminf(oY.x, yb.z), fminf(oY.y, yb.w));
                                const float2 lam = __fadd2_rn(L[r][cp], __fadd2_rn(oM, oY));
                                const float2 kk = mk2(gt0f(lam.x), gt0f(lam.y));
                                accM[h] = __ffma2_rn(kk, wq, accM[h]);
                                const float wp = kept_w(i0 + r);
                                accY[cp] = __ffma2_rn(kk, mk2(wp, wp), accY[cp]);
                                const int i = i0 + r, ka = k0 + 2 * cp;
                                if (need_lam) {
                                    Lam[i * LP + ka] = lam.x;
                                    Lam[ka * LP + i] = lam.x;
                                    Lam[i * LP + ka + 1] = lam.y;
                                    Lam[(ka + 1) * LP + i] = lam.y;
                                }
                                if (TRACE && tr_it && i < s) {
                                    const size_t base = (size_t)shot * a.s_cap;
                                    if (ka < s) {
                                        trl[(base + i) * a.s_cap + ka] = lam.x * (float)kLn2;
                                        trl[(base + ka) * a.s_cap + i] = lam.x * (float)kLn2;
                                    }
                                    if (ka + 1 < s) {
                                        trl[(base + i) * a.s_cap + ka + 1] = lam.y * (float)kLn2;
                                        trl[(base + ka + 1) * a.s_cap + i] = lam.y * (float)kLn2;
                                    }
                                }
                                X[r][cp] = __ffma2_rn(oY, ainv2, L[r][cp]);
                                Y[r][cp] = __ffma2_rn(oM, ainv2, L[r][cp]);
                                top2_add(sM1[h], sM2[h], X[r][cp].x, X[r][cp].y);
                            }
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            pm[Q * PP + i0 + 2 * rp + h] = mk2(sM1[h], sM2[h]);
                            pa[Q * PP + i0 + 2 * rp + h] = accM[h].x + accM[h].y;
                        }
                    }
#pragma unroll
                    for (int cp = 0; cp < BP; ++cp)
#pragma unroll
                        for (int rp = 0; rp < BP; ++rp) {
                            top2_add(sY1[2 * cp], sY2[2 * cp], Y[2 * rp][cp].x, Y[2 * rp + 1][cp].x);
                            top2_add(sY1[2 * cp + 1], sY2[2 * cp + 1], Y[2 * rp][cp].y, Y[2 * rp + 1][cp].y);
                        }
#pragma unroll
                    for (int cp = 0; cp < BP; ++cp) {
                        pm[P * PP + k0 + 2 * cp] = mk2(sY1[2 * cp], sY2[2 * cp]);
                        pm[P * PP + k0 + 2 * cp + 1] = mk2(sY1[2 * cp + 1], sY2[2 * cp + 1]);
                        pa[P * PP + k0 + 2 * cp] = accY[cp].x;
                        pa[P * PP + k0 + 2 * cp + 1] = accY[cp].y;
                    }
                } else {
                    // diagonal block: X[r][c] is element (i0 + r, i0 + c); first every output
#define GX(r, c) (((c) & 1) ? X[r][(c) >> 1].y : X[r][(c) >> 1].x)
#define GL(r, c) (((c) & 1) ? L[r][(c) >> 1].y : L[r][(c) >> 1].x)
                    float accD[B];
#pragma unroll
                    for (int r = 0; r < B; ++r) {
                        const float4 ka = rkA[(i0 + r) >> 1], kb = rkB[(i0 + r) >> 1];
                        const float ncf = (r & 1) ? ka.y : ka.x, A = (r & 1) ? ka.w : ka.z;
                        const float nm1 = (r & 1) ? kb.y : kb.x, SP = (r & 1) ? kb.w : kb.z;
                        accD[r] = 0.f;
#pragma unroll
                        for (int cp = 0; cp < BP; ++cp) {
                            const float2 y = __ffma2_rn(mk2(ncf, ncf), X[r][cp], mk2(A, A));
                            const float2 o = __ffma2_rn(lg2x2(y), mk2(-1.f, -1.f), mk2(nm1, nm1));
                            X[r][cp] = mk2(fminf(o.x, SP), fminf(o.y, SP));
                        }
                    }
                    // then each variable of the block: lambda, kept counts, next Q
#pragma unroll
                    for (int r = 0; r < B; ++r) {
#pragma unroll
                        for (int c = r; c < B; ++c) {
                            const int i = i0 + r, k = i0 + c;
                            const float l = GL(r, c);
                            float lam;
                            if (c == r) {
                                lam = l + GX(r, r);
                                GX(r, r) = l;
                            } else {
                                const float mrc = GX(r, c), mcr = GX(c, r);
                                lam = l + (mrc + mcr);
                                GX(r, c) = __fmaf_rn(mcr, ainv, l);
                                GX(c, r) = __fmaf_rn(mrc, ainv, l);
                            }
                            const float kk = gt0f(lam);
                            accD[r] = __fmaf_rn(kk, kept_w(k), accD[r]);
                            if (c != r) accD[c] = __fmaf_rn(kk, kept_w(i), accD[c]);
                            if (need_lam) {
                                Lam[i * LP + k] = lam;
                                Lam[k * LP + i] = lam;
                            }
                            if (TRACE && tr_it && i < s && k < s) {
                                const size_t base = (size_t)shot * a.s_cap;
                                trl[(base + i) * a.s_cap + k] = lam * (float)kLn2;
                                trl[(base + k) * a.s_cap + i] = lam * (float)kLn2;
                            }
                        }
                    }
#pragma unroll
                    for (int r = 0; r < B; ++r) {
                        float m1 = ninf, m2 = ninf;
#pragma unroll
                        for (int cp = 0; cp < BP; ++cp) top2_add(m1, m2, X[r][cp].x, X[r][cp].y);
                        pm[P * PP + i0 + r] = mk2(m1, m2);
                        pa[P * PP + i0 + r] = accD[r];
                    }
#undef GX
#undef GL
                }
            }
            ++t;
        }

        // ---- outputs of the shot
        if (tr_on && a.tr_partner) {
            for (int r = tid; r < a.s_cap; r += NT) {
                int pk = -1;
                if (r < s) pk = out_from_best ? (int)bestp[r] : choice[r];
                a.tr_partner[(size_t)shot * a.s_cap + r] = (int16_t)pk;
            }
        }
        if (tid == 0) {
            if (ic.obs_pred) ic.obs_pred[shot] = (uint8_t)out_par;
            if (ic.flags)
                ic.flags[shot] = (uint8_t)((any_conv ? F_CONVERGED : 0) | (forced_ran ? F_FORCED_RAN : 0) |
                                          (out_forced ? F_FROM_FORCED : 0));
            if (ic.iters) ic.iters[shot] = (int16_t)t;
            acc_it += (unsigned long long)t;
            acc_msg += (unsigned long long)s * s * t;
            acc_def += (unsigned long long)s;
            acc_shots += 1;
        }
        __syncthreads();
    }
    if (tid == 0 && a.ctr) {
        atomicAdd(a.ctr + C_ITERS, acc_it);
        atomicAdd(a.ctr + C_MSGS, acc_msg);
        atomicAdd(a.ctr + C_DEFECTS, acc_def);
        atomicAdd(a.ctr + C_TIER_MSGS + a.tier, acc_msg);
        atomicAdd(a.ctr + C_TIER_SHOTS + a.tier, acc_shots);
        atomicAdd(a.ctr + C_FC_RUNS, acc_fc);
        atomicAdd(a.ctr + C_FC_ROUNDS, acc_fcr);
    }
}

template <int NB, int B, bool TRACE>
cudaError_t run_reg_tier(const DecodeArgs& a, int num_sms, cudaStream_t st, bool prepare_only) {
    const size_t smem = RegSmem<NB, B>::bytes;
    auto kern = decode_reg_kernel<NB, B, TRACE>;
    if (prepare_only) return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, RegShape<NB>::NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<per_sm * num_sms, RegShape<NB>::NT, smem, st>>>(a);
    return cudaGetLastError();
}

// Production and traced instantiations of one register-tile tier
template <int NB, int B>
cudaError_t run_reg_tier2(const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep) {
    const bool tr = a.tr_lambda != nullptr || a.tr_partner != nullptr;
    if (prep) {
        cudaError_t e = run_reg_tier<NB, B, false>(a, num_sms, st, true);
        return e != cudaSuccess ? e : run_reg_tier<NB, B, true>(a, num_sms, st, true);
    }
    return tr ? run_reg_tier<NB, B, true>(a, num_sms, st, false) : run_reg_tier<NB, B, false>(a, num_sms, st, false);
}

}  // namespace
}  // namespace bp4m
