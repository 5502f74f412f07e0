#pragma once
// Streaming tier of the BP4M decoder: shots with more unsatisfied detectors than the
// shared-memory tiers hold, their message matrices in a per-block global scratch slot.
// Shared by the FP32/FP64 instantiations (kernels_decode.cu) and the 16-bit message
// storage ones (kernels_half.cu).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <type_traits>

#include "decode_smem.cuh"
#include "device.cuh"

namespace bp4m {
namespace {

namespace cg = cooperative_groups;

// ------------------------------------------------------------------ streaming tier
//
// Shots with more unsatisfied detectors than the shared-memory tiers hold.  One warp owns
// one factor row at a time (its CH*32 columns in registers); the shot's matrices live in a
// per-block scratch slot in global memory (L2-resident for the sizes this tier meets):
//   Lg[r][k]     prior l_rk in log2 units, -inf for k >= s          (ld = 32*CH columns)
//   Mt[b][r][k]  incoming message M[k][r], double buffered (b = iteration parity)
//   Mo[r][k]     the row's own outputs M[r][k], updated in place by the owning warp, for the
//                decision passes that read whole posterior rows (the last iteration, BP4MF,
//                full-T mode, traces; the fused decisions of the 16-bit and cluster forms and
//                of FP32 below 320 columns).  FP32 BP4M with early exit, one block per shot, from
//                320 columns judges an update's posteriors in the pass that produces it instead
//                and writes Mo only before the last iteration.
// The diagonal of Mt is kept 0, so Q_rr = l_rr and lambda_rr = l_rr + Mo[r][r].
// With 16-bit message storage (MS = __half or __nv_bfloat16; priors and arithmetic FP32)
// every message leaving row r is stored relative to the row's reference r_r (its largest Q
// of that update rounded to the format), as in the shared-memory tiers: Mt[k][r] and
// Mo[r][k] hold M[r][k] + r_r, the diagonal of Mt holds r_r (decoding to exactly 0), and
// readers add -r_r, kept in FP32 per row and iteration in shared memory (nref[2][LD]).  Outputs go
// to Mt[next][k][r]; a batch of W consecutive rows (one per warp) stages them in shared
// memory and writes W consecutive elements per column k.  Iteration = decision pass
// (lambda of the previous update, convergence vote, candidates / forced convergence), then
// the update pass.
//
// Cluster form (CL > 1, FP32 arithmetic): the CL blocks of a thread-block cluster share one
// shot and one slot, so that the slots of all shots in flight (one per cluster instead of
// one per block) stay resident in L2 instead of streaming from HBM every iteration.  Block
// q of the cluster owns the batches b = q, q + CL, ... (rows b W .. b W + W - 1): it
// initialises their rows, updates them and takes their decisions.  Messages cross blocks
// only through the slot (read with L1-bypassing loads); the small per-row state (choices,
// the 16-bit references, the static partition's block maxima) is written by the row's owner
// into every block's copy through distributed shared memory, after which every block runs
// the row-global steps (parity, candidate weights, forced-convergence matching) itself on
// identical data.  So every value a branch or loop bound depends on is the same in all
// blocks of a cluster, and every cluster barrier is reached by all of them.
constexpr int kStreamWarps = 16;
// Blocks per SM: the 256-column variant (shots of up to 256 defects) runs two, so that one
// block's L2 latency overlaps the other's arithmetic.  The cluster form (CL > 1) runs one
// 16-warp block per SM at these widths: its slots are L2-resident, and 128 registers per
// thread keep its rows' registers from spilling.
template <typename T, int CH, int CL = 1>
constexpr int kStreamBlocks = (sizeof(T) == 4 && CH <= 8 && CL == 1) ? 2 : 1;
// Warps per block (one row in flight per warp, each with a 3-row prefetch buffer in shared
// memory): FP32 320 and 384 columns run one 32-warp block per SM (twice the rows in flight
// per batch and half the batch barriers of 16 warps; 16 in the cluster form), 896 and 1024
// columns one 12-warp block (the largest count whose prefetch buffers and output stage fit
// in 227 KB), the others 16.
template <typename T, int CH, int CL = 1>
constexpr int kStreamWarpsOf = sizeof(T) != 4 ? kStreamWarps : CH >= 28 ? 12 : (CH >= 10 && CH <= 12 && CL == 1) ? 32 : kStreamWarps;
// Row prefetch of the update pass: each warp copies its next row of Lg, Mc and Mo into
// shared memory (asynchronous copies) while it updates the current one.
//   1: the row is moved into registers and the next copy issued at once (FP32, <= 256 columns)
//   2: the row is read in place and the next copy issued after its last read (FP32, 320 to
//      1024 columns, where the register copy would spill)
//   0: rows are read from global memory (FP64)
template <typename T, int CH>
constexpr int kStreamPrefetch = sizeof(T) != 4 ? 0 : CH <= 8 ? 1 : 2;

// Output stage pitch in elements: a batch's W rows are read back four rows of one column per
// thread (W/4 threads per column, 32/(W/4) columns per warp), which is free of bank
// conflicts with an odd pitch for 32 warps and with a pitch of twice an odd number for 16
// (and nearly so for 12).
template <typename T, int CH, int CL = 1>
constexpr int kStagePitch = 32 * CH + (kStreamWarpsOf<T, CH, CL> == 32 ? 1 : 2);

// Dynamic shared memory of one streaming block with `stages` output stages.
template <typename T, int CH, typename MS, int CL = 1>
constexpr size_t stream_smem_bytes_n(int stages) {
    return (kStreamPrefetch<T, CH> != 0 ? (size_t)kStreamWarpsOf<T, CH, CL> * 3 * (32 * CH) * sizeof(T) : 0) +
           (size_t)stages * kStreamWarpsOf<T, CH, CL> * kStagePitch<T, CH, CL> * sizeof(T) + sizeof(T) +
           (size_t)(32 * CH) * (sizeof(double) + 2 * sizeof(int) + sizeof(short) + 1) + 32 +
           (sizeof(MS) == 2 ? (size_t)2 * (32 * CH) * sizeof(float) : 0) + (size_t)(32 * CH) * sizeof(short) +
           (size_t)2 * (32 * CH) * sizeof(unsigned short);
}
// Two output stages where they fit: 227 KB per block, and for the two-block variants 113 KB.
template <typename T, int CH, typename MS, int CL = 1>
constexpr int kStreamStages =
    stream_smem_bytes_n<T, CH, MS, CL>(2) <= (kStreamBlocks<T, CH, CL> == 2 ? 113u : 227u) * 1024u ? 2 : 1;

// 16-byte asynchronous global->shared copies (cp.async, L2 only), used to fetch a warp's next
// factor row while it works on the current one
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    const size_t g = __cvta_generic_to_global(gmem_src);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v = B2<T>::mx(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

// Four consecutive message-matrix elements from FP32 values (exact in MS): one 16-byte store
// for FP32 storage, one 8-byte store for 16-bit storage.  p is aligned to 4 elements.
template <typename MS, typename T>
__device__ __forceinline__ void st4(MS* p, T a, T b, T c, T d) {
    if constexpr (sizeof(MS) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    } else if constexpr (sizeof(MS) == 2) {
        auto bits = [](T x) -> unsigned {
            const MS v = MS(x);
            return *reinterpret_cast<const unsigned short*>(&v);
        };
        *reinterpret_cast<uint2*>(p) = make_uint2(bits(a) | bits(b) << 16, bits(c) | bits(d) << 16);
    } else {
        p[0] = a;
        p[1] = b;
        p[2] = c;
        p[3] = d;
    }
}

// Bytes of one streaming slot: priors (T) and three message matrices (MS) of LD x LD.
template <typename T, typename MS>
__host__ __device__ constexpr size_t stream_slot_bytes(int ld) {
    return (size_t)ld * ld * (sizeof(T) + 3 * sizeof(MS));
}

template <typename T, int CH, bool TRACE, int W, typename MS = T, int CL = 1>
__global__ void __launch_bounds__(W * 32, W == kStreamWarps ? kStreamBlocks<T, CH, CL> : 1) decode_stream_kernel(const DecodeArgs a) {
    constexpr bool HALF = sizeof(MS) == 2;
    static_assert(!HALF || sizeof(T) == 4, "16-bit messages use FP32 arithmetic");
    static_assert(CL == 1 || (sizeof(T) == 4 && !TRACE && CL <= 16), "cluster form: FP32 arithmetic, no trace");
    static_assert(W % 4 == 0, "the transposed write takes four rows per thread");
    using IO = MsgIO<MS, T>;
    constexpr int NTH = W * 32;
    constexpr int LD = 32 * CH;
    constexpr int SP = kStagePitch<T, CH, CL>;  // output stage pitch
    // FP32 variants of up to 256 columns prefetch each warp's next row of Lg, Mc and Mo into
    // shared memory (pf[W][3][LD]) during the current row's update
    constexpr int PFM = kStreamPrefetch<T, CH>;
    constexpr bool PF = PFM != 0;
    extern __shared__ __align__(16) unsigned char smem[];
    T* const pf = reinterpret_cast<T*>(smem);
    // output stage [NST][W][SP]: with two stages a batch's rows go to one while the previous
    // batch's transposed write reads the other, one block barrier per batch instead of two
    constexpr int NST = kStreamStages<T, CH, MS, CL>;
    T* stage0 = pf + (PF ? W * 3 * LD : 0);
    double* rowacc = reinterpret_cast<double*>(stage0 + NST * W * SP + ((NST * W * SP) & 1));
    int* dets = reinterpret_cast<int*>(rowacc + LD);
    int* choice = dets + LD;
    short* bestp = reinterpret_cast<short*>(choice + LD);
    unsigned char* matched = reinterpret_cast<unsigned char*>(bestp + LD);
    // 16-bit: nref[b][k] = -r_k of the messages in Mtb[b] and of the own outputs (b = parity)
    float* nref = reinterpret_cast<float*>(reinterpret_cast<uintptr_t>(matched + LD + 15) & ~(uintptr_t)15);
    // static-partition forced convergence: factors in processing order
    short* order = reinterpret_cast<short*>(nref + (HALF ? 2 * LD : 0));
    // posteriors judged in the update pass (see `late` below): kept counts of the rows, two
    // 16-bit counters per word, one buffer per pass parity
    unsigned* kcnt = reinterpret_cast<unsigned*>(order + LD);
    __shared__ int sh_item2[2], sh_s, sh_best_par, sh_best_forced, sh_improve, sh_use_best;
    __shared__ int sh_votes[2][CL];  // cluster form: each block's vote, by iteration parity
    __shared__ double sh_best_w;

    // cluster form: this block's rank; writes of per-row state go to every block's copy
    const int crank = CL > 1 ? (int)cg::this_cluster().block_rank() : 0;
    auto csync = [&]() {
        if constexpr (CL > 1)
            cg::this_cluster().sync();
        else
            __syncthreads();
    };
    auto bcast = [&](auto* p, auto v) {
        if constexpr (CL > 1) {
            cg::cluster_group cl = cg::this_cluster();
#pragma unroll
            for (int q = 0; q < CL; ++q) *cl.map_shared_rank(p, q) = v;
        } else {
            *p = v;
        }
    };

    const size_t mat = (size_t)LD * LD;
    unsigned char* slot = reinterpret_cast<unsigned char*>(a.gscratch) + (size_t)(blockIdx.x / CL) * stream_slot_bytes<T, MS>(LD);
    T* Lg = reinterpret_cast<T*>(slot);
    MS* Mtb[2] = {reinterpret_cast<MS*>(slot + mat * sizeof(T)), reinterpret_cast<MS*>(slot + mat * (sizeof(T) + sizeof(MS)))};
    MS* Mo = reinterpret_cast<MS*>(slot + mat * (sizeof(T) + 2 * sizeof(MS)));

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t count = a.count ? (int64_t)*a.count : a.count_val;
    const T ainv = (T)(1.0 / a.alpha);
    const bool full = (a.decoder == 1) || !a.early_exit;
    T* trl = reinterpret_cast<T*>(a.tr_lambda);
    const T ninf = Num<T>::ninf();
    unsigned long long acc_it = 0, acc_msg = 0, acc_def = 0, acc_shots = 0, acc_fc = 0, acc_fcr = 0;

    // rows this block owns: r = crank W + warp + j W CL (all rows when CL = 1)
    const int row0 = crank * W + warp;
    constexpr int RSTEP = W * CL;
    // every block of the cluster runs before any block writes into another's shared memory
    if constexpr (CL > 1) csync();
    for (int fetch = 0;; ++fetch) {
        // the cluster's next shot, taken by block 0 and written into every block (two
        // buffers by fetch parity: a block may still be reading the previous one)
        const int fb = CL > 1 ? (fetch & 1) : 0;
        if (crank == 0 && tid == 0) bcast(&sh_item2[fb], atomicAdd(a.next, 1));
        csync();
        const int item = sh_item2[fb];
        if (item >= count) break;
        const ItemCtx ic = resolve_item(a, a.list ? (int64_t)a.list[item] : (int64_t)item);
        const int64_t shot = ic.shot;
        const int n = ic.tb.n_det;
        const T* __restrict__ Ltab = Num<T>::L(ic.tb);
        if (warp == 0) {
            const int s0 = compact_defects(ic.synd + (size_t)shot * ic.tb.n_words, ic.tb.n_words, dets, LD, lane);
            if (lane == 0) sh_s = s0;
        }
        __syncthreads();
        const int s = sh_s;
        if (s > LD || s < 2) {
            if (crank == 0 && tid == 0 && a.ctr) atomicAdd(a.ctr + C_ERRORS, 1ull);
            continue;
        }
        const bool tr_on = TRACE && s <= a.s_cap;
        for (int r = row0; r < s; r += RSTEP) {
            const T* trow = Ltab + (size_t)dets[r] * n;
            for (int k = lane; k < LD; k += 32) {
                Lg[(size_t)r * LD + k] = k < s ? (T)(__ldg(trow + dets[k]) * (T)kLog2e) : ninf;
                Mtb[0][(size_t)r * LD + k] = MS(0.f);
                Mtb[1][(size_t)r * LD + k] = MS(0.f);
                Mo[(size_t)r * LD + k] = MS(0.f);
            }
        }
        for (int r = tid; r < LD; r += NTH) {
            matched[r] = r >= s;
            bestp[r] = -1;
            if constexpr (HALF) nref[r] = nref[LD + r] = 0.f;
            if (r < LD / 2) kcnt[r] = kcnt[LD / 2 + r] = 0u;
        }
        if (tid == 0) {
            sh_best_w = Num<double>::pinf();
            sh_best_par = 0;
            sh_best_forced = 0;
            sh_use_best = 0;
        }
        // every block's rows of the slot are initialised before any block writes into them
        csync();

        int cur = 0;
        int t = 0;
        bool any_conv = false, forced_ran = false;
        int out_par = 0, out_forced = 0, out_from_best = 0;

        // BP4M with early exit, 16-bit messages, the cluster form or FP32 below 320 columns: the
        // decisions of lambda^t are taken inside the update pass that reads the same rows (Lg,
        // Mc, Mo once per iteration instead of twice); only the last iteration, which may need
        // forced convergence, keeps the separate decision pass.  The FP32 one-block form from
        // 320 columns judges late instead (below)
        const bool merged = !TRACE && a.decoder == 0 && a.early_exit;
        // FP32 messages, one block per shot, 320 columns and more: the posteriors of an update
        // are judged in the pass that produces it, each variable once, by the later of its two
        // rows (the earlier row's message to it is then in the next incoming matrix, or in the
        // batch's stage).  The own-output matrix is then neither read nor written, except in
        // the pass before the last iteration, whose decisions may need forced convergence.  A
        // variable whose posterior is bounded above by l + (own + -max_{j != r} Q_kj) <= 0 (the
        // partner's message never exceeds minus its largest other entry) is not read at all.
        // The 192- and 256-column variants keep the fused decisions: there the extra per-row
        // work cost more time than the saved bytes.
        constexpr bool LATE_OK = CL == 1 && !HALF && sizeof(T) == 4 && CH >= 10;
        const bool late = LATE_OK && merged;
        // kept variable v_rk (k == r: the boundary), counted at both ends; the kept column is
        // only read for rows that keep exactly one
        auto kept = [&](unsigned* cb, int r, int k) {
            atomicAdd(cb + (r >> 1), 1u << ((r & 1) * 16));
            choice[r] = k;
            if (k != r) {
                atomicAdd(cb + (k >> 1), 1u << ((k & 1) * 16));
                choice[k] = r;
            }
        };
        for (;;) {
            const MS* Mc = Mtb[cur];
            const float* nrc = nref + cur * LD;        // references of the messages read now
            float* nrn = nref + (cur ^ 1) * LD;        // references of the messages written now
            // the message from row k to row r, and row r's own output to column k
            auto dx = [&](const MS* p, int k) -> T {
                if constexpr (HALF) return IO::ld(p) + nrc[k];
                else return *p;
            };
            // the same from the slot in global memory (cluster form: rows of Mc are written by
            // every block of the cluster, so they are read from L2, bypassing this SM's L1)
            auto dxg = [&](const MS* p, int k) -> T {
                if constexpr (CL > 1) {
                    if constexpr (HALF) return IO::unpack((unsigned)__ldcg(reinterpret_cast<const unsigned short*>(p))).x + nrc[k];
                    else return __ldcg(p);
                } else {
                    return dx(p, k);
                }
            };
            auto down = [&](const MS* p, int r) -> T {
                if constexpr (HALF) return IO::ld(p) + nrc[r];
                else return *p;
            };
            const bool fuse = !LATE_OK && merged && t > 0 && t < a.T;
            // with late judging the decisions of lambda^t (t < T) were taken in the last pass
            if (t > 0 && !fuse && !(late && t < a.T)) {
                // ---- decisions of lambda^t = l + (M[r][k] + M[k][r])
                int ok_all = 1;
                for (int r = row0; r < s; r += RSTEP) {
                    const T* lrow = Lg + (size_t)r * LD;
                    const MS* xrow = Mc + (size_t)r * LD;
                    const MS* orow = Mo + (size_t)r * LD;
                    // kept count and a kept column of the row (the only one when the count is 1,
                    // the case in which it is used: otherwise forced convergence replaces it)
                    int cnt = 0, kl = -1;
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        const int k = lane + 32 * c;
                        const T lam = lrow[k] + (down(orow + k, r) + dxg(xrow + k, k));
                        const bool kp = lam > T(0);
                        cnt += kp ? 1 : 0;
                        kl = kp ? k : kl;
                        if (tr_on && trl && k < s) trl[((size_t)shot * a.s_cap + r) * a.s_cap + k] = lam * (T)kLn2;
                    }
#pragma unroll
                    for (int off = 16; off; off >>= 1) {
                        cnt += __shfl_xor_sync(kFull, cnt, off);
                        kl = max(kl, __shfl_xor_sync(kFull, kl, off));
                    }
                    if (lane == 0) bcast(&choice[r], kl >= 0 ? kl : 0x7fffffff);
                    ok_all &= (cnt == 1);
                }
                int conv;
                if constexpr (CL > 1) {
                    const int cta_ok = __syncthreads_and(ok_all);
                    if (tid == 0) bcast(&sh_votes[t & 1][crank], cta_ok);
                    csync();
                    conv = 1;
#pragma unroll
                    for (int q = 0; q < CL; ++q) conv &= sh_votes[t & 1][q];
                } else {
                    conv = __syncthreads_and(ok_all);
                }
                bool have_cand = false, cand_forced = false;
                if (conv) {
                    any_conv = true;
                    have_cand = true;
                } else if (a.decoder == 1 || t == a.T) {
                    // ---- forced convergence on lambda^t by locally dominant rounds
                    forced_ran = true;
                    for (int r = tid; r < s; r += NTH) matched[r] = 0;
                    __syncthreads();
                    if (a.forced_static) {
                        // the paper's static partition: row r's block is v_rk, k >= r; its
                        // maximum (ties: smaller k) represents factor r; representatives are
                        // ranked by posterior (ties: smaller r) and processed in that order
                        for (int r = row0; r < s; r += RSTEP) {
                            const T* lrow = Lg + (size_t)r * LD;
                            const MS* xrow = Mc + (size_t)r * LD;
                            const MS* orow = Mo + (size_t)r * LD;
                            T bl = ninf;
                            int bk = 0x7fffffff;
#pragma unroll
                            for (int c = 0; c < CH; ++c) {
                                const int k = lane + 32 * c;
                                if (k >= r && k < s) {
                                    const T lam = lrow[k] + (down(orow + k, r) + dxg(xrow + k, k));
                                    if (bk == 0x7fffffff || lam > bl) {
                                        bl = lam;
                                        bk = k;
                                    }
                                }
                            }
#pragma unroll
                            for (int off = 16; off; off >>= 1) {
                                const T ol = __shfl_xor_sync(kFull, bl, off);
                                const int okk = __shfl_xor_sync(kFull, bk, off);
                                if (okk != 0x7fffffff && (bk == 0x7fffffff || ol > bl || (ol == bl && okk < bk))) {
                                    bl = ol;
                                    bk = okk;
                                }
                            }
                            if (lane == 0) {
                                bcast(&choice[r], bk != 0x7fffffff ? bk : r);
                                bcast(&rowacc[r], (double)bl);
                            }
                        }
                        csync();
                        for (int r = tid; r < s; r += NTH) {
                            const double v = rowacc[r];
                            int rank = 0;
                            for (int j = 0; j < s; ++j) {
                                const double u = rowacc[j];
                                rank += (u > v || (u == v && j < r)) ? 1 : 0;
                            }
                            order[rank] = (short)r;
                        }
                        __syncthreads();
                        if (tid == 0) {
                            // a factor whose representative's other factor is taken goes to the
                            // boundary (a case the paper does not treat)
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
                            if (crank == 0) acc_fcr += 1;
                        }
                        __syncthreads();
                    }
                    for (int round = 0; round < s && !a.forced_static; ++round) {
                        for (int r = row0; r < s; r += RSTEP) {
                            if (matched[r]) continue;  // uniform per warp
                            const T* lrow = Lg + (size_t)r * LD;
                            const MS* xrow = Mc + (size_t)r * LD;
                            const MS* orow = Mo + (size_t)r * LD;
                            T bl = ninf;
                            int bk = 0x7fffffff;
#pragma unroll
                            for (int c = 0; c < CH; ++c) {
                                const int k = lane + 32 * c;
                                if (k < s && (k == r || !matched[k])) {
                                    const T lam = lrow[k] + (down(orow + k, r) + dxg(xrow + k, k));
                                    if (bk == 0x7fffffff || lam > bl) {
                                        bl = lam;
                                        bk = k;
                                    }
                                }
                            }
#pragma unroll
                            for (int off = 16; off; off >>= 1) {
                                const T ol = __shfl_xor_sync(kFull, bl, off);
                                const int okk = __shfl_xor_sync(kFull, bk, off);
                                if (okk != 0x7fffffff && (bk == 0x7fffffff || ol > bl || (ol == bl && okk < bk))) {
                                    bl = ol;
                                    bk = okk;
                                }
                            }
                            if (lane == 0) bcast(&choice[r], bk != 0x7fffffff ? bk : r);
                        }
                        csync();
                        int left = 0;
                        for (int r = tid; r < s; r += NTH) {
                            if (matched[r]) continue;
                            const int pk = choice[r];
                            const bool newm = (pk == r) || (choice[pk] == r);
                            rowacc[r] = newm ? 1.0 : 0.0;
                            left += !newm;
                        }
                        __syncthreads();
                        for (int r = tid; r < s; r += NTH)
                            if (!matched[r] && rowacc[r] != 0.0) matched[r] = 1;
                        if (tid == 0 && crank == 0) acc_fcr += 1;
                        const int left_all = __syncthreads_count(left);
                        // cluster form: the next round's choices overwrite every block's copy
                        if constexpr (CL > 1) csync();
                        if (left_all == 0) break;
                    }
                    if (tid == 0 && crank == 0) acc_fc += 1;
                    have_cand = true;
                    cand_forced = true;
                }
                if (have_cand) {
                    int pc = 0;
                    for (int r = tid; r < s; r += NTH) {
                        const int k = choice[r];
                        double w = 0.0;
                        if (k >= r) {
                            const size_t off = (size_t)dets[r] * n + dets[k];
                            pc ^= ic.tb.P[off];
                            if (full) w = ic.tb.W64[off];
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
                            for (int r = tid; r < s; r += NTH) bestp[r] = (short)choice[r];
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
            // ---- update pass: M' for every row, batch by batch
            MS* Mn = Mtb[cur ^ 1];
            const int nbatch = (s + W - 1) / W;
            int ok_w = 1;  // fused decisions: every row of this warp keeps exactly one variable
            // late judging of lambda^(t+1) in this pass (the last iteration's are judged from the
            // own outputs, which this pass then writes)
            const bool eval = late && t + 1 < a.T;
            unsigned* const kc = kcnt + (t & 1) * (LD / 2);
            if (late)
                for (int r = tid; r < LD / 2; r += NTH) kcnt[((t + 1) & 1) * (LD / 2) + r] = 0u;
            T* const pbuf = pf + warp * 3 * LD;
            // row rr of Lg, Mc and Mo into this warp's prefetch buffer (one commit group)
            // (16-bit message rows fill the first half of their buffer row).  In the FP32 one-block
            // form from 320 columns the own outputs are not fetched (only the fused decisions of
            // the other forms read them), and the prior rows alternate between the first and
            // third buffer rows (j = the warp's row count), so that a row's priors stay in place
            // while the next row is fetched
            auto lslot = [&](int j) -> T* { return pbuf + ((LATE_OK && (j & 1)) ? 2 * LD : 0); };
            auto prefetch = [&](int rr, int j) {
                const unsigned char* src[3] = {reinterpret_cast<const unsigned char*>(Lg + (size_t)rr * LD),
                                               reinterpret_cast<const unsigned char*>(Mc + (size_t)rr * LD),
                                               reinterpret_cast<const unsigned char*>(Mo + (size_t)rr * LD)};
                constexpr int VL = LD * (int)sizeof(T) / 16;   // 16-byte chunks per prior row
                constexpr int VM = LD * (int)sizeof(MS) / 16;  // and per message row
                const int nm = LATE_OK ? 2 : 3;  // the update pass reads own outputs only in the fused decisions
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    if (m >= nm) break;
                    unsigned char* dst = reinterpret_cast<unsigned char*>(m == 0 ? lslot(j) : pbuf + m * LD);
                    for (int v = lane; v < (m == 0 ? VL : VM); v += 32) cp_async16(dst + 16 * v, src[m] + 16 * v);
                }
                cp_async_commit();
            };
            const MS* pbx = reinterpret_cast<const MS*>(pbuf + LD);
            const MS* pbo = reinterpret_cast<const MS*>(pbuf + 2 * LD);
            // late judging: the rows' largest and second largest Q and argmax of this pass
            // (the bound of their messages), in the decision scratch
            float2* rstat = reinterpret_cast<float2*>(rowacc);
            int jrow = 0;  // rows this warp has taken in this pass
            if constexpr (PF)
                if (row0 < s) prefetch(row0, 0);
            // this block's batches b = crank, crank + CL, ...; the stage alternates with b / CL
            for (int b = crank; b < nbatch; b += CL) {
                const int r = b * W + warp;
                T* const stage = stage0 + (NST == 2 ? ((b / CL) & 1) : 0) * W * SP;
                T* srow = stage + warp * SP;
                if (r < s) {
                    const T* lrow = Lg + (size_t)r * LD;
                    const MS* xrow = Mc + (size_t)r * LD;
                    MS* orow = Mo + (size_t)r * LD;
                    const T* const pbl = lslot(jrow);  // this row's priors in the prefetch buffer
                    T lv[PFM == 1 ? CH : 1], xv[PFM == 1 ? CH : 1], ov[PFM == 1 ? CH : 1];
                    if constexpr (PF) {
                        cp_async_wait_all();
                        __syncwarp();
                    }
                    if constexpr (PFM == 1) {
#pragma unroll
                        for (int c = 0; c < CH; ++c) {
                            const int k = lane + 32 * c;
                            lv[c] = pbl[k];
                            xv[c] = dx(pbx + k, k);
                            if constexpr (!LATE_OK) ov[c] = down(pbo + k, r);
                        }
                        __syncwarp();
                        if (r + RSTEP < s) prefetch(r + RSTEP, jrow + 1);
                    }
                    // the row's prior, incoming message and own output at column lane + 32 c
                    auto LV = [&](int c) -> T {
                        if constexpr (PFM == 1) return lv[c];
                        else if constexpr (PFM == 2) return pbl[lane + 32 * c];
                        else return lrow[lane + 32 * c];
                    };
                    auto XV = [&](int c) -> T {
                        if constexpr (PFM == 1) return xv[c];
                        else if constexpr (PFM == 2) return dx(pbx + lane + 32 * c, lane + 32 * c);
                        else return dx(xrow + lane + 32 * c, lane + 32 * c);
                    };
                    auto OV = [&](int c) -> T {
                        if constexpr (PFM == 1) return ov[c];
                        else if constexpr (PFM == 2) return down(pbo + lane + 32 * c, r);
                        else return down(orow + lane + 32 * c, r);
                    };
                    // one pass over the row: Q = l + M[k][r]/alpha and its maximum, second
                    // maximum and argmax; with the fused decisions also the kept count of
                    // lambda^t = l + (M[r][k] + M[k][r]) and a kept column (the only one when
                    // the count is 1, the case in which it is used)
                    T q[CH];
                    T m1 = ninf, m2 = ninf;
                    int am = 0x7fffffff;
                    int cnt = 0, kl = -1;
                    auto row_pass = [&](auto fused) {
#pragma unroll
                        for (int c = 0; c < CH; ++c) {
                            const int k = lane + 32 * c;
                            const T lv = LV(c), xv = XV(c);
                            if constexpr (decltype(fused)::value) {
                                const T lam = lv + (OV(c) + xv);
                                const bool kp = lam > T(0);
                                cnt += kp ? 1 : 0;
                                kl = kp ? k : kl;
                            }
                            const T v = B2<T>::fma_(xv, ainv, lv);
                            q[c] = v;
                            const bool gt = v > m1;
                            m2 = B2<T>::mx(m2, B2<T>::mn(v, m1));
                            m1 = B2<T>::mx(m1, v);
                            am = gt ? k : am;
                        }
                    };
                    if (fuse)
                        row_pass(std::true_type{});
                    else
                        row_pass(std::false_type{});
                    if constexpr (PFM == 2) {
                        // the last read of this row's incoming messages (and, without late
                        // judging, of its priors): the next row may replace them
                        __syncwarp();
                        if (r + RSTEP < s) prefetch(r + RSTEP, jrow + 1);
                    }
#pragma unroll
                    for (int off = 16; off; off >>= 1) {
                        const T o1 = __shfl_xor_sync(kFull, m1, off);
                        const T o2 = __shfl_xor_sync(kFull, m2, off);
                        const int ok = __shfl_xor_sync(kFull, am, off);
                        combine_max(m1, m2, am, o1, o2, ok);
                    }
                    if (fuse) {
#pragma unroll
                        for (int off = 16; off; off >>= 1) {
                            cnt += __shfl_xor_sync(kFull, cnt, off);
                            kl = max(kl, __shfl_xor_sync(kFull, kl, off));
                        }
                        if (lane == 0) bcast(&choice[r], kl >= 0 ? kl : 0x7fffffff);
                        ok_w &= (cnt == 1);
                    }
                    if (eval && lane == 0) {
                        rstat[r] = make_float2((float)m1, (float)m2);
                        order[r] = (short)am;
                    }
                    T S = T(0);
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        const T u = B2<T>::ex2(B2<T>::mn(q[c], m2) - m2);
                        q[c] = u;
                        S += u;
                    }
                    S = warp_sum(S);
                    const T cf = B2<T>::ex2(m2 - m1);
                    const T Aa = B2<T>::fma_(cf, S - T(1), T(1));
                    if constexpr (HALF) {
                        // stored values out + r_r; the stage keeps the rounded value (exact in FP32)
                        const float rf = IO::unpack(IO::pack(m1, 0.f)).x, dref = rf - m1;
#pragma unroll
                        for (int c = 0; c < CH; ++c) {
                            const int k = lane + 32 * c;
                            const float sr = IO::unpack(IO::pack(__fmaf_rn(B2<float>::lg2(__fmaf_rn(-cf, q[c], Aa)), -1.f, dref), 0.f)).x;
                            orow[k] = MS(sr);  // exact: sr is a value of the format
                            srow[k] = sr;
                        }
                        if ((am & 31) == lane) {
                            const float sr = IO::unpack(IO::pack(__fmaf_rn(B2<float>::lg2(S - 1.f), -1.f, rf - m2), 0.f)).x;
                            orow[am] = MS(sr);
                            srow[am] = sr;
                        }
                        __syncwarp();
                        if (lane == 0) {
                            srow[r] = rf;  // the diagonal of Mt holds r_r, which decodes to 0
                            bcast(&nrn[r], -rf);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < CH; ++c) {
                            const int k = lane + 32 * c;
                            const T out = -m1 - B2<T>::lg2(B2<T>::fma_(-cf, q[c], Aa));
                            if (!eval) orow[k] = out;
                            srow[k] = out;
                        }
                        if ((am & 31) == lane) {
                            const T oam = -m2 - B2<T>::lg2(S - T(1));
                            if (!eval) orow[am] = oam;
                            srow[am] = oam;
                        }
                        __syncwarp();
                        if constexpr (LATE_OK) {
                            if (eval) {
                                // lambda^(t+1) of v_rr and of v_rk for the rows k whose transposed
                                // messages are complete in Mn (batches before b; with two stages
                                // before b - 1: batch b - 1 is judged after the barrier below)
                                const int kend = (NST == 2 ? b - 1 : b) * W;
#pragma unroll
                                for (int c = 0; c < CH; ++c) {
                                    const int k = lane + 32 * c;
                                    if (k < kend) {
                                        const float own = srow[k], lk = LV(c);
                                        const float2 st = rstat[k];
                                        const float bnd = lk + (own + -((int)order[k] == r ? st.y : st.x));
                                        if (bnd > -1e-3f) {
                                            const float lam = lk + (own + __ldcg(reinterpret_cast<const float*>(Mn) + (size_t)r * LD + k));
                                            if (lam > 0.f) kept(kc, r, k);
                                        }
                                    } else if (k == r) {
                                        if (LV(c) + (srow[r] + 0.f) > 0.f) kept(kc, r, r);
                                    }
                                }
                                __syncwarp();
                            }
                        }
                        if (lane == 0) srow[r] = T(0);  // the diagonal of Mt stays 0
                    }
                    ++jrow;
                }
                __syncthreads();
                if constexpr (LATE_OK) {
                    if (eval && r < s) {
                        // this batch's variables v_rk with k in the same batch (k < r): both
                        // messages are in the stage
                        const float* lrw = reinterpret_cast<const float*>(Lg) + (size_t)r * LD;
                        if (lane < warp) {
                            const int k = b * W + lane;
                            const float lam = __ldcg(lrw + k) + (srow[k] + stage[lane * SP + r]);
                            if (lam > 0.f) kept(kc, r, k);
                        }
                        // with two stages, those with k in batch b - 1, whose transposed messages
                        // are complete now (same bound as above)
                        if (NST == 2 && b > 0 && lane < W) {
                            const int k = (b - 1) * W + lane;
                            const float own = srow[k], lk = __ldcg(lrw + k);
                            const float2 st = rstat[k];
                            const float bnd = lk + (own + -((int)order[k] == r ? st.y : st.x));
                            if (bnd > -1e-3f) {
                                const float lam = lk + (own + __ldcg(reinterpret_cast<const float*>(Mn) + (size_t)r * LD + k));
                                if (lam > 0.f) kept(kc, r, k);
                            }
                        }
                    }
                }
                // transposed write of the batch: Mn[k][b*W + w] = stage[w][k]
                const int r0 = b * W;
                const int rows = min(W, s - r0);
                if (sizeof(T) == 4 && rows == W) {
                    // a full batch: four consecutive rows of one column per thread, one
                    // 16-byte (FP32) or 8-byte (16-bit) store
                    constexpr int W4 = W / 4;
                    for (int e = tid; e < s * W4; e += NTH) {
                        const int k = e / W4, w = (e - k * W4) * 4;
                        const T* sp = stage + w * SP + k;
                        st4(Mn + (size_t)k * LD + r0 + w, sp[0], sp[SP], sp[2 * SP], sp[3 * SP]);
                    }
                } else {
                    for (int e = tid; e < s * W; e += NTH) {
                        const int k = e / W, w = e % W;
                        if (w < rows) Mn[(size_t)k * LD + r0 + w] = MS(stage[w * SP + k]);
                    }
                }
                // one stage: the next batch may overwrite it only after this write; two stages:
                // the next batch writes the other one, and the barrier after its rows (which
                // every thread reaches only after this write) protects this one
                if (NST == 1) __syncthreads();
            }
            if constexpr (LATE_OK) {
                if (eval) {
                    // every variable of lambda^(t+1) judged: converged iff every row keeps one
                    __syncthreads();
                    int ok = 1;
                    for (int r = tid; r < s; r += NTH) ok &= (((kc[r >> 1] >> ((r & 1) * 16)) & 0xFFFFu) == 1u);
                    if (__syncthreads_and(ok)) {
                        any_conv = true;
                        int pc = 0;
                        for (int r = tid; r < s; r += NTH) {
                            const int k = choice[r];
                            if (k >= r) pc ^= ic.tb.P[(size_t)dets[r] * n + dets[k]];
                        }
                        out_par = __syncthreads_count(pc) & 1;
                        out_forced = 0;
                        ++t;
                        break;
                    }
                }
            }
            int fconv;
            if constexpr (CL > 1) {
                // every block's transposed writes, choices and references precede every read
                // of the next iteration
                if (fuse) {
                    const int cta_ok = __syncthreads_and(ok_w);
                    if (tid == 0) bcast(&sh_votes[t & 1][crank], cta_ok);
                }
                csync();
                fconv = fuse;
#pragma unroll
                for (int q = 0; q < CL; ++q) fconv &= sh_votes[t & 1][q];
            } else {
                if (NST == 2) __syncthreads();  // the last batch's transposed write precedes every read of Mn
                fconv = fuse && __syncthreads_and(ok_w);
            }
            if (fconv) {
                // lambda^t converged: its matching is the output (the update just made is unused)
                any_conv = true;
                int pc = 0;
                for (int r = tid; r < s; r += NTH) {
                    const int k = choice[r];
                    if (k >= r) pc ^= ic.tb.P[(size_t)dets[r] * n + dets[k]];
                }
                out_par = __syncthreads_count(pc) & 1;
                out_forced = 0;
                break;
            }
            cur ^= 1;
            ++t;
        }
        if (tr_on && a.tr_partner) {
            for (int r = tid; r < a.s_cap; r += NTH) {
                int pk = -1;
                if (r < s) pk = out_from_best ? (int)bestp[r] : choice[r];
                a.tr_partner[(size_t)shot * a.s_cap + r] = (int16_t)pk;
            }
        }
        if (tid == 0 && crank == 0) {
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
    if (tid == 0 && crank == 0 && a.ctr) {
        atomicAdd(a.ctr + C_ITERS, acc_it);
        atomicAdd(a.ctr + C_MSGS, acc_msg);
        atomicAdd(a.ctr + C_DEFECTS, acc_def);
        atomicAdd(a.ctr + C_TIER_MSGS + a.tier, acc_msg);
        atomicAdd(a.ctr + C_TIER_SHOTS + a.tier, acc_shots);
        atomicAdd(a.ctr + C_FC_RUNS, acc_fc);
        atomicAdd(a.ctr + C_FC_ROUNDS, acc_fcr);
    }
}


// Dynamic shared memory of one streaming block.
template <typename T, int CH, typename MS, int CL = 1>
size_t stream_smem_bytes() {
    return stream_smem_bytes_n<T, CH, MS, CL>(kStreamStages<T, CH, MS, CL>);
}

template <typename T, int CH, typename MS = T>
cudaError_t run_stream(const DecodeArgs& a, int slots, cudaStream_t st) {
    constexpr int W = kStreamWarpsOf<T, CH>;
    const size_t smem = stream_smem_bytes<T, CH, MS>();
    const bool tr = a.tr_lambda != nullptr || a.tr_partner != nullptr;
    auto kern = tr ? decode_stream_kernel<T, CH, true, W, MS> : decode_stream_kernel<T, CH, false, W, MS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<slots, W * 32, smem, st>>>(a);
    return cudaGetLastError();
}

// Cluster form: the largest number of clusters of CL blocks that can be resident at once
// on the current device (0 if none), cached per device.
template <typename T, int CH, typename MS, int CL>
int stream_cluster_capacity() {
    static_assert(CL > 1, "cluster form");
    constexpr int kDev = 16;
    static std::atomic<int> cache[kDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    if (dev < kDev) {
        const int v = cache[dev].load();
        if (v > 0) return v - 1;
    }
    constexpr int W = kStreamWarpsOf<T, CH, CL>;
    const size_t smem = stream_smem_bytes<T, CH, MS, CL>();
    auto kern = decode_stream_kernel<T, CH, false, W, MS, CL>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (CL > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(W * 32);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        n = 0;
    }
    if (dev < kDev) cache[dev].store(n + 1);
    return n;
}

// Launches min(slots, capacity) clusters of CL blocks; the caller's scratch holds `slots`
// slots of stream_slot_bytes (one per cluster).
template <typename T, int CH, typename MS, int CL>
cudaError_t run_stream_cluster(const DecodeArgs& a, int slots, cudaStream_t st) {
    const int cap = stream_cluster_capacity<T, CH, MS, CL>();
    if (cap <= 0) return cudaErrorInvalidConfiguration;
    const int clusters = slots < cap ? slots : cap;
    if (clusters <= 0) return cudaSuccess;
    constexpr int W = kStreamWarpsOf<T, CH, CL>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * CL));
    cfg.blockDim = dim3(W * 32);
    cfg.dynamicSmemBytes = stream_smem_bytes<T, CH, MS, CL>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, decode_stream_kernel<T, CH, false, W, MS, CL>, a);
}

}  // namespace
}  // namespace bp4m
