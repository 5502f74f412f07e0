#pragma once
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
// the factor k side; Lm[i][k] = l_ik.  With 16-bit message storage every message leaving
// factor k is stored relative to a per-row reference r_k (the row's largest Q of that
// update, rounded to the 16-bit format): Mt[i][k] holds M[k][i] + r_k, which lies in
// [-lg2(s), 0] for every column but the row's argmax, so the 11-bit (FP16) or 8-bit (BF16)
// mantissa resolves the message to a few 1e-4 instead of a few 1e-2 of its magnitude; the
// reader adds -r_k (kept in FP32 per row).  The diagonal holds r_k itself, which decodes
// to exactly 0.  Row i is processed by G threads, thread g taking
// the columns of col_off() (FP32: adjacent pairs 2g, 2g+1, then every 2G; FP64: g + G*c).  The update is in place: every thread caches its row in registers,
// the block synchronises, then each thread writes its outputs M'[i][k] into Mt[k][i].
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <type_traits>
#include <atomic>

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
__host__ __device__ constexpr int min_blocks(int nt) { return 65536 / (nt * 128) > 1 ? 65536 / (nt * 128) : 1; }

// Base-2 transcendental helpers of the shared-memory tiers: messages are kept in log2
// units (every prior is scaled by log2(e) when gathered), so exp and log are single
// ex2/lg2 operations.
template <typename T>
struct B2;

template <>
struct B2<float> {
    static __device__ __forceinline__ float ex2(float x) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float lg2(float x) {
        float y;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float fma_(float a, float b, float c) { return fmaf(a, b, c); }
    static __device__ __forceinline__ float mx(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float mn(float a, float b) { return fminf(a, b); }
};

template <>
struct B2<double> {
    static __device__ __forceinline__ double ex2(double x) { return exp2(x); }
    static __device__ __forceinline__ double lg2(double x) { return log2(x); }
    static __device__ __forceinline__ double fma_(double a, double b, double c) { return fma(a, b, c); }
    static __device__ __forceinline__ double mx(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ double mn(double a, double b) { return fmin(a, b); }
};

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kLn2 = 0.69314718055994530942;

// Column ownership.  FP32 (PAIR): thread g of a row owns adjacent column pairs, its
// register c holding column k0 + col_off(c) with k0 = 2g and col_off(c) = (c & 1) +
// 2G (c >> 1), so that one 64-bit shared load fetches both columns of a pair.  FP64:
// k0 = g, col_off(c) = G c.
template <bool PAIR, int G>
__host__ __device__ constexpr int col_off(int c) {
    return PAIR ? ((c & 1) + 2 * G * (c >> 1)) : G * c;
}
template <bool PAIR, int G>
__host__ __device__ constexpr int owner_of(int k) {
    return PAIR ? ((k >> 1) % G) : (k % G);
}
template <bool PAIR, int G>
__host__ __device__ constexpr int reg_of(int k) {
    return PAIR ? (2 * (k / (2 * G)) + (k & 1)) : (k / G);
}

// Row pitch in elements.  FP32: pitch = GP x odd (GP = max(G, 2)), the smallest such value
// >= smax.  Then both shared-memory access shapes are conflict free: a half warp's 64-bit
// row read (32/G rows x G pairs) starts the rows in distinct 4-byte bank groups, and a
// warp's transposed write or read (G rows k = 2g + b, G apart by 2, x 32/G consecutive
// rows i) places the G rows 2 x pitch = 8 x odd banks apart (G = 4).  FP64: smax + 1.
template <typename T>
__host__ __device__ constexpr int pitch_of(int smax, int g) {
    return sizeof(T) == 8 ? smax + 1 : (g < 2 ? 2 : g) * (((smax + (g < 2 ? 2 : g) - 1) / (g < 2 ? 2 : g)) | 1);
}

// Storage of the message matrix.  MS = T keeps messages in the arithmetic type; MS = __half
// or __nv_bfloat16 (with T = float) stores them in 16 bits, converted with round to nearest
// and saturation to the largest finite value on the way in, and exactly to FP32 on the way
// out; all arithmetic stays FP32.
template <typename MS, typename T>
struct MsgIO {
    static __device__ __forceinline__ T ld(const MS* p) { return *p; }
    static __device__ __forceinline__ void st(MS* p, T v) { *p = v; }
    static __device__ __forceinline__ T zero_store() { return T(0); }
};

template <>
struct MsgIO<__half, float> {
    static __device__ __forceinline__ float ld(const __half* p) { return __half2float(*p); }
    static __device__ __forceinline__ float2 ld2(const __half* p) {
        return __half22float2(*reinterpret_cast<const __half2*>(p));
    }
    // pack (lo, hi) with saturation; returns the packed pair
    static __device__ __forceinline__ unsigned pack(float lo, float hi) {
        unsigned r;
        asm("cvt.rn.satfinite.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
        return r;
    }
    static __device__ __forceinline__ float2 unpack(unsigned r) {
        return __half22float2(*reinterpret_cast<const __half2*>(&r));
    }
    static __device__ __forceinline__ void st(__half* p, float v) {
        const unsigned r = pack(v, 0.f);
        *reinterpret_cast<unsigned short*>(p) = (unsigned short)(r & 0xFFFFu);
    }
};

template <>
struct MsgIO<__nv_bfloat16, float> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float2 ld2(const __nv_bfloat16* p) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    }
    static __device__ __forceinline__ unsigned pack(float lo, float hi) {
        unsigned r;
        asm("cvt.rn.satfinite.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
        return r;
    }
    static __device__ __forceinline__ float2 unpack(unsigned r) {
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) {
        const unsigned r = pack(v, 0.f);
        *reinterpret_cast<unsigned short*>(p) = (unsigned short)(r & 0xFFFFu);
    }
};

// Pitch of the message matrix in elements.  16-bit storage: 2G x odd, so that the 32-bit
// pair reads of a warp (32/G rows x G pairs) and its transposed 16-bit writes (G rows,
// 2 apart, x 32/G consecutive columns) are free of bank conflicts.
template <typename T, typename MS>
__host__ __device__ constexpr int msg_pitch_of(int smax, int g) {
    return sizeof(MS) == 2 ? 2 * g * (((smax + 2 * g - 1) / (2 * g)) | 1) : pitch_of<T>(smax, g);
}

// Byte offset of the 16-bit path's reference array in the dynamic shared memory, after
// Mt, Lm, Dg, rowacc, dets, choice, bestp and matched (8-byte aligned).
template <typename T, typename MS>
__host__ __device__ constexpr size_t nref_offset(int smax, int g) {
    return (((size_t)smax * msg_pitch_of<T, MS>(smax, g) * sizeof(MS) + 15) / 16 * 16 +
            (size_t)(smax * pitch_of<T>(smax, g) + smax + (smax & 1)) * sizeof(T) +
            (size_t)smax * (sizeof(double) + 2 * sizeof(int) + sizeof(short) + 1) + 7) / 8 * 8;
}

// A thread's register-cached row entries (CH columns).  FP32 keeps them as float2 pairs,
// columns (2j, 2j+1) in one 64-bit register pair, so that the packed FP32x2 add and FMA of
// sm_100 and later apply to two columns per instruction.
template <typename T, int N>
struct Regs {
    T v[N];
    __device__ __forceinline__ T& operator[](int c) { return v[c]; }
    // runtime column index: a select chain, so that the array stays in registers
    __device__ __forceinline__ T get(int c) const {
        T r = T(0);
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k == c) r = v[k];
        return r;
    }
};

template <int N>
struct Regs<float, N> {
    static_assert(N % 2 == 0, "FP32 rows are cached in column pairs");
    float2 p[N / 2];
    __device__ __forceinline__ float& operator[](int c) { return (c & 1) ? p[c >> 1].y : p[c >> 1].x; }
    __device__ __forceinline__ float get(int c) const {
        float r = 0.f;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (k == c) r = (k & 1) ? p[k >> 1].y : p[k >> 1].x;
        return r;
    }
};

// 1 if lambda > 0, else 0 (NaN and -0 give 0), on the FMA pipe: saturate(lambda x 2^64).
// A positive lambda below 2^-64 would give a fraction; such a lambda is a tie by any margin
// the decoder distinguishes.
__device__ __forceinline__ float keep_f(float lam) { return __saturatef(__fmul_rn(lam, 0x1p64f)); }

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// (max, second max, column of the max) of two partial row scans; ties go to the smaller
// column.  Commutative, so every thread of a row group ends with the same triple.
template <typename T>
__device__ __forceinline__ void combine_max(T& m1, T& m2, int& k, T o1, T o2, int ok) {
    if (o1 > m1 || (o1 == m1 && ok < k)) {
        m2 = B2<T>::mx(m1, o2);
        m1 = o1;
        k = ok;
    } else {
        m2 = B2<T>::mx(m2, o1);
    }
}

// Blocks per SM the kernel is compiled for: the FP32 384- and 448-thread tiers (96 and 112
// rows, 79 and 106 KB of shared memory) run two blocks per SM, and so does the 512-thread
// tier (128 rows) with 16-bit messages (102 KB); the others are limited by shared memory or
// 128 registers.
__host__ __device__ constexpr int blocks_for(int nt, int elem_bytes, int msg_bytes) {
    return (elem_bytes == 4 && (nt == 384 || nt == 448 || (nt == 512 && msg_bytes == 2))) ? 2 : min_blocks(nt);
}

// REG = true keeps each thread's own outputs M[i][k] in registers between iterations (no
// strided shared-memory read per message); REG = false reads them back from Mt[k][i].
// RW = true: the B-BP4MF second stage.  The shot's priors, pair weights and parities are
// computed in the block by Dijkstra from every defect over per-qubit weights derived from
// the first stage's posteriors (instead of being gathered from the static tables).
template <typename T, int CH, int G, bool TRACE, bool REG, bool RW = false, typename MS = T>
__global__ void __launch_bounds__(CH * G * G, blocks_for(CH * G * G, (int)sizeof(T), (int)sizeof(MS))) decode_smem_kernel(const DecodeArgs a) {
    constexpr int SMAX = CH * G;
    constexpr int NT = SMAX * G;
    constexpr int R = 32 / G;
    constexpr int P = pitch_of<T>(SMAX, G);          // priors
    constexpr int PM = msg_pitch_of<T, MS>(SMAX, G);  // messages
    constexpr bool HALF = sizeof(MS) == 2;
    static_assert(!HALF || sizeof(T) == 4, "16-bit messages use FP32 arithmetic");
    using IO = MsgIO<MS, T>;
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    using Mask = typename std::conditional<(CH > 32), unsigned long long, unsigned int>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    MS* Mt = reinterpret_cast<MS*>(smem);        // Mt[i][k] = M[k][i]; diagonal kept 0
    T* Lm = reinterpret_cast<T*>(smem + ((size_t)SMAX * PM * sizeof(MS) + 15) / 16 * 16);  // Lm[i][k] = l_ik (log2), -inf past s
    T* Dg = Lm + SMAX * P;                          // Dg[i] = M[i][i] (factor i to its boundary variable)
    double* rowacc = reinterpret_cast<double*>(Dg + SMAX + (SMAX & 1));
    int* dets = reinterpret_cast<int*>(rowacc + SMAX);
    int* choice = dets + SMAX;
    short* bestp = reinterpret_cast<short*>(choice + SMAX);
    unsigned char* matched = reinterpret_cast<unsigned char*>(bestp + SMAX);
    // 16-bit messages: nrefv[k] = -r_k, minus the reference of the messages leaving factor k
    float* nrefv = reinterpret_cast<float*>(smem + nref_offset<T, MS>(SMAX, G));
    // static-partition forced convergence: factors in processing order
    short* order = reinterpret_cast<short*>(smem + nref_offset<T, MS>(SMAX, G) + (HALF ? (size_t)SMAX * 4 : 0));
    // RW only: per-shot W (FP64) and parity over local ranks, Dijkstra state per warp, in
    // this block's global scratch slot (layout of rw_slot_layout)
    const int rw_nodes = a.tb.n_det + 1;
    unsigned char* rw_slot = RW ? reinterpret_cast<unsigned char*>(a.gscratch) + (size_t)blockIdx.x * a.rw_slot_bytes
                                : nullptr;
    double* Wsh = reinterpret_cast<double*>(rw_slot);
    double* rw_dist = Wsh + SMAX * SMAX;
    unsigned char* Psh = reinterpret_cast<unsigned char*>(rw_dist + (NT / 32) * rw_nodes);
    unsigned char* rw_done = Psh + SMAX * SMAX;
    unsigned char* rw_par = rw_done + (NT / 32) * rw_nodes;
    __shared__ int sh_item, sh_s, sh_best_par, sh_best_forced, sh_improve, sh_use_best;
    __shared__ double sh_best_w;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i = warp * R + (lane % R);   // row (factor) of this thread
    const int g = lane / R;                // column group of this thread within the row
    constexpr bool PAIR = sizeof(T) == 4;
    const int k0 = PAIR ? 2 * g : g;       // first column of this thread
    const bool own_diag = owner_of<PAIR, G>(i) == g;   // this thread holds column k = i of its row
    const int c_diag = reg_of<PAIR, G>(i);
    const int count = *a.count;
    const T ainv = (T)(1.0 / a.alpha);
    const bool full = (a.decoder == 1) || !a.early_exit;
    T* trl = reinterpret_cast<T*>(a.tr_lambda);
    const T ninf = Num<T>::ninf();
    // counters of this block's shots: updated by thread 0 only, so kept in shared memory rather
    // than in twelve registers of every thread
    __shared__ unsigned long long sh_acc[6];
    unsigned long long &acc_it = sh_acc[0], &acc_msg = sh_acc[1], &acc_def = sh_acc[2], &acc_shots = sh_acc[3],
                       &acc_fc = sh_acc[4], &acc_fcr = sh_acc[5];
    if (tid == 0)
        for (int k = 0; k < 6; ++k) sh_acc[k] = 0;

    T* const row_l = Lm + i * P + k0;    // priors l_ik, register c at [col_off(c)]
    MS* const row_m = Mt + i * PM + k0;  // incoming messages M[k][i]
    MS* const col_m = Mt + k0 * PM + i;  // own outputs M[i][k] live at Mt[k][i], register c at [col_off(c) PM]
#define COL(c) (k0 + col_off<PAIR, G>(c))
#define RL(c) row_l[col_off<PAIR, G>(c)]
#define RM(c) m_ld1(row_m + col_off<PAIR, G>(c), COL(c))
#define CMP(c) (col_m + col_off<PAIR, G>(c) * PM)
#define CM(c) m_ld1(CMP(c), i)
#define RL2(j) (*reinterpret_cast<const float2*>(row_l + col_off<PAIR, G>(2 * (j))))
#define RM2(j) m_ld2(row_m + col_off<PAIR, G>(2 * (j)), k0 + col_off<PAIR, G>(2 * (j)))
    // messages arriving at row i from columns k, k + 1 (16-bit: decoded with the source rows'
    // references), and one arriving from column k
    auto m_ld2 = [&](const MS* p, int k) -> float2 {
        if constexpr (HALF)
            return __fadd2_rn(IO::ld2(p), *reinterpret_cast<const float2*>(nrefv + k));
        else
            return *reinterpret_cast<const float2*>(p);
    };
    auto m_ld1 = [&](const MS* p, int k) -> T {
        if constexpr (HALF)
            return IO::ld(p) + nrefv[k];
        else
            return IO::ld(p);
    };

    for (;;) {
        if (tid == 0) sh_item = atomicAdd(a.next, 1);
        __syncthreads();
        const int item = sh_item;
        if (item >= count) break;
        const ItemCtx ic = resolve_item(a, a.list[item]);
        const int64_t shot = ic.shot;
        const int n = ic.tb.n_det;
        const T* __restrict__ Ltab = Num<T>::L(ic.tb);
        if (warp == 0) {
            const int s0 = compact_defects(ic.synd + (size_t)shot * ic.tb.n_words, ic.tb.n_words,
                                           dets, SMAX, lane);
            if (lane == 0) sh_s = s0;
        }
        __syncthreads();
        const int s = sh_s;
        if (s > SMAX || s < 1) {
            if (tid == 0 && a.ctr) atomicAdd(a.ctr + C_ERRORS, 1ull);
            continue;
        }
        const bool tr_on = TRACE && s <= a.s_cap;
        if (s == 1 && !RW) {
            // a single factor with a single variable: the leave-one-out set is empty, the
            // message is +inf and v_00 is kept in every iteration
            if (tid == 0) {
                const int its = full ? a.T : 1;
                const int d0 = dets[0];
                if (ic.obs_pred) ic.obs_pred[shot] = ic.tb.P[(size_t)d0 * n + d0];
                if (ic.flags) ic.flags[shot] = F_CONVERGED;
                if (ic.iters) ic.iters[shot] = (int16_t)its;
                if (tr_on && trl) trl[(size_t)shot * a.s_cap * a.s_cap] = Num<T>::pinf();
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
        // ---- gather the shot's priors (log2 units); columns past s are -inf so that they
        // never win a max, add nothing to a sum and are never kept
        if (!RW) {
            for (int r = warp; r < s; r += NT / 32) {
                const T* trow = Ltab + (size_t)dets[r] * n;
                for (int k = lane; k < SMAX; k += 32) {
                    Lm[r * P + k] = k < s ? (T)(__ldg(trow + dets[k]) * (T)kLog2e) : ninf;
                    Mt[r * PM + k] = MS(0.f);
                }
            }
        } else {
            // Dijkstra from every defect (one warp per source): nodes popped in (distance,
            // index) order, predecessor changed only on a strict improvement, the boundary
            // node n a sink; edge weight |ln((1-P)/P)| of the qubit behind the edge (edges
            // above one half were flipped out of the syndrome), floored at kRwMinWeight
            double* dist = rw_dist + warp * rw_nodes;
            unsigned char* done = rw_done + warp * rw_nodes;
            unsigned char* par = rw_par + warp * rw_nodes;
            const double* post = a.rw_post + (size_t)shot * a.rw_units;
            const double dinf = Num<double>::pinf();
            for (int r = warp; r < s; r += NT / 32) {
                for (int v = lane; v < rw_nodes; v += 32) {
                    dist[v] = dinf;
                    done[v] = 0;
                    par[v] = 0;
                }
                __syncwarp();
                if (lane == 0) dist[dets[r]] = 0.0;
                __syncwarp();
                for (int step = 0; step < rw_nodes; ++step) {
                    double bd = dinf;
                    int bi = 0x7fffffff;
                    for (int v = lane; v < rw_nodes; v += 32)
                        if (!done[v] && dist[v] < bd) {
                            bd = dist[v];
                            bi = v;
                        }
#pragma unroll
                    for (int off = 16; off; off >>= 1) {
                        const double od = __shfl_xor_sync(kFull, bd, off);
                        const int oi = __shfl_xor_sync(kFull, bi, off);
                        if (od < bd || (od == bd && oi < bi)) {
                            bd = od;
                            bi = oi;
                        }
                    }
                    if (bd == dinf) break;
                    if (lane == 0) {
                        done[bi] = 1;
                        if (bi != n) {
                            for (int e = a.rw_off[bi]; e < a.rw_off[bi + 1]; ++e) {
                                const uint32_t pk = a.rw_adj[e];
                                const int v = (int)(pk & 0x7FFFu);
                                double pq = post[(pk >> 15) & 0x7FFFu];
                                pq = pq < 1e-300 ? 1e-300 : (pq > 1.0 - 1e-16 ? 1.0 - 1e-16 : pq);
                                // an edge above one half was taken as present (flipped out of
                                // the syndrome): it weighs as its complement
                                if (pq > 0.5) pq = 1.0 - pq;
                                const double nd = bd + fmax(log((1.0 - pq) / pq), kRwMinWeight);
                                if (nd < dist[v]) {
                                    dist[v] = nd;
                                    par[v] = par[bi] ^ (unsigned char)(pk >> 31);
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
                for (int k = r + lane; k < s; k += 32) {
                    const int tgt = k == r ? n : dets[k];
                    Wsh[r * SMAX + k] = dist[tgt];
                    Psh[r * SMAX + k] = par[tgt];
                }
                __syncwarp();
            }
            __syncthreads();
            for (int r = warp; r < s; r += NT / 32) {
                for (int k = lane; k < SMAX; k += 32) {
                    if (k < s) {
                        if (k < r) {
                            Wsh[r * SMAX + k] = Wsh[k * SMAX + r];
                            Psh[r * SMAX + k] = Psh[k * SMAX + r];
                        }
                        const double W = k < r ? Wsh[k * SMAX + r] : Wsh[r * SMAX + k];
                        const double l = W == dinf ? -1.0e30 : -W - log1p(-exp(-W));
                        Lm[r * P + k] = (T)(l * kLog2e);
                    } else {
                        Lm[r * P + k] = ninf;
                    }
                    Mt[r * PM + k] = MS(0.f);
                }
            }
        }
        if (tid < SMAX) {
            Dg[tid] = T(0);
            matched[tid] = tid >= s;
            bestp[tid] = -1;
            if constexpr (HALF) nrefv[tid] = 0.f;
        }
        if (tid == 0) {
            sh_best_w = Num<double>::pinf();
            sh_best_par = 0;
            sh_best_forced = 0;
            sh_use_best = 0;
        }
        __syncthreads();
        if (RW && s == 1) {
            // one defect: matched to the boundary along its reweighted path
            if (tid == 0) {
                const int its = full ? a.T : 1;
                if (ic.obs_pred) ic.obs_pred[shot] = Psh[0];
                if (ic.flags) ic.flags[shot] = F_CONVERGED;
                if (ic.iters) ic.iters[shot] = (int16_t)its;
                acc_it += (unsigned long long)its;
                acc_msg += (unsigned long long)its;
                acc_def += 1;
                acc_shots += 1;
            }
            continue;
        }

        const bool act = i < s;
        // rows warp*R .. warp*R+R-1 belong to this warp; a warp with none of them active
        // skips the read and compute phases (it still takes part in every barrier)
        const bool wact = warp * R < s;
        Regs<T, CH> q;
        Regs<T, REG ? CH : 2> mo;
        int am_prev = -1;          // REG: argmax column of the previous update and its output
        T out_am = T(0);
        T out_am_gen = T(0);       // REG, FP32: the generic formula's value held in registers for it
        int t = 0;
        bool any_conv = false, forced_ran = false;
        int out_par = 0, out_forced = 0, out_from_best = 0;
        int partner = -1;

        for (;;) {
            // ---- read phase: Q = l + M[k][i]/alpha for the next update; for t > 0 the
            // marginalization of lambda^t = l + (M[i][k] + M[k][i]).  FP32: the row's
            // maximum / second maximum scan of the next update runs in the same loop (it needs
            // only Q), so that the shared-memory loads and the scan's ALU work overlap; the
            // scan is over columns in the same order as a separate pass, so its result is the
            // same
            Mask bits = 0;
            float cntf = 0.f;
            float sa1 = Num<float>::ninf(), sa2 = Num<float>::ninf();
            int sac = 0x7fffffff;
            auto scan_pair = [&](int j, float v, float w) {
                // (max, second max, column) of the pairs so far; ties to the smaller column
                const float hi = fmaxf(v, w), lo = fminf(v, w);
                const int ih = v >= w ? 2 * j : 2 * j + 1;
                const bool gt = hi > sa1;
                sa2 = max3f(sa2, lo, fminf(sa1, hi));
                sa1 = fmaxf(sa1, hi);
                sac = gt ? ih : sac;
            };
            if (!wact) {
            } else if (!act) {
#pragma unroll
                for (int c = 0; c < CH; ++c) q[c] = ninf;
            } else {
                if (t == 0) {
                    if constexpr (std::is_same<T, float>::value) {
                        const float2 ainv2 = make_float2(ainv, ainv);
#pragma unroll
                        for (int j = 0; j < CH / 2; ++j) {
                            q.p[j] = __ffma2_rn(RM2(j), ainv2, RL2(j));
                            scan_pair(j, q.p[j].x, q.p[j].y);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < CH; ++c) q[c] = B2<T>::fma_(RM(c), ainv, RL(c));
                    }
                } else if constexpr (std::is_same<T, float>::value) {
                    // two columns per packed instruction; same roundings as the scalar form.
                    // The kept count is a sum of keep(lambda) in {0, 1} on the FMA pipe; the
                    // kept column itself is found only when every row has exactly one
                    // (row_kept_column below).
                    const float2 ainv2 = make_float2(ainv, ainv);
                    float2 cnt2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < CH / 2; ++j) {
                        const int c = 2 * j;
                        const float2 l = RL2(j);
                        const float2 x = RM2(j);
                        float2 own;
                        if constexpr (REG)
                            own = mo.p[j];
                        else
                            own = make_float2(CM(c), CM(c + 1));
                        q.p[j] = __ffma2_rn(x, ainv2, l);
                        scan_pair(j, q.p[j].x, q.p[j].y);
                        const float2 lam = __fadd2_rn(l, __fadd2_rn(own, x));
                        cnt2 = __fadd2_rn(cnt2, make_float2(keep_f(lam.x), keep_f(lam.y)));
                        if (tr_on && trl && COL(c) < s)
                            trl[((size_t)shot * a.s_cap + i) * a.s_cap + COL(c)] = lam.x * (float)kLn2;
                        if (tr_on && trl && COL(c + 1) < s)
                            trl[((size_t)shot * a.s_cap + i) * a.s_cap + COL(c + 1)] = lam.y * (float)kLn2;
                    }
                    cntf = cnt2.x + cnt2.y;
                    if (!REG && own_diag) {
                        // the generic term used Mt[i][i] = 0 on both sides: lambda_ii = l_ii
                        const float lii = Lm[i * P + i];
                        const float lam = lii + Dg[i];
                        cntf += keep_f(lam) - keep_f(lii + (0.f + 0.f));
                        if (tr_on && trl) trl[((size_t)shot * a.s_cap + i) * a.s_cap + i] = lam * (float)kLn2;
                    }
                    if (REG && owner_of<PAIR, G>(am_prev) == g) {
                        // the register copy of the argmax column holds the generic output
                        const float l = Lm[i * P + am_prev], x = m_ld1(Mt + i * PM + am_prev, am_prev);
                        const float lam = l + (out_am + x);
                        cntf += keep_f(lam) - keep_f(l + (out_am_gen + x));
                        if (tr_on && trl) trl[((size_t)shot * a.s_cap + i) * a.s_cap + am_prev] = lam * (float)kLn2;
                    }
                } else {
                    Mask b0 = 0, b1 = 0;
#pragma unroll
                    for (int c = 0; c < CH; ++c) {
                        const T l = RL(c);
                        const T x = RM(c);
                        const T own = REG ? mo[REG ? c : 0] : CM(c);
                        q[c] = B2<T>::fma_(x, ainv, l);
                        const T lam = l + (own + x);
                        if (c & 1)
                            b1 |= (Mask)(lam > T(0) ? 1u : 0u) << c;
                        else
                            b0 |= (Mask)(lam > T(0) ? 1u : 0u) << c;
                        if (tr_on && trl && COL(c) < s)
                            trl[((size_t)shot * a.s_cap + i) * a.s_cap + COL(c)] = lam * (T)kLn2;
                    }
                    bits = b0 | b1;
                    if (!REG && own_diag) {
                        // the boundary variable v_ii: lambda_ii = l_ii + M[i][i]
                        const T lam = Lm[i * P + i] + Dg[i];
                        bits = (bits & ~((Mask)1 << c_diag)) | ((Mask)(lam > T(0) ? 1u : 0u) << c_diag);
                        if (tr_on && trl) trl[((size_t)shot * a.s_cap + i) * a.s_cap + i] = lam * (T)kLn2;
                    }
                    if (REG && owner_of<PAIR, G>(am_prev) == g) {
                        // the argmax column's own output is out_am, not the generic formula's
                        const int ca = reg_of<PAIR, G>(am_prev);
                        const T lam = Lm[i * P + am_prev] + (out_am + m_ld1(Mt + i * PM + am_prev, am_prev));
                        bits = (bits & ~((Mask)1 << ca)) | ((Mask)(lam > T(0) ? 1u : 0u) << ca);
                        if (tr_on && trl) trl[((size_t)shot * a.s_cap + i) * a.s_cap + am_prev] = lam * (T)kLn2;
                    }
                }
            }
            // FP32: the row's (m1, m2, argmax column) of the next update, over the G threads
            T m1 = ninf, m2 = ninf;
            int am = 0x7fffffff;
            if constexpr (std::is_same<T, float>::value) {
                if (wact) {
                    m1 = sa1;
                    m2 = sa2;
                    am = sac < CH ? COL(sac) : 0x7fffffff;
#pragma unroll
                    for (int off = R; off < 32; off <<= 1) {
                        const T o1 = __shfl_xor_sync(kFull, m1, off);
                        const T o2 = __shfl_xor_sync(kFull, m2, off);
                        const int ok = __shfl_xor_sync(kFull, am, off);
                        combine_max(m1, m2, am, o1, o2, ok);
                    }
                }
            }
            int cnt, chosen = -1;
            if constexpr (std::is_same<T, float>::value) {
#pragma unroll
                for (int off = R; off < 32; off <<= 1) cntf += __shfl_xor_sync(kFull, cntf, off);
                cnt = (int)cntf;
            } else {
                // kept count << 16 plus (first kept column + 1), summed over the row's G threads:
                // the count is exact, the column is the row's only kept one when the count is 1
                int pk = ((sizeof(Mask) == 8 ? __popcll((unsigned long long)bits) : __popc((unsigned)bits)) << 16) +
                         (bits ? COL((sizeof(Mask) == 8 ? __ffsll((long long)bits) : __ffs((int)bits)) - 1) + 1 : 0);
#pragma unroll
                for (int off = R; off < 32; off <<= 1) pk += __shfl_xor_sync(kFull, pk, off);
                cnt = pk >> 16;
                chosen = (pk & 0xFFFF) - 1;
            }
            const int conv = __syncthreads_and(t > 0 && (!act || cnt == 1));
            if constexpr (std::is_same<T, float>::value) {
                if (conv && wact) {
                    // every row keeps exactly one variable: find it (the same lambdas as above)
                    int k1 = -1;
                    if (act) {
#pragma unroll
                        for (int j = 0; j < CH / 2; ++j) {
                            const int c = 2 * j;
                            const float2 l = RL2(j);
                            const float2 x = RM2(j);
                            float2 own;
                            if constexpr (REG)
                                own = mo.p[j];
                            else
                                own = make_float2(CM(c), CM(c + 1));
                            float2 lam = __fadd2_rn(l, __fadd2_rn(own, x));
                            if (!REG && own_diag && c == c_diag) lam.x = Lm[i * P + i] + Dg[i];
                            if (!REG && own_diag && c + 1 == c_diag) lam.y = Lm[i * P + i] + Dg[i];
                            if (REG && owner_of<PAIR, G>(am_prev) == g) {
                                const float fix = Lm[i * P + am_prev] + (out_am + m_ld1(Mt + i * PM + am_prev, am_prev));
                                if (c == reg_of<PAIR, G>(am_prev)) lam.x = fix;
                                if (c + 1 == reg_of<PAIR, G>(am_prev)) lam.y = fix;
                            }
                            if (lam.x > 0.f) k1 = COL(c);
                            if (lam.y > 0.f) k1 = COL(c + 1);
                        }
                    }
#pragma unroll
                    for (int off = R; off < 32; off <<= 1) k1 = max(k1, __shfl_xor_sync(kFull, k1, off));
                    chosen = k1;
                }
            }

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
                    const T lii = act ? (REG ? Lm[i * P + i] + (mo.get(c_diag) + T(0)) : Lm[i * P + i] + Dg[i]) : ninf;
                    if (a.forced_static) {
                        // the paper's static partition: row i's block is v_ik, k >= i; its
                        // maximum (ties: smaller k) represents factor i; representatives are
                        // ranked by posterior (ties: smaller i) and processed in that order
                        T bl = ninf;
                        int bk = -1;
                        if (act) {
#pragma unroll
                            for (int c = 0; c < CH; ++c) {
                                const int k = COL(c);
                                if (k >= i && k < s) {
                                    const T own = REG ? mo[REG ? c : 0] : CM(c);
                                    T lam = RL(c) + (own + RM(c));
                                    if (!REG && k == i) lam = lii;
                                    if (REG && k == am_prev) lam = RL(c) + (out_am + RM(c));
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
                        if (act && g == 0) {
                            choice[i] = bk >= 0 ? bk : i;
                            rowacc[i] = (double)bl;
                        }
                        __syncthreads();
                        if (tid < s) {
                            const double v = rowacc[tid];
                            int rank = 0;
                            for (int j = 0; j < s; ++j) {
                                const double u = rowacc[j];
                                rank += (u > v || (u == v && j < tid)) ? 1 : 0;
                            }
                            order[rank] = (short)tid;
                        }
                        __syncthreads();
                        if (tid == 0) {
                            // a factor whose representative's other factor is taken goes to
                            // the boundary (a case the paper does not treat)
                            for (int r = 0; r < s; ++r) {
                                const int ii = order[r];
                                if (matched[ii]) continue;
                                const int k = choice[ii];
                                matched[ii] = 1;
                                if (k == ii || matched[k]) {
                                    choice[ii] = ii;
                                } else {
                                    matched[k] = 1;
                                    choice[k] = ii;
                                }
                            }
                            acc_fcr += 1;
                        }
                        __syncthreads();
                    }
                    for (int round = 0; round < s && !a.forced_static; ++round) {
                        const bool open = act && !matched[i];
                        T bl = ninf;
                        int bk = -1;
                        if (open) {
#pragma unroll
                            for (int c = 0; c < CH; ++c) {
                                const int k = COL(c);
                                if (k == i || !matched[k]) {
                                    const T own = REG ? mo[REG ? c : 0] : CM(c);
                                    T lam = RL(c) + (own + RM(c));
                                    if (!REG && k == i) lam = lii;
                                    if (REG && k == am_prev) lam = RL(c) + (out_am + RM(c));
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
                        if (tid == 0) acc_fcr += 1;
                        if (left == 0) break;
                    }
                    if (tid == 0) acc_fc += 1;
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
                            if (RW) {
                                pc = Psh[i * SMAX + k];
                                if (full) w = Wsh[i * SMAX + k];
                            } else {
                                const size_t off = (size_t)dets[i] * n + dets[k];
                                pc = ic.tb.P[off];
                                if (full) w = ic.tb.W64[off];
                            }
                        }
                        rowacc[i] = w;
                    }
                    const int par = __syncthreads_count(pc) & 1;
                    bool finish = false;
                    if (!full) {
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

            // ---- compute phase: leave-one-out max* of every row, in place.  With m1 (at
            // column am) and m2 the two largest Q of the row and S = sum_k 2^(min(Q_k, m2) - m2)
            // (the max clamped to m2, so S - 1 = sum_{k != am} 2^(Q_k - m2) >= 1):
            //   k != am: M'[i][k] = -(m1 + lg2(1 + 2^(m2 - m1) (S - 1 - 2^(Q_k - m2))))
            //   k == am: M'[i][k] = -(m2 + lg2(S - 1))
            // (the generic value is written for every column, the owner of am then overwrites;
            // row i's outputs M'[i][k] go to Mt[k][i]).  FP32: (m1, m2, am) come from the read
            // phase; FP64: from the scan below.
            if (wact) {
                if constexpr (std::is_same<T, float>::value) {
                    const float2 nm2 = make_float2(-m2, -m2);
                    float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < CH / 2; ++j) {
                        const float2 dq = __fadd2_rn(make_float2(fminf(q.p[j].x, m2), fminf(q.p[j].y, m2)), nm2);
                        const float2 u = make_float2(B2<float>::ex2(dq.x), B2<float>::ex2(dq.y));
                        q.p[j] = u;
                        s2 = __fadd2_rn(s2, u);
                    }
                    float S32 = s2.x + s2.y;
#pragma unroll
                    for (int off = R; off < 32; off <<= 1) S32 += __shfl_xor_sync(kFull, S32, off);
                    const float cf32 = B2<float>::ex2(m2 - m1);
                    const float Aa32 = __fmaf_rn(cf32, S32 - 1.f, 1.f);
                    // 16-bit storage: this row's reference r_i = m1 rounded to the format (so
                    // that it is exact there); stored values out + r_i = -lg2(Aa - cf u) + (r_i - m1)
                    float rf32 = 0.f, dref32 = 0.f;
                    if constexpr (HALF) {
                        rf32 = IO::unpack(IO::pack(m1, 0.f)).x;
                        dref32 = rf32 - m1;
                    }
                    if (act) {
                        const float rf = rf32;
                        // out = -m1 - lg2(Aa - cf u), the subtraction as an exact fma with -1
                        const float2 ncf = make_float2(-cf32, -cf32), A2 = make_float2(Aa32, Aa32);
                        const float2 nm1 = HALF ? make_float2(dref32, dref32) : make_float2(-m1, -m1);
                        const float2 neg1 = make_float2(-1.f, -1.f);
#pragma unroll
                        for (int j = 0; j < CH / 2; ++j) {
                            const float2 y = __ffma2_rn(ncf, q.p[j], A2);
                            const float2 lg = make_float2(B2<float>::lg2(y.x), B2<float>::lg2(y.y));
                            const float2 out = __ffma2_rn(lg, neg1, nm1);
                            if constexpr (HALF) {
                                // store the rounded pair (relative to r_i); the register copy is
                                // the stored value decoded as every reader decodes it, so that
                                // both ends of a variable see the same message
                                const unsigned pk2 = IO::pack(out.x, out.y);
                                *reinterpret_cast<unsigned short*>(CMP(2 * j)) = (unsigned short)(pk2 & 0xFFFFu);
                                *reinterpret_cast<unsigned short*>(CMP(2 * j + 1)) = (unsigned short)(pk2 >> 16);
                                if constexpr (REG) mo.p[j] = __fadd2_rn(IO::unpack(pk2), make_float2(-rf, -rf));
                            } else {
                                *CMP(2 * j) = out.x;
                                *CMP(2 * j + 1) = out.y;
                                if constexpr (REG) mo.p[j] = out;
                            }
                        }
                        float oam = -m2 - B2<float>::lg2(S32 - 1.f);
                        if constexpr (HALF) {
                            const float st_am = __fmaf_rn(B2<float>::lg2(S32 - 1.f), -1.f, rf - m2);
                            if (owner_of<PAIR, G>(am) == g) IO::st(Mt + am * PM + i, st_am);
                            oam = IO::unpack(IO::pack(st_am, 0.f)).x + (-rf);
                        } else if (owner_of<PAIR, G>(am) == g) {
                            IO::st(Mt + am * PM + i, oam);
                        }
                        if (REG) {
                            am_prev = am;
                            out_am = oam;
                            // what the packed output loop produced for the argmax column: u = ex2(0)
                            const float u0 = B2<float>::ex2(0.f);
                            float og = __fmaf_rn(B2<float>::lg2(__fmaf_rn(-cf32, u0, Aa32)), -1.f, HALF ? dref32 : -m1);
                            if constexpr (HALF) og = IO::unpack(IO::pack(og, 0.f)).x + (-rf);
                            out_am_gen = og;
                        }
                        if (own_diag) {
                            if constexpr (HALF) {
                                // the diagonal holds r_i, which decodes to exactly 0
                                if (!REG) Dg[i] = IO::ld(Mt + i * PM + i) + (-rf);
                                IO::st(Mt + i * PM + i, rf);
                                nrefv[i] = -rf;
                            } else {
                                if (!REG) Dg[i] = IO::ld(Mt + i * PM + i);
                                Mt[i * PM + i] = MS(0.f);
                            }
                        }
                    }
                } else {
                    T a1 = ninf, a2 = ninf, b1 = ninf, b2 = ninf;
                    int ac = 0x7fffffff, bc = 0x7fffffff;
#pragma unroll
                    for (int c = 0; c < CH; c += 2) {
                        const T v = q[c];
                        const bool gt = v > a1;
                        a2 = B2<T>::mx(a2, B2<T>::mn(v, a1));
                        a1 = B2<T>::mx(a1, v);
                        ac = gt ? c : ac;
                        if (c + 1 < CH) {
                            const T w = q[c + 1];
                            const bool gw = w > b1;
                            b2 = B2<T>::mx(b2, B2<T>::mn(w, b1));
                            b1 = B2<T>::mx(b1, w);
                            bc = gw ? c + 1 : bc;
                        }
                    }
                    // column indices of the two partial maxima (ties to the smaller column)
                    int ka = ac < CH ? COL(ac) : 0x7fffffff;
                    int kb = bc < CH ? COL(bc) : 0x7fffffff;
                    combine_max(a1, a2, ka, b1, b2, kb);
                    m1 = a1;
                    m2 = a2;
                    am = ka;
#pragma unroll
                    for (int off = R; off < 32; off <<= 1) {
                        const T o1 = __shfl_xor_sync(kFull, m1, off);
                        const T o2 = __shfl_xor_sync(kFull, m2, off);
                        const int ok = __shfl_xor_sync(kFull, am, off);
                        combine_max(m1, m2, am, o1, o2, ok);
                    }
                    // FP64 (16-bit storage runs only with FP32 arithmetic)
                    static_assert(!HALF, "16-bit storage is FP32 only");
                    T sa = T(0), sb = T(0);
#pragma unroll
                    for (int c = 0; c < CH; c += 2) {
                        const T u = B2<T>::ex2(B2<T>::mn(q[c], m2) - m2);
                        q[c] = u;
                        sa += u;
                        if (c + 1 < CH) {
                            const T w = B2<T>::ex2(B2<T>::mn(q[c + 1], m2) - m2);
                            q[c + 1] = w;
                            sb += w;
                        }
                    }
                    T S = sa + sb;
#pragma unroll
                    for (int off = R; off < 32; off <<= 1) S += __shfl_xor_sync(kFull, S, off);
                    const T cf = B2<T>::ex2(m2 - m1);
                    const T Aa = B2<T>::fma_(cf, S - T(1), T(1));
                    if (act) {
#pragma unroll
                        for (int c = 0; c < CH; ++c) {
                            const T out = -m1 - B2<T>::lg2(B2<T>::fma_(-cf, q[c], Aa));
                            *CMP(c) = out;
                            if (REG) mo[REG ? c : 0] = out;
                        }
                        const T oam = -m2 - B2<T>::lg2(S - T(1));
                        if (owner_of<PAIR, G>(am) == g) IO::st(Mt + am * PM + i, oam);
                        if (REG) {
                            am_prev = am;
                            out_am = oam;
                        }
                        if (own_diag) {
                            if (!REG) Dg[i] = IO::ld(Mt + i * PM + i);
                            Mt[i * PM + i] = MS(0.f);
                        }
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
#undef COL
#undef RL
#undef RM
#undef CM
#undef CMP
#undef RL2
#undef RM2
}

// ------------------------------------------------------------------ tier table

struct TierCfg {
    int smax;
    int ch, g;
};

// FP32: 32/64/96/112/128/144/160 rows in shared memory; FP64: 32/64/112 (tiers 4..7
// unused).  The 16-row steps from 96 rows up follow the defect counts of circuit-level
// shots (d = 13, p = 0.005: s = 126 +- 16), where padding rows and columns cost issue slots.
constexpr int kSmemTiers = 7;
constexpr TierCfg kCfg32[kSmemTiers + 1] = {{0, 0, 0},     {32, 32, 1},  {64, 32, 2},  {96, 24, 4},
                                            {112, 28, 4}, {128, 32, 4}, {144, 36, 4}, {160, 40, 4}};
constexpr TierCfg kCfg64[kSmemTiers + 1] = {{0, 0, 0},     {32, 16, 2},  {64, 16, 4},  {112, 28, 4},
                                            {112, 28, 4}, {112, 28, 4}, {112, 28, 4}, {112, 28, 4}};
// FP32 tiers that keep their own outputs in registers (the others have no register room).
constexpr bool kReg32[kSmemTiers + 1] = {false, true, true, false, false, true, false, false};

// Bytes of one RW scratch slot: W [SMAX][SMAX] doubles, Dijkstra distances [warps][nodes]
// doubles, parity [SMAX][SMAX] bytes, done and parity flags [warps][nodes] bytes.
inline int64_t rw_slot_layout(int smax, int nt, int nodes) {
    const int64_t b = 8 * ((int64_t)smax * smax + (int64_t)(nt / 32) * nodes) + (int64_t)smax * smax +
                      2 * (int64_t)(nt / 32) * nodes;
    return (b + 255) / 256 * 256;
}

template <typename T, int CH, int G, typename MS = T>
size_t smem_bytes_of() {
    constexpr int SMAX = CH * G;
    return nref_offset<T, MS>(SMAX, G) + (sizeof(MS) == 2 ? (size_t)SMAX * sizeof(float) : 0) + (size_t)SMAX * 2 + 16;
}

template <typename T, int CH, int G, bool TRACE, bool REG, typename MS = T>
cudaError_t run_tier(const DecodeArgs& a, int num_sms, cudaStream_t st, bool prepare_only) {
    const size_t smem = smem_bytes_of<T, CH, G, MS>();
    auto kern = decode_smem_kernel<T, CH, G, TRACE, REG, false, MS>;
    if (prepare_only)
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CH * G * G, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    kern<<<per_sm * num_sms, CH * G * G, smem, st>>>(a);
    return cudaGetLastError();
}

// Every tier has a production instantiation and a traced one (tests).
template <typename T, int CH, int G, bool REG, typename MS = T>
cudaError_t run_tier2(const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep) {
    const bool tr = a.tr_lambda != nullptr || a.tr_partner != nullptr;
    if (prep) {
        cudaError_t e = run_tier<T, CH, G, false, REG, MS>(a, num_sms, st, true);
        return e != cudaSuccess ? e : run_tier<T, CH, G, true, REG, MS>(a, num_sms, st, true);
    }
    return tr ? run_tier<T, CH, G, true, REG, MS>(a, num_sms, st, false)
              : run_tier<T, CH, G, false, REG, MS>(a, num_sms, st, false);
}

}  // namespace
}  // namespace bp4m
