// Decoding kernels for shots that do not fit the shared-memory tiers (global-memory and
// streaming tiers, the allocation-free entry point) and the dispatch of every tier.
// The shared-memory kernel and its tier table are in decode_smem.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <initializer_list>
#include <cfloat>
#include <cmath>

#include "decode_smem.cuh"
#include "decode_stream.cuh"
#include "device.cuh"

namespace bp4m {
namespace {

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
    // static-partition forced convergence: factors in processing order
    short* order = reinterpret_cast<short*>(reinterpret_cast<uintptr_t>(matched + gsmax + 1) & ~(uintptr_t)1);
    __shared__ int sh_item, sh_s, sh_best_par, sh_best_forced, sh_improve, sh_use_best;
    __shared__ double sh_best_w;
    T* slot = reinterpret_cast<T*>(a.gscratch) + (size_t)blockIdx.x * 3 * a.gslot_elems;
    T* Lg = slot;
    T* Ma = slot + a.gslot_elems;
    T* Mb = slot + 2 * a.gslot_elems;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = a.tb.n_det;
    const T* __restrict__ Ltab = Num<T>::L(a.tb);
    const int64_t count = a.count ? (int64_t)*a.count : a.count_val;
    const bool plain = a.alpha == 1.0;
    const T ainv = (T)(1.0 / a.alpha);
    const bool full = (a.decoder == 1) || !a.early_exit;
    T* trl = reinterpret_cast<T*>(a.tr_lambda);
    unsigned long long acc_it = 0, acc_msg = 0, acc_def = 0, acc_shots = 0, acc_fc = 0, acc_fcr = 0;

    for (;;) {
        if (tid == 0) sh_item = atomicAdd(a.next, 1);
        __syncthreads();
        const int item = sh_item;
        if (item >= count) break;
        const int64_t shot = a.list ? (int64_t)a.list[item] : (int64_t)item;
        if (warp == 0) {
            const int s0 = compact_defects(a.synd + (size_t)shot * a.tb.n_words, a.tb.n_words,
                                           dets, gsmax, lane);
            if (lane == 0) sh_s = s0;
        }
        __syncthreads();
        const int s = sh_s;
        if (s > gsmax) {
            if (tid == 0) {
                if (a.ctr) atomicAdd(a.ctr + C_ERRORS, 1ull);
                if (a.err_flag) atomicOr(a.err_flag, 1);
                if (a.obs_pred) a.obs_pred[shot] = 0;
                if (a.flags) a.flags[shot] = 0;
                if (a.iters) a.iters[shot] = 0;
            }
            continue;
        }
        if (s < 2) {
            // no defect: nothing to match; one defect: it goes to the boundary in every
            // iteration (empty leave-one-out set)
            if (tid == 0) {
                const int its = s == 0 ? 0 : (full ? a.T : 1);
                if (a.obs_pred) a.obs_pred[shot] = s == 0 ? 0 : a.tb.P[(size_t)dets[0] * n + dets[0]];
                if (a.flags) a.flags[shot] = a.flags_mode ? 1 : F_CONVERGED;
                if (a.iters) a.iters[shot] = (int16_t)its;
                acc_it += (unsigned long long)its;
                acc_msg += (unsigned long long)(s * its);
                acc_def += (unsigned long long)s;
                acc_shots += 1;
            }
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
                    if (a.forced_static) {
                        // the paper's static partition: row r's block is v_rk, k >= r; its
                        // maximum (ties: smaller k) represents factor r; representatives are
                        // ranked by posterior (ties: smaller r) and processed in that order
                        for (int r = tid; r < s; r += kGlobThreads) {
                            T bl = Num<T>::ninf();
                            int bk = -1;
                            for (int k = r; k < s; ++k) {
                                const T l = Lg[(size_t)r * s + k];
                                const T own = Mc[(size_t)k * s + r];
                                const T lam = (k == r) ? l + own : l + (own + Mc[(size_t)r * s + k]);
                                if (bk < 0 || lam > bl) {
                                    bl = lam;
                                    bk = k;
                                }
                            }
                            choice[r] = bk >= 0 ? bk : r;
                            rowacc[r] = (double)bl;
                        }
                        __syncthreads();
                        for (int r = tid; r < s; r += kGlobThreads) {
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
                            acc_fcr += 1;
                        }
                        __syncthreads();
                    }
                    for (int round = 0; round < s && !a.forced_static; ++round) {
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
                        if (tid == 0) acc_fcr += 1;
                        if (__syncthreads_count(left) == 0) break;
                    }
                    if (tid == 0) acc_fc += 1;
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
                a.flags[shot] = a.flags_mode ? (uint8_t)(any_conv ? 1 : 0)
                                             : (uint8_t)((any_conv ? F_CONVERGED : 0) | (forced_ran ? F_FORCED_RAN : 0) |
                                                         (out_forced ? F_FROM_FORCED : 0));
            if (a.iters) a.iters[shot] = (int16_t)t;
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

// Dynamic shared memory of the general global-memory kernel for shots of up to gsmax defects.
inline size_t global_kernel_smem(int gsmax) {
    return (size_t)gsmax * (sizeof(double) + 2 * sizeof(int) + 2 * sizeof(short) + 1) + 32;
}

// ------------------------------------------------------------------ no-allocation scratch
//
// bp4m_decode_noalloc serves callers that cannot allocate device memory.  Its scratch is
// this file-scope array: a 256-byte header (work counter, error flag) and 16 slots of
// three 192 x 192 FP64 matrices, 14.2 MB held by every GPU that loads the library until the
// process exits.  Host code must not use the array's name as a device address; the
// address is looked up once per device with cudaGetSymbolAddress and cached.
constexpr int kNoAllocMaxDefects = 192;
constexpr int kNoAllocSlots = 16;
constexpr size_t kNoAllocHeader = 256;
constexpr size_t kNoAllocSlotElems = (size_t)kNoAllocMaxDefects * kNoAllocMaxDefects;
constexpr size_t kNoAllocBytes = kNoAllocHeader + (size_t)kNoAllocSlots * 3 * kNoAllocSlotElems * sizeof(double);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::atomic<void*> g_noalloc_addr[kMaxDevices];

template <typename T>
cudaError_t dispatch_tier(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep);

// Form of the FP32 tiers that have both when the caller leaves the choice to the library
constexpr bool kRegTilesDefault = false;

template <>
cudaError_t dispatch_tier<float>(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep) {
    // the register-tile form where the tier has one (both forms are prepared)
    if (reg_tier_available(tier)) {
        if (prep) {
            cudaError_t e = launch_decode_tier_reg(tier, a, num_sms, st, true);
            if (e != cudaSuccess) return e;
        } else if (a.tile_form == 2 || (a.tile_form == 0 && kRegTilesDefault)) {
            return launch_decode_tier_reg(tier, a, num_sms, st, false);
        }
    }
    switch (tier) {
        case 1: return run_tier2<float, 32, 1, kReg32[1]>(a, num_sms, st, prep);
        case 2: return run_tier2<float, 32, 2, kReg32[2]>(a, num_sms, st, prep);
        case 3: return run_tier2<float, 24, 4, kReg32[3]>(a, num_sms, st, prep);
        case 4: return run_tier2<float, 28, 4, kReg32[4]>(a, num_sms, st, prep);
        case 5: return run_tier2<float, 32, 4, kReg32[5]>(a, num_sms, st, prep);
        case 6: return run_tier2<float, 36, 4, kReg32[6]>(a, num_sms, st, prep);
        case 7: return run_tier2<float, 40, 4, kReg32[7]>(a, num_sms, st, prep);
        default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t dispatch_tier<double>(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prep) {
    switch (tier) {
        case 1: return run_tier2<double, 16, 2, false>(a, num_sms, st, prep);
        case 2: return run_tier2<double, 16, 4, false>(a, num_sms, st, prep);
        case 3: return run_tier2<double, 28, 4, false>(a, num_sms, st, prep);
        case 4: case 5: case 6: case 7: return cudaSuccess;  // same bound as tier 3: never populated
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

TierPlan tier_plan(int precision) {
    TierPlan p{};
    const TierCfg* c = precision == 0 ? kCfg64 : kCfg32;
    for (int k = 0; k < kGlobalTier; ++k) p.smax[k] = c[k].smax;
    p.smax[kGlobalTier] = 0x7fffffff;
    return p;
}

cudaError_t prepare_decode_kernels(int precision) {
    DecodeArgs dummy;
    for (int tier = 1; tier < kGlobalTier; ++tier) {
        cudaError_t e = precision == 0   ? dispatch_tier<double>(tier, dummy, 0, 0, true)
                        : precision == 1 ? dispatch_tier<float>(tier, dummy, 0, 0, true)
                                         : launch_decode_tier_half(precision, tier, dummy, 0, 0, true);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_decode_tier(int precision, int tier, const DecodeArgs& a, int num_sms,
                               cudaStream_t st) {
    if (precision >= 2) return launch_decode_tier_half(precision, tier, a, num_sms, st, false);
    return precision == 0 ? dispatch_tier<double>(tier, a, num_sms, st, false)
                          : dispatch_tier<float>(tier, a, num_sms, st, false);
}

int noalloc_max_defects() { return kNoAllocMaxDefects; }
int64_t noalloc_max_shots() { return (int64_t)0x7fffffff - kNoAllocSlots; }

cudaError_t launch_decode_noalloc(int precision, DecodeArgs a, int64_t shots, cudaStream_t st,
                                  int* too_many) {
    *too_many = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void* base = g_noalloc_addr[dev].load();
    if (!base) {
        // set-up, once per device with that device current: the device address of the array
        e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev].store(base);
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    // the header (work counter and error flag) must start at zero; the matrices are
    // initialised per shot by the kernel
    e = cudaMemsetAsync(b, 0, kNoAllocHeader, st);
    if (e != cudaSuccess) return e;
    a.list = nullptr;
    a.count = nullptr;
    a.count_val = shots;
    a.next = reinterpret_cast<int32_t*>(b);
    a.err_flag = reinterpret_cast<int*>(b) + 1;
    a.gscratch = b + kNoAllocHeader;
    a.gslot_elems = (int64_t)kNoAllocSlotElems;
    a.gsmax = kNoAllocMaxDefects;
    const size_t smem = global_kernel_smem(a.gsmax);
    if (precision == 0)
        decode_global_kernel<double><<<kNoAllocSlots, kGlobThreads, smem, st>>>(a);
    else
        decode_global_kernel<float><<<kNoAllocSlots, kGlobThreads, smem, st>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int flag = 0;
    e = cudaMemcpyAsync(&flag, a.err_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (flag) {
        *too_many = 1;
        return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

namespace {

// Columns per lane of the streaming kernel for shots of up to max_s defects; 0 when the
// general global kernel takes them.
// FP32 steps of 64 columns up to 512 and of 128 columns up to 1024 keep the padding of a
// shot of more than 160 defects below 1.3x in each dimension (d = 15..25 circuits at
// p = 0.005 average 194, 283, 395, 534, 702 and 902 defects).
int stream_ch(int precision, int max_s) {
    if (precision != 0) {
        if (max_s <= 192) return 6;
        if (max_s <= 256) return 8;
        if (max_s <= 320) return 10;
        if (max_s <= 384) return 12;
        if (max_s <= 448) return 14;
        if (max_s <= 512) return 16;
        if (max_s <= 640) return 20;
        if (max_s <= 768) return 24;
        if (max_s <= 896) return 28;
        if (max_s <= 1024) return 32;
        return 0;
    }
    if (max_s <= 256) return 8;
    if (max_s <= 512) return 16;
    return 0;
}

}  // namespace

int stream_cluster_for(int precision, int gsmax, int requested, int64_t shots, int full_blocks) {
    const int ch = stream_ch(precision, gsmax);
    if (precision == 0 || ch == 0 || 32 * ch != gsmax) return 1;
    if (requested != 0) return stream_cluster_size(precision, ch, requested);
    // automatic: one block per shot while the class fills the device at least half; below
    // that, the size that finishes the class soonest, with the cluster form's measured cost
    // per shot and SM of about 1.25 + 0.03 CL times one block's
    if (shots <= 0 || 2 * shots >= full_blocks) return 1;
    double best = 1.0;
    int best_cl = 1;
    for (int cl : {2, 4, 8, 16}) {
        const int cap = stream_cluster_capacity_of(precision, ch, cl);
        if (cap <= 0) continue;
        const int64_t rounds = (shots + cap - 1) / cap;
        const double t = (double)rounds * (1.25 + 0.03 * cl) / cl;
        if (t < best) {
            best = t;
            best_cl = cl;
        }
    }
    return best_cl;
}

int global_blocks_per_sm(int precision, int max_s) {
    const int ch = stream_ch(precision, max_s);
    return (precision != 0 && ch != 0 && ch <= 8) ? kStreamBlocks<float, 8> : 1;
}

size_t global_slot_bytes(int precision, int max_s, int* gsmax_out) {
    const size_t esz = precision == 0 ? sizeof(double) : sizeof(float);
    const int ch = stream_ch(precision, max_s);
    if (ch) {
        const int ld = 32 * ch;
        *gsmax_out = ld;
        return precision == 0   ? stream_slot_bytes<double, double>(ld)
               : precision == 1 ? stream_slot_bytes<float, float>(ld)
                                : stream_slot_bytes<float, __half>(ld);  // 16-bit messages, FP32 priors
    }
    const int gsmax = (max_s + 63) / 64 * 64;
    *gsmax_out = gsmax;
    return (size_t)3 * gsmax * gsmax * esz;
}

cudaError_t launch_decode_global(int precision, const DecodeArgs& a, int slots, cudaStream_t st) {
    if (slots <= 0) return cudaSuccess;
    const int ch = stream_ch(precision, a.gsmax);
    if (ch && 32 * ch == a.gsmax) {
        // the cluster form where a size above 1 is asked for (not with a lambda/partner trace)
        if (precision != 0 && a.stream_cl > 1 && a.tr_lambda == nullptr && a.tr_partner == nullptr) {
            const int cl = stream_cluster_size(precision, ch, a.stream_cl);
            if (cl > 1) return launch_stream_cluster(precision, ch, cl, a, slots, st);
        }
        if (precision >= 2) return launch_stream_half(precision, ch, a, slots, st);
        if (precision == 0) {
            if (ch == 8) return run_stream<double, 8>(a, slots, st);
            return run_stream<double, 16>(a, slots, st);
        }
        switch (ch) {
            case 6: return run_stream<float, 6>(a, slots, st);
            case 8: return run_stream<float, 8>(a, slots, st);
            case 10: return run_stream<float, 10>(a, slots, st);
            case 12: return run_stream<float, 12>(a, slots, st);
            case 14: return run_stream<float, 14>(a, slots, st);
            case 16: return run_stream<float, 16>(a, slots, st);
            case 20: return run_stream<float, 20>(a, slots, st);
            case 24: return run_stream<float, 24>(a, slots, st);
            case 28: return run_stream<float, 28>(a, slots, st);
            default: return run_stream<float, 32>(a, slots, st);
        }
    }
    const size_t smem = global_kernel_smem(a.gsmax);
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

// ------------------------------------------------------------------ width classes
//
// The streaming kernel's width follows the largest defect count it may meet, and its work
// per shot is s rows x width columns, so one shot far above the others would widen the
// whole global tier.  The tier is therefore split by width: class k takes the shots with
// smax[k-1] < s <= smax[k] and runs at its own width.

GlobalClasses global_classes(int precision, int max_s) {
    GlobalClasses gc{};
    int widths[kMaxGlobalClasses];
    int nw = 0;
    if (precision != 0) {
        for (int ch : {6, 8, 10, 12, 14, 16, 20, 24, 28, 32}) widths[nw++] = 32 * ch;
    } else {
        widths[nw++] = 256;
        widths[nw++] = 512;
    }
    for (int k = 0; k < nw; ++k) {
        gc.smax[gc.n++] = widths[k];
        if (max_s <= widths[k]) return gc;
    }
    gc.smax[gc.n++] = max_s;  // the general kernel takes everything above the widest variant
    return gc;
}

namespace {

constexpr int kPartThreads = 256;

__global__ void __launch_bounds__(kPartThreads) partition_global_kernel(const DecodeArgs a, GlobalClasses gc,
                                                                        int32_t* sub, int64_t stride,
                                                                        int32_t* sub_counts) {
    const int64_t count = a.count ? (int64_t)*a.count : a.count_val;
    for (int64_t i = (int64_t)blockIdx.x * kPartThreads + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * kPartThreads) {
        const int32_t code = a.list[i];
        const ItemCtx ic = resolve_item(a, code);
        const uint32_t* w = ic.synd + (size_t)ic.shot * ic.tb.n_words;
        int sdef = 0;
        for (int k = 0; k < ic.tb.n_words; ++k) sdef += __popc(__ldg(w + k));
        // a shot above the last bound goes to the last class, whose kernel reports it
        int c = gc.n - 1;
        for (int k = 0; k < gc.n; ++k)
            if (sdef <= gc.smax[k]) {
                c = k;
                break;
            }
        const int pos = atomicAdd(sub_counts + c, 1);
        sub[(size_t)c * stride + pos] = code;
    }
}

}  // namespace

cudaError_t launch_partition_global(const DecodeArgs& a, const GlobalClasses& gc, int32_t* sub, int64_t stride,
                                    int32_t* sub_counts, int64_t max_items, int num_sms, cudaStream_t st) {
    if (max_items <= 0) return cudaSuccess;
    const int64_t want = (max_items + kPartThreads - 1) / kPartThreads;
    const int grid = (int)std::min<int64_t>(want, (int64_t)num_sms * 8);
    partition_global_kernel<<<grid, kPartThreads, 0, st>>>(a, gc, sub, stride, sub_counts);
    return cudaGetLastError();
}

}  // namespace bp4m
