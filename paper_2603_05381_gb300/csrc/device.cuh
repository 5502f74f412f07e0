// Internal interface between the C-ABI layer and the CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bp4m {

// Device copy of one type's per-pair tables (row-major n_det x n_det, diagonal = boundary).
struct DevTables {
    int n_det = 0;
    int n_words = 0;
    const float* L32 = nullptr;   // prior LLR, FP32
    const double* L64 = nullptr;  // prior LLR, FP64
    const double* W64 = nullptr;  // shortest-path weight, FP64 (candidate weights)
    const uint8_t* P = nullptr;   // observable parity of the path
};

// One graph (and Pauli type) of a fused multi-graph launch: its tables, its syndromes and
// its output arrays.  List items of such a launch are entry << kMultiShift | shot.
struct MultiEntry {
    DevTables tb;
    const uint32_t* synd = nullptr;  // [shots][n_words]
    uint8_t* obs_pred = nullptr;
    uint8_t* flags = nullptr;
    int16_t* iters = nullptr;
};
constexpr int kMultiShift = 21;  // shots per entry < 2^21, entries < 2^10
constexpr int64_t kMultiMask = ((int64_t)1 << kMultiShift) - 1;

// The graph, syndrome row and outputs of one decode item.
struct ItemCtx {
    DevTables tb;
    const uint32_t* synd;
    uint8_t* obs_pred;
    uint8_t* flags;
    int16_t* iters;
    int64_t shot;
};

// Counter slots (unsigned long long) in the device counter block.
enum CounterSlot {
    C_SHOTS = 0,
    C_FAIL_X, C_FAIL_Z, C_FAIL_ANY,
    C_UNCONV_X, C_UNCONV_Z,
    C_FORCED_X, C_FORCED_Z,
    C_CONVFAIL_X, C_CONVFAIL_Z,
    C_ITERS, C_MSGS, C_DEFECTS,
    C_ERRORS,          // shots the kernels refused (internal consistency checks)
    C_TIER_MSGS,       // 9 slots: message updates per decode tier
    C_TIER_SHOTS = C_TIER_MSGS + 9,  // 9 slots: shots per decode tier
    C_FC_RUNS = C_TIER_SHOTS + 9,    // forced-convergence runs
    C_FC_ROUNDS,                     // locally-dominant rounds summed over runs
    C_UNCONV_ANY,                    // shots with at least one unconverged type
    C_CONVFAIL_ANY,                  // shots with every type converged and some type failed
    C_NUM
};

// Per-shot result flags.
enum : uint8_t { F_CONVERGED = 1, F_FORCED_RAN = 2, F_FROM_FORCED = 4, F_FROM_QBP = 8 };

// Number of s tiers and the per-tier bookkeeping in the workspace.
constexpr int kTiers = 9;      // tier 0: s == 0 (done in classify), 1..7 shared memory, 8 global
constexpr int kGlobalTier = 8;

struct TierPlan {
    int smax[kTiers];  // inclusive upper bound of s for the tier (global tier: unbounded)
};

struct DecodeArgs {
    DevTables tb;
    const uint32_t* synd = nullptr;  // [shots][n_words]
    int64_t shots = 0;
    const int32_t* list = nullptr;   // this tier's shot indices
    const int32_t* count = nullptr;  // number of entries in `list`
    int32_t* next = nullptr;         // work-stealing counter
    int T = 0;
    int early_exit = 1;
    int decoder = 0;                 // 0 = BP4M, 1 = BP4MF
    int forced_static = 0;           // forced convergence: 0 = global greedy, 1 = static partition
    double alpha = 1.0;
    int pitch = 0;                   // shared-memory row pitch in elements
    int tier = 0;                    // decode tier (per-tier counters)
    // outputs (any may be null)
    uint8_t* obs_pred = nullptr;
    uint8_t* flags = nullptr;
    int16_t* iters = nullptr;
    unsigned long long* ctr = nullptr;
    // trace (tests): lambda [shots][s_cap][s_cap] of the compute type, partner [shots][s_cap]
    void* tr_lambda = nullptr;
    int16_t* tr_partner = nullptr;
    int32_t* tr_defects = nullptr;
    int s_cap = 0;
    // shot source when `list`/`count` are null: shots 0 .. count_val-1 in order
    int64_t count_val = 0;
    int* err_flag = nullptr;         // set to 1 by a block that meets a shot it cannot hold
    int flags_mode = 0;              // 0: `flags` gets F_* bits; 1: `flags` gets converged 0/1
    // B-BP4MF second stage: the shot's priors come from Dijkstra over per-qubit weights
    // max(ln((1-P)/P), kRwMinWeight), P = the first stage's posterior (rw_post
    // [shots][n_units]); adjacency in CSR over n_det + 1 nodes, entries packed
    // neighbour | unit << 15 | obs << 31, each node's entries sorted by (neighbour, obs).
    // Per-shot W, parity and Dijkstra state live in a per-block slot of gscratch of
    // rw_slot_bytes bytes (rw_scratch_bytes()).
    const double* rw_post = nullptr;
    const int* rw_off = nullptr;
    const uint32_t* rw_adj = nullptr;
    int rw_units = 0;
    int64_t rw_slot_bytes = 0;
    // fused multi-graph launch: per-entry tables and buffers (tb / synd / outputs unused)
    const MultiEntry* multi = nullptr;
    // global tier: scratch slots
    void* gscratch = nullptr;
    int64_t gscratch_bytes = 0;      // size of gscratch (checked by the reweighting launches)
    int64_t gslot_elems = 0;         // elements per slot for each of the three matrices
    int gsmax = 0;                   // largest s a slot holds
    int stream_cl = 0;               // streaming tier's cluster size (stream_cluster_for); 0 or 1: none
    int tile_form = 0;               // FP32 shared-memory tiers: 0 = library default, 1 = rows, 2 = register tiles
};

#ifdef __CUDACC__
__device__ __forceinline__ ItemCtx resolve_item(const DecodeArgs& a, int64_t code) {
    ItemCtx c;
    if (a.multi) {
        const MultiEntry& e = a.multi[code >> kMultiShift];
        c.tb = e.tb;
        c.synd = e.synd;
        c.obs_pred = e.obs_pred;
        c.flags = e.flags;
        c.iters = e.iters;
        c.shot = code & kMultiMask;
    } else {
        c.tb = a.tb;
        c.synd = a.synd;
        c.obs_pred = a.obs_pred;
        c.flags = a.flags;
        c.iters = a.iters;
        c.shot = code;
    }
    return c;
}
#endif

struct SampleArgs {
    uint64_t first_shot = 0;
    int64_t shots = 0;
    uint64_t seed = 0;
    uint32_t stream_id = 0;
    int n_units = 0;
    int n_types = 1;
    int n_det[2] = {0, 0};
    int n_words[2] = {0, 0};
    // circuit: per edge threshold and packed (u | v << 15 | obs << 31)
    const uint32_t* thr = nullptr;
    const uint32_t* uvo = nullptr;
    // code capacity: per qubit and type packed (u | v << 15 | obs << 31); thresholds t1..t3
    const uint32_t* cc_uvo = nullptr;  // [2][n_units]
    uint32_t cc_thr[3] = {0, 0, 0};
    uint32_t* synd = nullptr;          // [n_types][shots][n_words]
    uint8_t* obs = nullptr;            // [n_types][shots]
};

struct QbpArgs {
    int64_t shots = 0;
    int T = 0;
    double p = 0.0;
    double clamp = 1e-15;            // |prod tanh| is kept at most 1 - clamp
    int n_qubits = 0, n_checks = 0, n_xchecks = 0;
    int n_words[2] = {0, 0};
    const uint32_t* synd0 = nullptr;  // type 0 syndromes (Z-checks)
    const uint32_t* synd1 = nullptr;  // type 1 syndromes (X-checks)
    const int* chk_q = nullptr;       // [n_checks][4] qubit or -1; X-checks first
    const int* q_edge = nullptr;      // [n_qubits][4] Tanner edge c*4+j or -1
    const uint8_t* in_zl = nullptr;
    const uint8_t* in_xl = nullptr;
    uint8_t* qconv = nullptr;         // [shots]
    uint8_t* qobs = nullptr;          // [2][shots]
    int16_t* qiters = nullptr;        // [shots]
    double* post = nullptr;           // [2][shots][n_qubits]: P(X comp), P(Z comp)
};

// B-BP4MF second-stage preparation: per shot and type, every qubit whose posterior of that
// type's error component is above one half is taken as present (its edge's endpoints flip
// in a copy of the syndrome, its observable bit goes into a base parity).
struct RwFlipArgs {
    int64_t shots = 0;
    int n_units = 0;
    int n_det[2] = {0, 0};
    int n_words[2] = {0, 0};
    const uint32_t* synd[2] = {nullptr, nullptr};  // [shots][n_words[ty]]
    const double* post = nullptr;                  // [2][shots][n_units]
    const uint32_t* cc_uvo = nullptr;              // [2][n_units] packed u | v << 15 | obs << 31
    uint32_t* out[2] = {nullptr, nullptr};         // flipped syndromes, same layout as synd
    uint8_t* base = nullptr;                       // [2][shots]
};

// ---- launchers (kernels_*.cu) ----
cudaError_t launch_qbp(int precision, const QbpArgs& a, int num_sms, cudaStream_t st);
cudaError_t launch_rw_flip(const RwFlipArgs& a, int num_sms, cudaStream_t st);
// obs_pred[ty][shot] ^= base[ty][shot] for the shots the first stage did not resolve
cudaError_t launch_rw_base(uint8_t* obs_pred, const uint8_t* skip, const uint8_t* base, int64_t shots,
                           cudaStream_t st);
cudaError_t launch_sample_circuit(const SampleArgs& a, cudaStream_t st);
cudaError_t launch_sample_code_capacity(const SampleArgs& a, cudaStream_t st);

// classify: per shot s = popcount; s == 0 results are written directly; the others are
// appended to their tier's list.  counts[kTiers], max_s (int) must be zeroed before.
// With `skip` (per-shot flag) non-null, flagged shots are not decoded: their outputs are
// taken from skip_obs (the first stage of B-BP4MF) and skip_iters.
cudaError_t launch_classify(const uint32_t* synd, int64_t shots, int n_words,
                            const TierPlan& plan, int32_t* lists /*[kTiers][shots]*/,
                            int32_t* counts, int32_t* max_s, uint8_t* obs_pred, uint8_t* flags,
                            int16_t* iters, int32_t* tr_defects, const uint8_t* skip,
                            const uint8_t* skip_obs, const int16_t* skip_iters, cudaStream_t st,
                            int64_t list_stride = 0 /* 0: shots */, int32_t item_base = 0);

// Register-tile form of the FP32 shared-memory tiers (decode_reg.cuh): tiers that have one,
// and its launch (or, with prepare_only, its one-time kernel attributes).
bool reg_tier_available(int tier);
cudaError_t launch_decode_tier_reg(int tier, const DecodeArgs& a, int num_sms, cudaStream_t st, bool prepare_only);
// 16-bit message storage (precision 2 = IEEE half, 3 = bfloat16) of the shared-memory tiers.
cudaError_t launch_decode_tier_half(int precision, int tier, const DecodeArgs& a, int num_sms, cudaStream_t st,
                                    bool prepare_only);
// Launch the decoding kernel of shared-memory tier `tier` (1..7) for precision
// (0 = FP64, 1 = FP32).  Returns cudaSuccess if the tier is empty by construction.
cudaError_t launch_decode_tier(int precision, int tier, const DecodeArgs& a, int num_sms,
                               cudaStream_t st);
// Reweighting (B-BP4MF second stage) decode of the shared-memory tiers (FP32 1..7, FP64
// 1..3).  rw_scratch_bytes() is the global scratch the launch of `tier` needs for a graph
// of n_det detectors (one slot per resident block) and sets *slot_bytes; the caller
// passes that scratch in a.gscratch and the slot size in a.rw_slot_bytes.
size_t rw_scratch_bytes(int precision, int tier, int n_det, int num_sms, int64_t* slot_bytes);
cudaError_t launch_decode_tier_rw(int precision, int tier, const DecodeArgs& a, int num_sms,
                                  cudaStream_t st);
// Highest shared-memory tier per precision (FP64 tiers 4..7 are never populated).
constexpr int kRwMaxTier32 = 7;
constexpr int kRwMaxTier64 = 3;
// Smallest edge weight of the reweighted graph: posteriors at or above one half would give
// weights <= 0, for which shortest paths do not exist on an undirected graph.
constexpr double kRwMinWeight = 9.5367431640625e-07;  // 2^-20
// Global-memory tier.  `slots` CTAs each own one scratch slot of global_slot_bytes() for
// shots of up to max_s defects (a width class's bound); a.gsmax must be the value that
// function reports.
size_t global_slot_bytes(int precision, int max_s, int* gsmax_out);
// Resident blocks per SM of the global-memory tier for shots of up to max_s defects.
int global_blocks_per_sm(int precision, int max_s);
cudaError_t launch_decode_global(int precision, const DecodeArgs& a, int slots,
                                 cudaStream_t st);
// Streaming tier with 16-bit message storage (precision 2 = IEEE half, 3 = bfloat16) for
// ch columns per lane (kernels_half.cu).
cudaError_t launch_stream_half(int precision, int ch, const DecodeArgs& a, int slots, cudaStream_t st);
// Cluster form of the streaming tier (kernels_cluster.cu, kernels_cluster_half.cu): the
// blocks of a thread-block cluster share one shot and one slot.  stream_cluster_size() is the
// cluster size a launch of ch columns per lane uses (1: one block per shot) for a requested
// size (0: the default of the width); launch_stream_cluster() runs min(slots, resident
// clusters) clusters, one slot of the width's size each.
int stream_cluster_default(int ch);
bool stream_cluster_instantiated(int precision, int ch, int cl);
int stream_cluster_capacity_of(int precision, int ch, int cl);
int stream_cluster_capacity_half(int precision, int ch, int cl);
int stream_cluster_size(int precision, int ch, int requested);
// Cluster size for a streaming launch of a class of `shots` shots at slot width gsmax:
// `requested` if non-zero (as stream_cluster_size), else 1 when the class fills at least half
// of full_blocks (the resident blocks of one block per shot), else the size that finishes
// the class soonest.  1 for the general kernel's widths and FP64.
int stream_cluster_for(int precision, int gsmax, int requested, int64_t shots, int full_blocks);
cudaError_t launch_stream_cluster(int precision, int ch, int cl, const DecodeArgs& a, int slots, cudaStream_t st);
cudaError_t launch_stream_cluster_half(int precision, int ch, int cl, const DecodeArgs& a, int slots,
                                       cudaStream_t st);
// Width classes of the global tier for a batch whose largest defect count is max_s: class k
// takes the shots with smax[k-1] < s <= smax[k] (smax ascending; the last class is max_s's
// own, the general kernel's when max_s is above the widest streaming variant).
constexpr int kMaxGlobalClasses = 12;
struct GlobalClasses {
    int n;
    int smax[kMaxGlobalClasses];
};
GlobalClasses global_classes(int precision, int max_s);
// Splits the global tier's list (a.list, a.count) into the classes' lists: class k's items go
// to sub[k * stride ..], its count to sub_counts[k] (zeroed by the caller); a shot above the
// last bound goes to the last class.  max_items bounds a.count (sizes the grid).
cudaError_t launch_partition_global(const DecodeArgs& a, const GlobalClasses& gc, int32_t* sub, int64_t stride,
                                    int32_t* sub_counts, int64_t max_items, int num_sms, cudaStream_t st);
// Shared-memory tier plan for a precision.
TierPlan tier_plan(int precision);
cudaError_t prepare_decode_kernels(int precision);

// Decodes shots 0 .. shots-1 with the global-memory kernel using the library's file-scope
// device scratch array instead of allocated memory (see bp4m_decode_noalloc).  Returns
// cudaErrorInvalidValue with *too_many set when a shot exceeds the array's defect limit.
cudaError_t launch_decode_noalloc(int precision, DecodeArgs a, int64_t shots, cudaStream_t st,
                                  int* too_many);
int noalloc_max_defects();
int64_t noalloc_max_shots();

// MUFU throughput probe (measurement support): `blocks` blocks of 1024 threads, one per
// SM, each timing `steps` rounds of its special-function chains with the SM cycle counter
// (cycles[blocks]); sink[blocks * 1024] keeps the results live.  mode 0 = ex2, 1 = lg2,
// 2 = ex2 and lg2 alternating.
cudaError_t launch_mufu_probe(int mode, int blocks, int steps, long long* cycles, float* sink, cudaStream_t st);
int mufu_probe_ops_per_thread(int mode, int steps);

cudaError_t launch_count(const uint8_t* obs_true, const uint8_t* obs_pred, const uint8_t* flags,
                         int64_t shots, int n_types, unsigned long long* ctr, cudaStream_t st);

}  // namespace bp4m
