/*
 * bp4m.h - C ABI of the GB300 (sm_103a) BP4M decoding library.
 *
 * The library decodes surface-code syndromes with belief propagation run on the
 * per-shot decoding graph (one node per unsatisfied detector plus a boundary node per
 * detector, an edge for every pair and one to the boundary), as defined in Sec.
 * "MWPM on the surface code" and Sec. "Bipartite Graph Representation" of
 * "Achieving Thresholds via Standalone Belief Propagation on Surface Codes"
 * (arXiv 2603.05381).  Every decoding step runs in the library's own CUDA kernels.
 *
 * Conventions for every entry point:
 *   - Return value: 0 on success, a negative BP4M_E* code on failure; the message of the
 *     last failure on the calling thread is returned by bp4m_last_error().
 *   - Buffers are owned by the caller.  Each buffer argument may be host memory (pageable
 *     or pinned) or device memory of the current device; the kind is detected with
 *     cudaPointerGetAttributes.  Host buffers are staged through library-owned device
 *     memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Entry points that
 *     return host-visible results synchronise that stream before returning.
 *   - Graphs are owned by the library (bp4m_free_graph releases them).  A graph may be
 *     used by one thread at a time.
 */
#ifndef BP4M_H
#define BP4M_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define BP4M_OK            0
#define BP4M_EINVAL       -1   /* bad argument (null pointer, size, option) */
#define BP4M_ENOMEM       -2   /* device or host allocation failed */
#define BP4M_EUNSUPPORTED -3   /* valid request the library does not implement */
#define BP4M_ETIMEOUT     -4   /* a bounded device-side wait ran out */
#define BP4M_ECUDA        -5   /* a CUDA runtime call failed (message has the CUDA error) */

/* ---- code, noise and decoder descriptions ---- */
#define BP4M_ROTATED   0       /* d^2 data qubits, weight-2 boundary plaquettes */
#define BP4M_UNROTATED 1       /* d^2 + (d-1)^2 data qubits on a (2d-1) x (2d-1) grid */

#define BP4M_MEMORY_Z  0

#define BP4M_CODE_CAPACITY 0   /* i.i.d. depolarizing on data qubits: X, Y, Z with p/3 each */
#define BP4M_CIRCUIT       1   /* rotated memory-Z circuit, uniform depolarizing noise p */

#define BP4M_PRIOR_P     0     /* code capacity prior (p/(1-p))^w with the printed p */
#define BP4M_PRIOR_2P3   1     /* code capacity prior with the X (or Z) marginal 2p/3 */

/* Code: surface code of distance d.  rounds = 0 with BP4M_CODE_CAPACITY;
   with BP4M_CIRCUIT rounds = 0 means d rounds (Sec. "Numerical Results": R = d). */
typedef struct {
    int family;   /* BP4M_ROTATED or BP4M_UNROTATED */
    int d;        /* odd distance >= 3 */
    int rounds;   /* syndrome-extraction rounds (circuit only) */
    int basis;    /* BP4M_MEMORY_Z */
} bp4m_code;

typedef struct {
    int model;                  /* BP4M_CODE_CAPACITY or BP4M_CIRCUIT */
    double p;                   /* physical error rate, 0 < p < 0.5 */
    int prior_conv;             /* BP4M_PRIOR_P (default) or BP4M_PRIOR_2P3 (code capacity) */
    int pair_through_boundary;  /* 0 (default): pair paths may not pass through the boundary */
} bp4m_noise;

#define BP4M_FP64 0
#define BP4M_FP32 1
/* 16-bit message storage with FP32 priors and arithmetic: messages are rounded to nearest
   (saturating at the largest finite value), relative to a per-row reference, when stored and
   read back exactly.  Shared-memory and streaming tiers (up to 1024 unsatisfied detectors);
   the general kernel above them uses FP32 messages.  Not for B-BP4MF or
   bp4m_decode_noalloc (BP4M_EUNSUPPORTED). */
#define BP4M_FP16 2
#define BP4M_BF16 3

#define BP4M_DEC_BP4M   0  /* Sec. "Belief Propagation for Matching (BP4M)" */
#define BP4M_DEC_BP4MF  1  /* Sec. "BP4M Forced (BP4MF)"; alpha != 1 gives Memory-BP4MF */
#define BP4M_DEC_BBP4MF 2  /* Sec. "Belief-BP4MF (B-BP4MF)", code capacity only: quaternary BP on
                              the Tanner graph, then BP4MF on priors reweighted by its posteriors */

typedef struct {
    int precision;   /* BP4M_FP64, BP4M_FP32 (messages and arithmetic), BP4M_FP16, BP4M_BF16 */
    int early_exit;  /* BP4M only. 1: output the first converged iteration.
                        0: run all iterations, keep the lightest converged candidate */
    int decoder;     /* BP4M_DEC_BP4M, BP4M_DEC_BP4MF or (sample_and_decode, code capacity)
                        BP4M_DEC_BBP4MF */
    double alpha;    /* variable-update memory parameter (Sec. "BP Improvements"); 1 = plain */
    int type;        /* code capacity only: 0 = X errors on the Z-check graph,
                        1 = Z errors on the X-check graph.  Ignored for circuits. */
    int forced;      /* forced convergence (Sec. "Forced convergence"): BP4M_FORCED_GREEDY
                        (default) or BP4M_FORCED_STATIC */
    int stream_cluster; /* streaming tier (shots above the shared-memory tiers, FP32 or 16-bit
                        messages): the thread blocks of a cluster that share one shot.
                        0 (default): one block per shot when a width class has enough shots
                        to fill half the device, else the size that finishes the class
                        soonest (a few heavy shots then run on up to 16 SMs each; the fused
                        multi-graph decode keeps one block per shot); 1: one block per shot;
                        2, 4, 8, 16: that size where the width has it and the device can hold
                        such clusters, else the width's default.  The outputs do not depend
                        on it. */
    int tile_form;   /* FP32 shared-memory tiers of 113..144 unsatisfied detectors: 0 (default)
                        = the library's choice, which is the row form (measured faster on
                        GB300); 1 = the row form (messages in shared memory, a row per thread
                        group); 2 = register tiles (each thread holds a block of the message
                        matrix and its mirror, so a message meets its partner in registers and
                        only per-row statistics pass through shared memory).  Same arithmetic;
                        results agree within the FP32 rounding of the row sums.  Other tiers
                        and precisions ignore it. */
} bp4m_opts;

/* Forced convergence orders the variables by posterior and picks a matching.
   GREEDY: all variables sorted by posterior (descending; ties: smaller i, then smaller j),
   each accepted iff its factors are unmatched (the global greedy; it reproduces the
   paper's worked example).  STATIC: the paper's static partition, each pair v_ij (i <= j)
   in the block of factor c_i; each block's maximum (ties: smaller j) represents its factor,
   the representatives are processed by posterior (descending; ties: smaller i); a factor
   not yet matched is matched along its representative (to the boundary for v_ii, else
   together with the other factor), and to the boundary when the representative's other
   factor is already matched, a case the paper does not treat. */
#define BP4M_FORCED_GREEDY 0
#define BP4M_FORCED_STATIC 1

/* Aggregate counts of one sample_and_decode call (all u64). */
typedef struct {
    uint64_t shots;
    uint64_t fail[3];          /* per type (X, Z) and "any"; circuits use fail[0] = fail[2] */
    uint64_t unconverged[2];   /* shots of each type whose marginalization never converged */
    uint64_t forced_output[2]; /* shots whose output came from forced convergence */
    uint64_t conv_fail[2];     /* failures among shots that converged (converged LER) */
    uint64_t iterations;       /* sum over shots and types of executed iterations */
    uint64_t msg_updates;      /* sum over shots and types of s^2 per executed iteration */
    uint64_t defects;          /* sum over shots and types of s */
    uint64_t forced_runs;      /* forced-convergence runs */
    uint64_t forced_rounds;    /* rounds of locally dominant choices summed over those runs */
    uint64_t unconverged_any;  /* shots with at least one type never converged (r_nc) */
    uint64_t conv_fail_any;    /* shots with every type converged and a failure */
} bp4m_counts;

typedef struct {
    int n_types;          /* 2 for code capacity (X then Z), 1 for circuits */
    int n_det[2];         /* detectors per type */
    int n_words[2];       /* 32-bit syndrome words per shot and type = ceil(n_det / 32) */
    int n_edges[2];       /* merged detector-graph edges per type */
    int n_units;          /* sampler draws per shot (qubits or graph edges) */
    int model;            /* BP4M_CODE_CAPACITY or BP4M_CIRCUIT */
    int d;
    int rounds;
    double p;
    int64_t table_bytes;  /* device bytes of the per-graph tables once uploaded */
    double mean_defects[2];  /* expected unsatisfied detectors per shot and type: the sum over
                                detectors of the probability that an odd number of their edges
                                flip, (1 - prod_e (1 - 2 q_e)) / 2 (circuit edges carry their
                                merged q; a code-capacity edge flips with 2p/3) */
} bp4m_graph_info_t;

typedef struct bp4m_graph bp4m_graph;

/* Builds the static detector graph and its per-pair tables on the host (Sec. "MWPM on the
   surface code"; the prior of Eq. (two-syn var factors) with w_ij read as a shortest-path
   weight of edge weights ln((1-q_e)/q_e)).  No device memory is touched: the tables are
   uploaded on the first decoding call.  *out receives a new graph. */
int bp4m_build_graph(const bp4m_code* code, const bp4m_noise* noise, bp4m_graph** out);

int bp4m_graph_info(const bp4m_graph* g, bp4m_graph_info_t* out);

/* Copies a host-side table for inspection.  what: */
#define BP4M_EXPORT_W       0  /* double [n_det][n_det]: W_ij, diagonal = to the boundary */
#define BP4M_EXPORT_L       1  /* double [n_det][n_det]: prior LLR l_ij (Eq. priorllr) */
#define BP4M_EXPORT_PARITY  2  /* uint8  [n_det][n_det]: observable parity of the chosen path */
#define BP4M_EXPORT_EDGES   3  /* bp4m_edge [n_edges]: merged graph edges, canonical order */
#define BP4M_EXPORT_THRESH  4  /* uint32 [n_units or 3]: sampler thresholds (circuit: per edge;
                                  code capacity: t1, t2, t3) */
typedef struct { int32_t u, v, obs, pad; double q; } bp4m_edge;
int bp4m_graph_export(const bp4m_graph* g, int type, int what, void* out, size_t bytes);

/* Draws `shots` shots with global indices first_shot .. first_shot+shots-1 and writes their
   bit-packed syndromes, uint32 [n_types][shots][n_words] (detector j at word j>>5, bit
   j&31), and true observable flips, uint8 [n_types][shots].  Counter-based: a shot's
   draws depend only on (seed, stream_id, shot index). */
int bp4m_sample(bp4m_graph* g, uint64_t first_shot, int64_t shots, uint64_t seed,
                uint32_t stream_id, uint32_t* syndromes, uint8_t* obs_true, void* stream);

/* Decodes `shots` bit-packed syndromes of one type (uint32 [shots][n_words]) with
   `iters` BP iterations (Sec. "Belief Propagation").  Outputs per shot (any may be NULL):
   obs_pred = predicted observable flip; converged = 1 if some iteration's marginalization
   converged; iters_used = iterations executed.  Synchronises `stream`. */
int bp4m_decode_batch(bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                      const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* converged,
                      int16_t* iters_used, void* stream);

/* Per-shot internals for testing, all optional (NULL = not written):
   lambda: float or double (per opts->precision) [shots][s_cap][s_cap], posterior LLRs of
           the last executed iteration over the shot's sorted unsatisfied detectors;
   partner: int16 [shots][s_cap], partner[i] = j if the output pairs detector i with j,
           i if it matches i to the boundary; entries past s are -1;
   defects: int32 [shots], s;  flags: uint8 [shots], bit0 converged, bit1 forced
           convergence ran, bit2 output came from forced convergence.
   Shots with s > s_cap are decoded but their lambda/partner rows are not written. */
typedef struct {
    void* lambda;
    int16_t* partner;
    int32_t* defects;
    uint8_t* flags;
    int s_cap;
} bp4m_trace;
int bp4m_decode_trace(bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                      const bp4m_opts* opts, uint8_t* obs_pred, const bp4m_trace* trace,
                      void* stream);

/* Samples and decodes `shots` shots (all types of the graph) and adds up failures:
   a shot fails for a type iff the decoded observable flip differs from the sampled one.
   Sampling (Sec. "Numerical Results": code-capacity depolarizing noise or the circuit-level
   memory experiment at physical error rate p) and the priors of Eq. (two-syn var factors)
   and Eq. (priorllr) both follow p.  When p differs from the graph's p (0 < p < 0.5), the
   tables are re-derived for p from the graph's code and noise options (code capacity: the
   path weights hops x ln((1-p)/p) and priors; circuit: the merged edge probabilities, every
   shortest path, prior and parity), exactly as bp4m_build_graph would build them for p,
   cached inside the graph per p (the 8 most recently used values; each cached value holds
   its own device tables and workspace) and uploaded on first use, so the counts are
   bit-identical to those of a graph built at p.  Shots 0..shots-1, Philox stream 0.  Work
   is split into device-resident batches.  *out is overwritten.  Synchronises `stream`. */
int bp4m_sample_and_decode(bp4m_graph* g, double p, int64_t shots, uint64_t seed, int iters,
                           const bp4m_opts* opts, bp4m_counts* out, void* stream);

/* Same as bp4m_sample_and_decode for the global shot range [first_shot, first_shot+shots)
   with a Philox stream id: independent ranges can be decoded on different devices or
   processes and their counts added. */
int bp4m_sample_and_decode_range(bp4m_graph* g, uint64_t first_shot, int64_t shots,
                                 uint64_t seed, uint32_t stream_id, int iters,
                                 const bp4m_opts* opts, bp4m_counts* out, void* stream);

/* B-BP4MF (Sec. "Belief-BP4MF (B-BP4MF)" and Sec. "Correlated decoding") on code-capacity
   graphs.  First stage: quaternary BP on the Tanner graph with `iters` iterations and the
   graph's p as the depolarizing prior; a shot whose hard decision reproduces its syndrome
   takes that decision.  Otherwise, per type, every data qubit is an edge of the decoding
   graph with P its posterior of an error component of that type.  An edge with P > 1/2
   (negative weight, a case the paper does not treat) is taken as present, as matching
   decoders with negative weights do: its endpoints flip in the shot's syndrome, its
   observable bit is added to the output, and it weighs as its complement.  Every edge then
   weighs max(|ln((1-P)/P)|, 2^-20), Dijkstra from every unsatisfied check of the flipped
   syndrome yields the shot's priors, and BP4MF (alpha from opts) runs for `iters`
   iterations.  At most 160 (FP32) or 112 (FP64) unsatisfied checks
   of a type per shot (BP4M_EUNSUPPORTED beyond).  syndromes: uint32 [2][shots][n_words] (type 0 then type 1, the layout of
   bp4m_sample); outputs obs_pred and flags (bit0 converged, bit3 first stage): uint8
   [2][shots]; flags may be NULL.  Host or device buffers.  Synchronises `stream`. */
int bp4m_decode_bbp4mf(bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                       const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* flags, void* stream);

/* Decoding without any device allocation.  The paper has no counterpart: this entry point
   exists for callers that cannot call cudaMalloc, such as a decoding service that must
   keep a fixed device-memory footprint after start-up, or code running where an
   allocation would synchronise the device or is not permitted.  Every other decoding
   entry point allocates its workspace on first use; this one allocates nothing.

   Decodes `shots` bit-packed syndromes of one type exactly like bp4m_decode_batch with the
   same opts, but every shot goes through the library's global-memory decoding kernel, whose
   scratch is a file-scope device array of fixed size (16 slots of 192 x 192 x 3 FP64
   values, 14.2 MB) that every GPU loading the library holds until the process exits.
   Arguments: `syndromes` uint32 [shots][n_words], `obs_pred`, `converged` (0/1) and
   `iters_used` per shot: all DEVICE memory of the current device (outputs may be NULL).
   Preconditions and limits:
     - the graph's tables must already be on this device: any other decoding call on the
       graph (for example one bp4m_decode_batch) uploads them during set-up;
     - the first call on a device looks up the device address of the scratch array
       (cudaGetSymbolAddress); make that first call before any stream capture;
     - a shot with more than 192 unsatisfied detectors is rejected: the call returns
       BP4M_EINVAL and that shot's outputs are 0;
     - at most 2^31 - 17 shots per call (BP4M_EINVAL beyond);
     - every call shares the one array, which keeps the last call's contents: calls that
       overlap on the GPU (other streams, other threads) race and must be serialised by
       the caller.
   Synchronises `stream`. */
int bp4m_decode_noalloc(const bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                        const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* converged,
                        int16_t* iters_used, void* stream);

/* Kernel timing for measurement.  While enabled, every kernel the library launches for
   this graph is bracketed by CUDA events recorded on the launch stream, and the
   algorithmic message updates of each decoding tier are counted.  Enabling resets the
   accumulators; reading synchronises the events.  Slots: 0 = defect classification,
   1..7 = shared-memory decode tiers (s <= 32, 64, 96, 112, 128, 144, 160 in FP32; 32, 64,
   112 in FP64), 8 = global-memory decode tier, 9 = sampler, 10 = failure counting. */
#define BP4M_PROF_SLOTS 11
typedef struct {
    int64_t launches[BP4M_PROF_SLOTS];
    double ms[BP4M_PROF_SLOTS];                /* summed event-timed durations */
    uint64_t msg_updates[BP4M_PROF_SLOTS];     /* decode tiers: sum of s^2 per executed iteration */
    uint64_t shots[BP4M_PROF_SLOTS];           /* decode tiers: shots decoded */
} bp4m_profile_t;
int bp4m_profile_enable(bp4m_graph* g, int on);
int bp4m_profile_read(bp4m_graph* g, bp4m_profile_t* out);

/* Measurement support (no counterpart in the paper): the throughput of the GPU's
   special-function (MUFU) unit, the roofline denominator of the shared-memory decoding
   tiers, whose every message update takes one ex2 and one lg2 (Sec. "Belief Propagation":
   one exponential and one logarithm per leave-one-out soft maximum).  Launches one block
   of 1024 threads per SM running `steps` (1..2^20) rounds of 8 independent chains and
   times each block with its SM's cycle counter.  Writes out[0] = ex2, out[1] = lg2,
   out[2] = ex2 and lg2 alternating (results per SM per clock, median over the SMs), and
   out[3] = the SM count.  Allocates and frees a few KB of device memory; synchronises
   `stream`. */
int bp4m_probe_mufu(int steps, double* out, void* stream);

void bp4m_free_graph(bp4m_graph* g);

/* ---- Decoding service (no counterpart in the paper: serving infrastructure around the
   BP4M decode of Sec. "Belief Propagation").

   A request loop over device-resident graphs.  bp4m_server_create starts n_slots worker
   threads, each with its own non-blocking CUDA stream on the current device.  A worker
   takes the oldest pending request and merges into it every pending request of the same
   graph, iterations and options while the merged batch stays within max_batch_shots
   (continuous batching); its host-to-device copy, decode kernels and device-to-host copy
   run on its stream, so the slots' batches overlap on the GPU, except that a batch of a
   heavy graph (one whose shots average more than 160 unsatisfied detectors, estimated
   from its edge probabilities when it is added) runs alone: it waits for the batches in
   flight and holds back new ones until it ends.  A heavy graph's request is decoded in
   pieces of at most 1024 shots; after each piece the rest of the request goes to the back
   of the queue, so requests that arrived meanwhile are served between its pieces.
   Message state and tables stay resident: each slot keeps one workspace per graph it has
   decoded, sized for max_batch_shots.  Admission by device memory: before a workspace
   grows, its per-shot buffers must fit device_budget_bytes (summed over all workspaces),
   or, with device_budget_bytes = 0, leave at least max(1 GiB, 1/32 of the device) of the
   device's memory free (cudaMemGetInfo); otherwise the slot frees its least recently used
   workspaces, and a batch that still does not fit fails with BP4M_ENOMEM.  (Scratch of
   the global-memory tier, for shots with more than 160 unsatisfied detectors, grows on
   demand outside the budget; its allocation failing fails the batch with BP4M_ENOMEM.)
   A graph's per-iteration results are
   bit-identical to bp4m_decode_batch on the same syndromes, alone or merged with others.
   bp4m_profile_* does not see the service's launches.  Decoders BP4M and BP4MF (any
   precision); B-BP4MF is BP4M_EUNSUPPORTED. */
typedef struct bp4m_server bp4m_server;

typedef struct {
    double t_submit, t_start, t_done;  /* steady-clock seconds */
    double latency_s;                  /* t_done - t_submit */
    int64_t batch_shots;               /* shots of the merged batch the request ran in */
    int slot;                          /* worker slot that ran it */
} bp4m_request_info;

typedef struct {
    int64_t batches;               /* batches run */
    int64_t merged_requests;       /* requests that joined another request's batch */
    int64_t shots;                 /* shots decoded */
    int64_t evictions;             /* workspaces freed to stay within the budget */
    int64_t max_inflight_batches;  /* most batches running at the same time */
    int64_t pending;               /* requests waiting now */
    int64_t device_bytes;          /* device bytes of the workspaces' per-shot buffers now (what
                                      device_budget_bytes limits; streaming-tier scratch excluded) */
} bp4m_server_stats_t;

/* n_slots in [1, 64]; max_batch_shots in [1, 2^20]; device_budget_bytes >= 0 (0: admission by
   free device memory).  NULL on error (bp4m_last_error). */
bp4m_server* bp4m_server_create(int n_slots, int64_t max_batch_shots, int64_t device_budget_bytes);
/* Registers a graph (uploading its tables); returns its id >= 0 or a negative error code.
   The graph must outlive the server. */
int bp4m_server_add_graph(bp4m_server* s, bp4m_graph* g);
/* Queues `shots` syndromes (host, uint32 [shots][n_words] of opts->type, copied before
   returning) for decoding with `iters` iterations.  obs_pred and converged (uint8 [shots],
   host; converged may be NULL) are written before the request completes and must stay
   valid until bp4m_server_wait returns for it.  Returns the request id >= 0 or a negative
   error code. */
int64_t bp4m_server_submit(bp4m_server* s, int graph_id, const uint32_t* syndromes, int64_t shots, int iters,
                           const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* converged);
/* Waits up to timeout_s seconds (< 0: no limit) for a request; BP4M_OK when it finished
   (info filled, the request is then forgotten), BP4M_ETIMEOUT if not yet, or the error the
   request's batch met. */
int bp4m_server_wait(bp4m_server* s, int64_t request, double timeout_s, bp4m_request_info* info);
int bp4m_server_stats(bp4m_server* s, bp4m_server_stats_t* out);
/* Finishes the queued requests, stops the workers and frees the service's device memory. */
int bp4m_server_destroy(bp4m_server* s);

/* ---- Fused decode of several graphs (no counterpart in the paper: batching of the BP4M
   decode of Sec. "Belief Propagation" across graphs).

   n graphs (a code-capacity graph with its Pauli type in types[k]; types may be NULL for
   type 0) are decoded together: each graph's syndromes are classified into shared tier
   lists and every decode tier is one persistent launch over the shots of all graphs, so
   uneven distances and shot counts share the GPU in one pass.  bp4m_multi_create
   allocates device buffers for max_shots[k] shots per graph (< 2^21) and pinned staging.
   The first bp4m_multi_run times each candidate tier plan on its shots and keeps the
   fastest (autotuner; that run decodes six times); later runs with use_cuda_graph capture
   the whole run (copies, classification, tier launches, streaming tier, copies back) once
   per shot vector in a CUDA graph and replay it.  Results equal bp4m_decode_batch of each
   graph.  FP32, FP16 or BF16 messages; BP4M or BP4MF.  Shots with more than max_defects
   (161..1024) unsatisfied detectors are not decoded and make the run return
   BP4M_EUNSUPPORTED.  Not thread-safe per plan. */
typedef struct bp4m_multi bp4m_multi;

typedef struct {
    int plan;             /* index of the chosen tier plan */
    double plan_ms[3];    /* autotuner timings of the candidate plans (ms) */
    int64_t runs;         /* completed runs */
    int64_t graph_replays;/* runs replayed from the captured CUDA graph */
    uint64_t msg_updates; /* message updates of the last run */
    int stream_cluster;   /* streaming tier's cluster size the autotuner kept (1: one block per
                             shot), or the one opts asked for */
    double stream_ms[2];  /* autotuner timings of the chosen plan with one block per shot and
                             with the cluster form (ms; 0 where not timed) */
} bp4m_multi_info_t;

bp4m_multi* bp4m_multi_create(int n, bp4m_graph* const* graphs, const int* types, const int64_t* max_shots,
                              int iters, const bp4m_opts* opts, int max_defects, int use_cuda_graph);
/* syndromes[k]: host uint32 [shots[k]][n_words]; obs_pred[k] / converged[k] (may be NULL):
   host uint8 [shots[k]].  Synchronous. */
int bp4m_multi_run(bp4m_multi* m, const uint32_t* const* syndromes, const int64_t* shots, uint8_t* const* obs_pred,
                   uint8_t* const* converged);
int bp4m_multi_info(const bp4m_multi* m, bp4m_multi_info_t* out);
void bp4m_multi_destroy(bp4m_multi* m);

const char* bp4m_last_error(void);

/* Library version string. */
const char* bp4m_version(void);

#ifdef __cplusplus
}
#endif
#endif /* BP4M_H */
