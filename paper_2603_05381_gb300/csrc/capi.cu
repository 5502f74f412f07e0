// C ABI of the BP4M decoding library: graph lifecycle, device upload, workspaces and the
// decode / sample entry points declared in include/bp4m.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "bp4m.h"
#include "device.cuh"
#include "host_graph.h"

using namespace bp4m;

namespace {

thread_local std::string g_last_error;
// set on the decoding service's worker threads: their launches are not profiled (the
// profile of a graph is single-threaded state)
thread_local bool tl_no_prof = false;

int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(e == cudaErrorMemoryAllocation ? BP4M_ENOMEM : BP4M_ECUDA, m);
}

#define CK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
}

__global__ void finalize_kernel(const uint8_t* flags, int64_t shots, uint8_t* converged) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < shots;
         k += (int64_t)gridDim.x * blockDim.x)
        converged[k] = (flags[k] & F_CONVERGED) ? 1 : 0;
}

}  // namespace

struct Workspace {
    int64_t cap = 0;
    int n_types = 1;
    size_t words_total = 0;   // sum over types of n_words
    uint32_t* synd = nullptr;     // [types][cap][n_words[type]] (type 1 starts at cap*n_words[0])
    uint8_t* obs_true = nullptr;  // [types][cap]
    uint8_t* obs_pred = nullptr;
    uint8_t* flags = nullptr;
    int16_t* iters = nullptr;
    int32_t* lists = nullptr;     // [kTiers][cap]
    int32_t* small = nullptr;     // counts[kTiers], next[kTiers], max_s
    unsigned long long* ctr = nullptr;
    int32_t* host_small = nullptr;  // pinned mirror of `small`
    unsigned long long* host_ctr = nullptr;
    void* gscratch = nullptr;
    size_t gscratch_bytes = 0;
    int32_t* sub = nullptr;       // [kMaxGlobalClasses][sub_cap]: global-tier items by width class
    int32_t* subctr = nullptr;    // counts[kMaxGlobalClasses], next[kMaxGlobalClasses]
    int64_t sub_cap = 0;
    int32_t* host_sub = nullptr;  // pinned mirror of the class counts
    cudaStream_t aux = nullptr;   // second stream: classes of few shots run beside the others
    cudaEvent_t ev_sub = nullptr, ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_small = nullptr;
    // B-BP4MF first stage
    int64_t qcap = 0;
    uint8_t* qconv = nullptr;
    uint8_t* qobs = nullptr;     // [2][qcap]
    int16_t* qiters = nullptr;
    double* post = nullptr;      // [2][qcap][n_units]
    uint32_t* fsynd = nullptr;   // second-stage syndromes with likely edges flipped: [qcap][nw0] then [qcap][nw1]
    uint8_t* fbase = nullptr;    // [2][qcap] observable parity of the flipped edges
};

struct bp4m_graph {
    HostGraph host;
    int device = -1;
    bool uploaded = false;
    int num_sms = 0;
    float* L32[2] = {nullptr, nullptr};
    double* L64[2] = {nullptr, nullptr};
    double* W64[2] = {nullptr, nullptr};
    uint8_t* P[2] = {nullptr, nullptr};
    uint32_t* thr = nullptr;
    uint32_t* uvo = nullptr;
    uint32_t* cc_uvo = nullptr;
    // code capacity, B-BP4MF: Tanner graph and per-type CSR adjacency
    int* chk_q = nullptr;
    int* q_edge = nullptr;
    uint8_t* in_zl = nullptr;
    uint8_t* in_xl = nullptr;
    int* rw_off[2] = {nullptr, nullptr};
    uint32_t* rw_adj[2] = {nullptr, nullptr};
    int64_t table_bytes = 0;
    bool prepared[4] = {false, false, false, false};
    Workspace ws;
    // measurement: event pairs around every launch while profiling is on
    struct ProfEvent {
        int slot;
        cudaEvent_t a, b;
    };
    bool prof_on = false;
    std::vector<ProfEvent> prof_events;
    bp4m_profile_t prof{};
    // graphs of the same code and noise model re-derived for another p by
    // bp4m_sample_and_decode (least recently used last; at most kMaxDerived)
    std::vector<bp4m_graph*> derived;
};

namespace {
constexpr size_t kMaxDerived = 8;
}  // namespace

namespace {

int n_words_of(const bp4m_graph* g, int ty) { return (g->host.t[ty].n_det + 31) / 32; }

enum { PROF_CLASSIFY = 0, PROF_GLOBAL = kGlobalTier, PROF_SAMPLE = kGlobalTier + 1, PROF_COUNT = kGlobalTier + 2 };
static_assert(PROF_COUNT + 1 == BP4M_PROF_SLOTS, "profile slots");

// Brackets one kernel launch with events when profiling is on.
struct ProfScope {
    bp4m_graph* g;
    int slot;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(bp4m_graph* g_, int slot_, cudaStream_t st_) : g(g_), slot(slot_), st(st_) {
        if (g->prof_on && !tl_no_prof && cudaEventCreate(&a) == cudaSuccess) cudaEventRecord(a, st);
    }
    void end() {
        if (!a) return;
        cudaEvent_t b;
        if (cudaEventCreate(&b) == cudaSuccess) {
            cudaEventRecord(b, st);
            g->prof_events.push_back(bp4m_graph::ProfEvent{slot, a, b});
        } else {
            cudaEventDestroy(a);
        }
        a = nullptr;
    }
};

void prof_clear(bp4m_graph* g) {
    for (auto& e : g->prof_events) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    g->prof_events.clear();
    std::memset(&g->prof, 0, sizeof(g->prof));
}

void prof_add_counters(bp4m_graph* g, const unsigned long long* c) {
    if (!g->prof_on || tl_no_prof) return;
    for (int t = 0; t < kTiers; ++t) {
        g->prof.msg_updates[t] += c[C_TIER_MSGS + t];
        g->prof.shots[t] += c[C_TIER_SHOTS + t];
    }
}

DevTables dev_tables(const bp4m_graph* g, int ty) {
    DevTables t;
    t.n_det = g->host.t[ty].n_det;
    t.n_words = n_words_of(g, ty);
    t.L32 = g->L32[ty];
    t.L64 = g->L64[ty];
    t.W64 = g->W64[ty];
    t.P = g->P[ty];
    return t;
}

int ensure_uploaded(bp4m_graph* g) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (g->uploaded) {
        if (dev != g->device) return fail(BP4M_EINVAL, "graph was uploaded to another device");
        return BP4M_OK;
    }
    g->device = dev;
    CK(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev));
    const HostGraph& h = g->host;
    g->table_bytes = 0;
    for (int ty = 0; ty < h.n_types; ++ty) {
        const size_t nn = (size_t)h.t[ty].n_det * h.t[ty].n_det;
        std::vector<float> l32(nn);
        for (size_t k = 0; k < nn; ++k) {
            const double v = h.t[ty].L[k];
            // a disconnected pair keeps a finite, overwhelmingly unlikely prior
            l32[k] = std::isinf(v) ? -1.0e30f : (float)v;
        }
        std::vector<double> l64(h.t[ty].L);
        for (double& v : l64)
            if (std::isinf(v)) v = -1.0e300;
        CK(dalloc(&g->L32[ty], nn));
        CK(dalloc(&g->L64[ty], nn));
        CK(dalloc(&g->W64[ty], nn));
        CK(dalloc(&g->P[ty], nn));
        CK(cudaMemcpy(g->L32[ty], l32.data(), nn * sizeof(float), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(g->L64[ty], l64.data(), nn * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(g->W64[ty], h.t[ty].W.data(), nn * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(g->P[ty], h.t[ty].P.data(), nn, cudaMemcpyHostToDevice));
        g->table_bytes += (int64_t)nn * (sizeof(float) + 2 * sizeof(double) + 1);
    }
    auto pack = [](int u, int v, int obs) -> uint32_t {
        return (uint32_t)u | ((uint32_t)v << 15) | ((uint32_t)(obs & 1) << 31);
    };
    if (h.model == BP4M_CIRCUIT) {
        const auto& e = h.t[0].edges;
        std::vector<uint32_t> uvo(e.size());
        for (size_t k = 0; k < e.size(); ++k) uvo[k] = pack(e[k].u, e[k].v, e[k].obs);
        CK(dalloc(&g->thr, e.size()));
        CK(dalloc(&g->uvo, e.size()));
        CK(cudaMemcpy(g->thr, h.thr.data(), e.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(g->uvo, uvo.data(), e.size() * 4, cudaMemcpyHostToDevice));
        g->table_bytes += (int64_t)e.size() * 8;
    } else {
        std::vector<uint32_t> cc(2 * (size_t)h.n_units);
        for (int ty = 0; ty < 2; ++ty)
            for (int q = 0; q < h.n_units; ++q)
                cc[(size_t)ty * h.n_units + q] = pack(h.cc_u[ty][q], h.cc_v[ty][q], h.cc_obs[ty][q]);
        CK(dalloc(&g->cc_uvo, cc.size()));
        CK(cudaMemcpy(g->cc_uvo, cc.data(), cc.size() * 4, cudaMemcpyHostToDevice));
        g->table_bytes += (int64_t)cc.size() * 4;
        // Tanner graph for quaternary BP: X-checks (type 1 detectors) first, then Z-checks
        const int n = h.n_units, nx = h.t[1].n_det, nz = h.t[0].n_det, nc = nx + nz;
        std::vector<std::vector<int>> cq(nc);
        for (int q = 0; q < n; ++q) {
            for (int ty = 1; ty >= 0; --ty) {
                const int off = ty == 1 ? 0 : nx;
                cq[off + h.cc_u[ty][q]].push_back(q);
                if (h.cc_v[ty][q] < h.t[ty].n_det) cq[off + h.cc_v[ty][q]].push_back(q);
            }
        }
        std::vector<int> chk_q(4 * (size_t)nc, -1), q_edge(4 * (size_t)n, -1), qdeg(n, 0);
        for (int c = 0; c < nc; ++c) {
            std::sort(cq[c].begin(), cq[c].end());
            if (cq[c].size() > 4) return fail(BP4M_EUNSUPPORTED, "a check of weight > 4");
            for (size_t j = 0; j < cq[c].size(); ++j) {
                const int q = cq[c][j];
                chk_q[4 * c + j] = q;
                if (qdeg[q] >= 4) return fail(BP4M_EUNSUPPORTED, "a qubit in more than 4 checks");
                q_edge[4 * q + qdeg[q]++] = 4 * c + (int)j;
            }
        }
        std::vector<uint8_t> zl(n), xl(n);
        for (int q = 0; q < n; ++q) {
            zl[q] = h.cc_obs[0][q];
            xl[q] = h.cc_obs[1][q];
        }
        CK(dalloc(&g->chk_q, chk_q.size()));
        CK(dalloc(&g->q_edge, q_edge.size()));
        CK(dalloc(&g->in_zl, n));
        CK(dalloc(&g->in_xl, n));
        CK(cudaMemcpy(g->chk_q, chk_q.data(), chk_q.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(g->q_edge, q_edge.data(), q_edge.size() * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(g->in_zl, zl.data(), n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(g->in_xl, xl.data(), n, cudaMemcpyHostToDevice));
        // decoding-graph adjacency per type: entries (neighbour, qubit, obs) sorted per node by
        // (neighbour, obs, qubit), so that among equal-weight parallel edges the obs-0 one is
        // relaxed first
        for (int ty = 0; ty < 2; ++ty) {
            const int nd = h.t[ty].n_det;
            std::vector<std::vector<std::tuple<int, int, int>>> adj(nd + 1);
            for (int q = 0; q < n; ++q) {
                const int u = h.cc_u[ty][q], v = h.cc_v[ty][q], ob = h.cc_obs[ty][q];
                adj[u].emplace_back(v, ob, q);
                adj[v].emplace_back(u, ob, q);
            }
            std::vector<int> off(nd + 2, 0);
            std::vector<uint32_t> ent;
            for (int u = 0; u <= nd; ++u) {
                std::sort(adj[u].begin(), adj[u].end());
                off[u] = (int)ent.size();
                for (auto& e : adj[u])
                    ent.push_back((uint32_t)std::get<0>(e) | ((uint32_t)std::get<2>(e) << 15) |
                                  ((uint32_t)std::get<1>(e) << 31));
            }
            off[nd + 1] = (int)ent.size();
            CK(dalloc(&g->rw_off[ty], off.size()));
            CK(dalloc(&g->rw_adj[ty], ent.size()));
            CK(cudaMemcpy(g->rw_off[ty], off.data(), off.size() * 4, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(g->rw_adj[ty], ent.data(), ent.size() * 4, cudaMemcpyHostToDevice));
        }
    }
    g->uploaded = true;
    return BP4M_OK;
}

void free_ws(Workspace& w) {
    cudaFree(w.synd);
    cudaFree(w.obs_true);
    cudaFree(w.obs_pred);
    cudaFree(w.flags);
    cudaFree(w.iters);
    cudaFree(w.lists);
    cudaFree(w.small);
    cudaFree(w.ctr);
    cudaFree(w.gscratch);
    cudaFree(w.sub);
    cudaFree(w.subctr);
    cudaFreeHost(w.host_sub);
    if (w.aux) cudaStreamDestroy(w.aux);
    if (w.ev_sub) cudaEventDestroy(w.ev_sub);
    if (w.ev_fork) cudaEventDestroy(w.ev_fork);
    if (w.ev_join) cudaEventDestroy(w.ev_join);
    cudaFreeHost(w.host_small);
    cudaFreeHost(w.host_ctr);
    if (w.ev_small) cudaEventDestroy(w.ev_small);
    cudaFree(w.qconv);
    cudaFree(w.qobs);
    cudaFree(w.qiters);
    cudaFree(w.post);
    cudaFree(w.fsynd);
    cudaFree(w.fbase);
    w = Workspace();
}

int ensure_ws(bp4m_graph* g, Workspace& w, int64_t cap) {
    if (w.cap >= cap && w.small) return BP4M_OK;
    const int nt = g->host.n_types;
    void* gs = w.gscratch;
    size_t gsb = w.gscratch_bytes;
    w.gscratch = nullptr;
    free_ws(w);
    w.gscratch = gs;
    w.gscratch_bytes = gsb;
    w.cap = cap;
    w.n_types = nt;
    w.words_total = 0;
    for (int ty = 0; ty < nt; ++ty) w.words_total += n_words_of(g, ty);
    CK(dalloc(&w.synd, (size_t)cap * w.words_total));
    CK(dalloc(&w.obs_true, (size_t)cap * nt));
    CK(dalloc(&w.obs_pred, (size_t)cap * nt));
    CK(dalloc(&w.flags, (size_t)cap * nt));
    CK(dalloc(&w.iters, (size_t)cap * nt));
    CK(dalloc(&w.lists, (size_t)cap * kTiers));
    CK(dalloc(&w.small, 2 * kTiers + 1));
    CK(dalloc(&w.ctr, C_NUM));
    CK(cudaMallocHost(reinterpret_cast<void**>(&w.host_small), (2 * kTiers + 1) * sizeof(int32_t)));
    CK(cudaMallocHost(reinterpret_cast<void**>(&w.host_ctr), C_NUM * sizeof(unsigned long long)));
    CK(cudaEventCreateWithFlags(&w.ev_small, cudaEventDisableTiming));
    return BP4M_OK;
}

int ensure_ws(bp4m_graph* g, int64_t cap) { return ensure_ws(g, g->ws, cap); }

int ensure_gscratch(Workspace& w, size_t bytes) {
    if (w.gscratch_bytes >= bytes) return BP4M_OK;
    cudaFree(w.gscratch);
    w.gscratch = nullptr;
    w.gscratch_bytes = 0;
    CK(cudaMalloc(&w.gscratch, bytes));
    w.gscratch_bytes = bytes;
    return BP4M_OK;
}

int ensure_split(Workspace& w, int64_t cap) {
    if (w.sub_cap >= cap) return BP4M_OK;
    cudaFree(w.sub);
    cudaFree(w.subctr);
    w.sub = nullptr;
    w.subctr = nullptr;
    w.sub_cap = 0;
    CK(dalloc(&w.sub, (size_t)kMaxGlobalClasses * cap));
    CK(dalloc(&w.subctr, 2 * kMaxGlobalClasses));
    w.sub_cap = cap;
    if (!w.host_sub) CK(cudaMallocHost(reinterpret_cast<void**>(&w.host_sub), kMaxGlobalClasses * sizeof(int32_t)));
    if (!w.aux) CK(cudaStreamCreateWithFlags(&w.aux, cudaStreamNonBlocking));
    if (!w.ev_sub) CK(cudaEventCreateWithFlags(&w.ev_sub, cudaEventDisableTiming));
    if (!w.ev_fork) CK(cudaEventCreateWithFlags(&w.ev_fork, cudaEventDisableTiming));
    if (!w.ev_join) CK(cudaEventCreateWithFlags(&w.ev_join, cudaEventDisableTiming));
    return BP4M_OK;
}

// Scratch of the global tier split into width classes: per class its slot size, the slot
// count (one per resident block, bounded by 16 GB) and the scratch bytes of the widest need.
struct GlobalPlan {
    GlobalClasses gc;
    size_t slot_bytes[kMaxGlobalClasses];
    int gsmax[kMaxGlobalClasses];
    int full[kMaxGlobalClasses];
    size_t need = 0;        // the largest class with a slot per resident block
    size_t need_small = 0;  // a class of fewer shots than half its resident blocks
};

GlobalPlan global_plan(int prec, int max_s, int num_sms) {
    GlobalPlan p;
    p.gc = global_classes(prec, max_s);
    const size_t budget = (size_t)16 << 30;
    for (int c = 0; c < p.gc.n; ++c) {
        p.slot_bytes[c] = global_slot_bytes(prec, p.gc.smax[c], &p.gsmax[c]);
        int full = num_sms * global_blocks_per_sm(prec, p.gc.smax[c]);
        while (full > 1 && (size_t)full * p.slot_bytes[c] > budget) --full;
        p.full[c] = full;
        p.need = std::max(p.need, (size_t)full * p.slot_bytes[c]);
        p.need_small = std::max(p.need_small, (size_t)((full + 1) / 2) * p.slot_bytes[c]);
    }
    p.need = (p.need + 255) / 256 * 256;
    return p;
}

// Launches the global tier (list a.list, device count a.count) class by class: one launch
// when a single class can occur, else a partition of the list and one launch per class.
// `items` bounds the tier's count; `stride` is the per-class list capacity in w_sub.
int launch_global_classes(DecodeArgs a, const GlobalPlan& p, int prec, int64_t items, int32_t* w_sub,
                          int32_t* w_subctr, int64_t stride, int32_t* next_single, int num_sms, cudaStream_t st) {
    const size_t esz = prec == 0 ? sizeof(double) : sizeof(float);
    if (p.gc.n == 1) {
        a.next = next_single;
        a.gslot_elems = (int64_t)(p.slot_bytes[0] / esz / 3);
        a.gsmax = p.gsmax[0];
        CK(launch_decode_global(prec, a, (int)std::min<int64_t>(items, p.full[0]), st));
        return BP4M_OK;
    }
    CK(cudaMemsetAsync(w_subctr, 0, 2 * kMaxGlobalClasses * sizeof(int32_t), st));
    CK(launch_partition_global(a, p.gc, w_sub, stride, w_subctr, items, num_sms, st));
    for (int c = 0; c < p.gc.n; ++c) {
        DecodeArgs b = a;
        b.list = w_sub + (size_t)c * stride;
        b.count = w_subctr + c;
        b.next = w_subctr + kMaxGlobalClasses + c;
        b.gslot_elems = (int64_t)(p.slot_bytes[c] / esz / 3);
        b.gsmax = p.gsmax[c];
        CK(launch_decode_global(prec, b, (int)std::min<int64_t>(items, p.full[c]), st));
    }
    return BP4M_OK;
}

int ensure_qbp_ws(bp4m_graph* g, Workspace& w, int64_t cap) {
    if (w.qcap >= cap) return BP4M_OK;
    cudaFree(w.qconv);
    cudaFree(w.qobs);
    cudaFree(w.qiters);
    cudaFree(w.post);
    cudaFree(w.fsynd);
    cudaFree(w.fbase);
    w.qconv = nullptr;
    w.qobs = nullptr;
    w.qiters = nullptr;
    w.post = nullptr;
    w.fsynd = nullptr;
    w.fbase = nullptr;
    w.qcap = 0;
    CK(dalloc(&w.qconv, cap));
    CK(dalloc(&w.qobs, 2 * (size_t)cap));
    CK(dalloc(&w.qiters, cap));
    CK(dalloc(&w.post, 2 * (size_t)cap * g->host.n_units));
    CK(dalloc(&w.fsynd, (size_t)cap * (n_words_of(g, 0) + n_words_of(g, 1))));
    CK(dalloc(&w.fbase, 2 * (size_t)cap));
    w.qcap = cap;
    return BP4M_OK;
}

int check_opts(const bp4m_graph* g, const bp4m_opts* o, int iters) {
    if (!o) return fail(BP4M_EINVAL, "opts is NULL");
    if (o->precision != BP4M_FP64 && o->precision != BP4M_FP32 && o->precision != BP4M_FP16 &&
        o->precision != BP4M_BF16)
        return fail(BP4M_EINVAL, "precision must be BP4M_FP64, BP4M_FP32, BP4M_FP16 or BP4M_BF16");
    if (o->decoder == BP4M_DEC_BBP4MF && (o->precision == BP4M_FP16 || o->precision == BP4M_BF16))
        return fail(BP4M_EUNSUPPORTED, "B-BP4MF runs in FP32 or FP64");
    if (o->decoder != BP4M_DEC_BP4M && o->decoder != BP4M_DEC_BP4MF && o->decoder != BP4M_DEC_BBP4MF)
        return fail(BP4M_EINVAL, "unknown decoder");
    if (o->decoder == BP4M_DEC_BBP4MF && g->host.model != BP4M_CODE_CAPACITY)
        return fail(BP4M_EUNSUPPORTED, "B-BP4MF is implemented for code-capacity noise");
    if (!(o->alpha > 0.0)) return fail(BP4M_EINVAL, "alpha must be positive");
    if (iters < 1 || iters > 30000) return fail(BP4M_EINVAL, "iters must be in [1, 30000]");
    if (g->host.n_types == 2 && (o->type < 0 || o->type > 1))
        return fail(BP4M_EINVAL, "type must be 0 (X) or 1 (Z)");
    if (o->forced != BP4M_FORCED_GREEDY && o->forced != BP4M_FORCED_STATIC)
        return fail(BP4M_EINVAL, "forced must be BP4M_FORCED_GREEDY or BP4M_FORCED_STATIC");
    if (o->stream_cluster != 0 && o->stream_cluster != 1 && o->stream_cluster != 2 && o->stream_cluster != 4 &&
        o->stream_cluster != 8 && o->stream_cluster != 16)
        return fail(BP4M_EINVAL, "stream_cluster must be 0, 1, 2, 4, 8 or 16");
    if (o->tile_form < 0 || o->tile_form > 2) return fail(BP4M_EINVAL, "tile_form must be 0, 1 or 2");
    return BP4M_OK;
}

// Decodes `shots` device-resident syndromes of type `ty`; results go to the given device
// arrays (obs_pred / flags / iters are required here).
// B-BP4MF second stage inputs of decode_device.
struct Stage2 {
    const uint8_t* skip = nullptr;      // shots resolved by the first stage
    const uint8_t* skip_obs = nullptr;
    const int16_t* skip_iters = nullptr;
    const double* post = nullptr;       // [shots][n_units] posteriors of this type
};

int decode_device(bp4m_graph* g, Workspace& w, int ty, const uint32_t* synd, int64_t shots, int T,
                  const bp4m_opts* o, uint8_t* obs_pred, uint8_t* flags, int16_t* iters,
                  const bp4m_trace* tr, cudaStream_t st, const Stage2* rw = nullptr) {
    // pio: storage of the shared-memory tiers (0 FP64, 1 FP32, 2 FP16, 3 BF16); prec: the
    // arithmetic type of everything else (tables, global tier)
    const int pio = o->precision == BP4M_FP64 ? 0 : o->precision == BP4M_FP32 ? 1 : o->precision;
    const int prec = pio == 0 ? 0 : 1;
    if (!g->prepared[pio]) {
        CK(prepare_decode_kernels(pio));
        g->prepared[pio] = true;
    }
    const TierPlan plan = tier_plan(prec);
    CK(cudaMemsetAsync(w.small, 0, (2 * kTiers + 1) * sizeof(int32_t), st));
    {
        ProfScope ps(g, PROF_CLASSIFY, st);
        CK(launch_classify(synd, shots, n_words_of(g, ty), plan, w.lists, w.small, w.small + 2 * kTiers,
                           obs_pred, flags, iters, tr ? tr->defects : nullptr, rw ? rw->skip : nullptr,
                           rw ? rw->skip_obs : nullptr, rw ? rw->skip_iters : nullptr, st));
        ps.end();
    }
    CK(cudaMemcpyAsync(w.host_small, w.small, (2 * kTiers + 1) * sizeof(int32_t),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(w.ev_small, st));
    DecodeArgs a;
    a.tb = dev_tables(g, ty);
    a.synd = synd;
    a.shots = shots;
    a.T = T;
    a.early_exit = o->early_exit ? 1 : 0;
    a.decoder = o->decoder;
    a.forced_static = o->forced == BP4M_FORCED_STATIC ? 1 : 0;
    a.stream_cl = o->stream_cluster;
    a.tile_form = o->tile_form;
    a.alpha = o->alpha;
    a.obs_pred = obs_pred;
    a.flags = flags;
    a.iters = iters;
    a.ctr = w.ctr;
    if (tr) {
        a.tr_lambda = tr->lambda;
        a.tr_partner = tr->partner;
        a.tr_defects = tr->defects;
        a.s_cap = tr->s_cap;
    }
    if (rw) {
        // second stage of B-BP4MF: BP4MF on the reweighted priors, shared-memory tiers only
        a.decoder = BP4M_DEC_BP4MF;
        a.rw_post = rw->post;
        a.rw_off = g->rw_off[ty];
        a.rw_adj = g->rw_adj[ty];
        a.rw_units = g->host.n_units;
        const int max_tier = prec == 0 ? kRwMaxTier64 : kRwMaxTier32;
        // the tiers run one after another on `st` and share the scratch; each launch has
        // its own grid and slot size
        size_t need = 0;
        int64_t slot[kTiers] = {};
        for (int tier = 1; tier <= max_tier; ++tier) {
            const size_t b = rw_scratch_bytes(prec, tier, g->host.t[ty].n_det, g->num_sms, &slot[tier]);
            if (b == 0) return fail(BP4M_ECUDA, "B-BP4MF: no launch configuration for a reweighting tier");
            need = std::max(need, b);
        }
        int rc = ensure_gscratch(w, need);
        if (rc) return rc;
        a.gscratch = w.gscratch;
        a.gscratch_bytes = (int64_t)w.gscratch_bytes;
        for (int tier = 1; tier <= max_tier; ++tier) {
            a.rw_slot_bytes = slot[tier];
            a.list = w.lists + (size_t)tier * shots;
            a.count = w.small + tier;
            a.next = w.small + kTiers + tier;
            a.tier = tier;
            ProfScope ps(g, tier, st);
            CK(launch_decode_tier_rw(prec, tier, a, g->num_sms, st));
            ps.end();
        }
        CK(cudaEventSynchronize(w.ev_small));
        for (int tier = max_tier + 1; tier < kTiers; ++tier)
            if (w.host_small[tier] > 0)
                return fail(BP4M_EUNSUPPORTED, prec == 0 ? "B-BP4MF (FP64) decodes at most 112 unsatisfied checks of a type per shot"
                                                         : "B-BP4MF (FP32) decodes at most 160 unsatisfied checks of a type per shot");
        return BP4M_OK;
    }
    for (int tier = 1; tier < kGlobalTier; ++tier) {
        a.list = w.lists + (size_t)tier * shots;
        a.count = w.small + tier;
        a.next = w.small + kTiers + tier;
        a.tier = tier;
        ProfScope ps(g, tier, st);
        CK(launch_decode_tier(pio, tier, a, g->num_sms, st));
        ps.end();
    }
    CK(cudaEventSynchronize(w.ev_small));
    const int n_glob = w.host_small[kGlobalTier];
    if (n_glob > 0) {
        const int max_s = w.host_small[2 * kTiers];
        // width classes up to the batch's largest defect count; the scratch holds a slot for
        // every resident block of the class that needs most, whatever this batch's count, so
        // that it is reallocated (a device-wide synchronisation) only for a wider slot
        const GlobalPlan p = global_plan(pio, max_s, g->num_sms);
        int rc = ensure_gscratch(w, p.need + (p.gc.n > 1 ? p.need_small : 0));
        if (rc) return rc;
        if (p.gc.n > 1) {
            rc = ensure_split(w, shots);
            if (rc) return rc;
        }
        a.list = w.lists + (size_t)kGlobalTier * shots;
        a.count = w.small + kGlobalTier;
        a.gscratch = w.gscratch;
        a.gscratch_bytes = (int64_t)w.gscratch_bytes;
        a.tier = kGlobalTier;
        ProfScope ps(g, PROF_GLOBAL, st);
        if (p.gc.n == 1) {
            a.stream_cl = stream_cluster_for(pio, p.gsmax[0], o->stream_cluster, n_glob, p.full[0]);
            rc = launch_global_classes(a, p, pio, n_glob, w.sub, w.subctr, shots, w.small + kTiers + kGlobalTier,
                                       g->num_sms, st);
            if (rc) return rc;
        } else {
            // partition, then read the class counts: a class of fewer shots than half its
            // resident blocks (typically a few shots above the bulk's width) runs on the
            // second stream beside the others with its own scratch, instead of holding the
            // stream for a whole shot's decode on a few SMs; empty classes are skipped
            const size_t esz = prec == 0 ? sizeof(double) : sizeof(float);
            CK(cudaMemsetAsync(w.subctr, 0, 2 * kMaxGlobalClasses * sizeof(int32_t), st));
            CK(launch_partition_global(a, p.gc, w.sub, shots, w.subctr, n_glob, g->num_sms, st));
            CK(cudaMemcpyAsync(w.host_sub, w.subctr, p.gc.n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CK(cudaEventRecord(w.ev_sub, st));
            CK(cudaEventSynchronize(w.ev_sub));
            CK(cudaEventRecord(w.ev_fork, st));
            CK(cudaStreamWaitEvent(w.aux, w.ev_fork, 0));
            // small classes first, so that their few blocks hold their SMs before the large
            // classes' persistent blocks fill the rest
            for (int pass = 0; pass < 2; ++pass)
                for (int c = 0; c < p.gc.n; ++c) {
                    const int cnt = w.host_sub[c];
                    const bool small = 2 * cnt < p.full[c];
                    if (cnt <= 0 || small != (pass == 0)) continue;
                    DecodeArgs b = a;
                    b.list = w.sub + (size_t)c * shots;
                    b.count = w.subctr + c;
                    b.next = w.subctr + kMaxGlobalClasses + c;
                    b.gslot_elems = (int64_t)(p.slot_bytes[c] / esz / 3);
                    b.gsmax = p.gsmax[c];
                    b.stream_cl = stream_cluster_for(pio, b.gsmax, o->stream_cluster, cnt, p.full[c]);
                    if (small) b.gscratch = static_cast<unsigned char*>(w.gscratch) + p.need;
                    CK(launch_decode_global(pio, b, small ? cnt : std::min(cnt, p.full[c]), small ? w.aux : st));
                }
            CK(cudaEventRecord(w.ev_join, w.aux));
            CK(cudaStreamWaitEvent(st, w.ev_join, 0));
        }
        ps.end();
    }
    return BP4M_OK;
}

// B-BP4MF on device-resident syndromes of both types (type 1 = X-checks, type 0 = Z-checks).
int bbp4mf_device(bp4m_graph* g, Workspace& w, const uint32_t* synd0, const uint32_t* synd1, int64_t shots, int T,
                  const bp4m_opts* o, uint8_t* obs_pred, uint8_t* flags, int16_t* iters, cudaStream_t st) {
    int rc = ensure_qbp_ws(g, w, shots);
    if (rc) return rc;
    const int prec = o->precision == BP4M_FP64 ? 0 : 1;
    QbpArgs q;
    q.shots = shots;
    q.T = T;
    q.p = g->host.p;
    q.clamp = prec == 0 ? 1e-15 : 2.384185791015625e-07;
    q.n_qubits = g->host.n_units;
    q.n_xchecks = g->host.t[1].n_det;
    q.n_checks = g->host.t[1].n_det + g->host.t[0].n_det;
    q.n_words[0] = n_words_of(g, 0);
    q.n_words[1] = n_words_of(g, 1);
    q.synd0 = synd0;
    q.synd1 = synd1;
    q.chk_q = g->chk_q;
    q.q_edge = g->q_edge;
    q.in_zl = g->in_zl;
    q.in_xl = g->in_xl;
    q.qconv = w.qconv;
    q.qobs = w.qobs;
    q.qiters = w.qiters;
    q.post = w.post;
    {
        ProfScope ps(g, PROF_CLASSIFY, st);
        CK(launch_qbp(prec, q, g->num_sms, st));
        ps.end();
    }
    // edges above one half are taken as present: flipped syndromes and base parities
    RwFlipArgs f;
    f.shots = shots;
    f.n_units = g->host.n_units;
    for (int ty = 0; ty < 2; ++ty) {
        f.n_det[ty] = g->host.t[ty].n_det;
        f.n_words[ty] = n_words_of(g, ty);
    }
    f.synd[0] = synd0;
    f.synd[1] = synd1;
    f.post = w.post;
    f.cc_uvo = g->cc_uvo;
    f.out[0] = w.fsynd;
    f.out[1] = w.fsynd + (size_t)shots * n_words_of(g, 0);
    f.base = w.fbase;
    {
        ProfScope ps(g, PROF_CLASSIFY, st);
        CK(launch_rw_flip(f, g->num_sms, st));
        ps.end();
    }
    bp4m_opts o2 = *o;
    o2.decoder = BP4M_DEC_BP4MF;
    for (int ty = 0; ty < 2; ++ty) {
        Stage2 s2;
        s2.skip = w.qconv;
        s2.skip_obs = w.qobs + (size_t)ty * shots;
        s2.skip_iters = w.qiters;
        s2.post = w.post + (size_t)ty * shots * g->host.n_units;
        o2.type = ty;
        rc = decode_device(g, w, ty, f.out[ty], shots, T, &o2, obs_pred + (size_t)ty * shots,
                           flags + (size_t)ty * shots, iters + (size_t)ty * shots, nullptr, st, &s2);
        if (rc) return rc;
    }
    CK(launch_rw_base(obs_pred, w.qconv, w.fbase, shots, st));
    return BP4M_OK;
}

constexpr int64_t kBbpBatch = (int64_t)1 << 17;

void fill_counts(const unsigned long long* c, int n_types, bp4m_counts* out) {
    std::memset(out, 0, sizeof(*out));
    out->shots = c[C_SHOTS];
    out->fail[0] = c[C_FAIL_X];
    out->fail[1] = n_types == 2 ? c[C_FAIL_Z] : 0;
    out->fail[2] = c[C_FAIL_ANY];
    out->unconverged[0] = c[C_UNCONV_X];
    out->unconverged[1] = c[C_UNCONV_Z];
    out->forced_output[0] = c[C_FORCED_X];
    out->forced_output[1] = c[C_FORCED_Z];
    out->conv_fail[0] = c[C_CONVFAIL_X];
    out->conv_fail[1] = c[C_CONVFAIL_Z];
    out->iterations = c[C_ITERS];
    out->msg_updates = c[C_MSGS];
    out->defects = c[C_DEFECTS];
    out->forced_runs = c[C_FC_RUNS];
    out->forced_rounds = c[C_FC_ROUNDS];
    out->unconverged_any = c[C_UNCONV_ANY];
    out->conv_fail_any = c[C_CONVFAIL_ANY];
}

int sample_into(bp4m_graph* g, uint64_t first_shot, int64_t shots, uint64_t seed, uint32_t sid,
                uint32_t* synd_dev, uint8_t* obs_dev, cudaStream_t st) {
    const HostGraph& h = g->host;
    SampleArgs a;
    a.first_shot = first_shot;
    a.shots = shots;
    a.seed = seed;
    a.stream_id = sid;
    a.n_units = h.n_units;
    a.n_types = h.n_types;
    for (int ty = 0; ty < h.n_types; ++ty) {
        a.n_det[ty] = h.t[ty].n_det;
        a.n_words[ty] = n_words_of(g, ty);
    }
    a.synd = synd_dev;
    a.obs = obs_dev;
    ProfScope ps(g, PROF_SAMPLE, st);
    if (h.model == BP4M_CIRCUIT) {
        a.thr = g->thr;
        a.uvo = g->uvo;
        CK(launch_sample_circuit(a, st));
    } else {
        a.cc_uvo = g->cc_uvo;
        for (int k = 0; k < 3; ++k) a.cc_thr[k] = h.cc_thr[k];
        CK(launch_sample_code_capacity(a, st));
    }
    ps.end();
    return BP4M_OK;
}

constexpr int64_t kBatch = (int64_t)1 << 20;

}  // namespace

// ------------------------------------------------------------------ decoding service
//
// A request loop over device-resident graphs: callers submit batches of syndromes (host
// buffers) for any registered graph; worker threads, one per slot, each with its own CUDA
// stream and per-graph workspaces, take the oldest pending request and merge into it every
// pending request of the same graph and options that still fits (continuous batching).  The
// slots' copies and kernels overlap on the device.  A workspace is created the first time a
// slot decodes a graph; when the device bytes of all workspaces would exceed the budget, the
// slot frees its least recently used workspaces first, and a request whose workspace cannot
// fit at all fails with BP4M_ENOMEM.

struct bp4m_server;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct SrvRequest {
    int64_t id = 0;
    int graph = 0;
    int iters = 0;
    bp4m_opts opts{};
    int64_t shots = 0;
    std::vector<uint32_t> synd;  // [shots][n_words], copied at submission
    uint8_t* out_obs = nullptr;
    uint8_t* out_conv = nullptr;
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t batch_shots = 0;
    int slot = -1;
    int rc = 0;
    std::string err;
    bool done = false;
    // a request of a heavy graph is decoded in pieces of at most kHeavyPiece shots, each
    // piece queued behind the requests that arrived meanwhile
    int64_t taken = 0;       // shots handed to workers
    int64_t finished = 0;    // shots whose piece has completed
};

// One piece of a batch: shots [off, off + cnt) of a request.
struct SrvPiece {
    SrvRequest* r;
    int64_t off, cnt;
};

// Largest piece of a heavy graph's request: a 4096-shot request of a d = 25 circuit takes
// the whole GPU for most of a second, so it is cut into pieces and requests that arrive
// meanwhile are served between them.
constexpr int64_t kHeavyPiece = 1024;

struct SrvSlot {
    int index = 0;
    cudaStream_t st = nullptr;
    std::map<int, Workspace> ws;          // graph id -> workspace
    std::map<int, int64_t> last_use;      // graph id -> batch counter
    uint32_t* h_in = nullptr;             // pinned staging
    uint8_t* h_out = nullptr;             // [2][cap] obs, flags
    int64_t h_cap = 0, h_words = 0;
    std::thread th;
};

// Bytes of a workspace's per-shot buffers: what the service's device budget counts (the
// streaming tier's scratch, which depends on the shots' defect counts and not on the
// batch size, grows outside the budget).  The same expression sizes the admission check
// in srv_run_batch, so what a batch is admitted for is what it adds.
size_t ws_bytes(const Workspace& w) {
    return (size_t)w.cap * (w.words_total * 4 + 5 * w.n_types) + (size_t)w.cap * kTiers * 4;
}

// Mean number of unsatisfied detectors of a shot of type ty: each detector is unsatisfied
// when an odd number of its edges flip, with probability (1 - prod_e (1 - 2 q_e)) / 2
// (circuit edges carry their merged q; a code-capacity edge flips with 2p/3).
double expected_defects(const bp4m_graph* g, int ty) {
    const TypeTables& t = g->host.t[ty];
    std::vector<double> prod((size_t)t.n_det, 1.0);
    for (const Edge& e : t.edges) {
        const double q = g->host.model == BP4M_CIRCUIT ? e.q : 2.0 * g->host.p / 3.0;
        prod[(size_t)e.u] *= 1.0 - 2.0 * q;
        if (e.v < t.n_det) prod[(size_t)e.v] *= 1.0 - 2.0 * q;
    }
    double m = 0.0;
    for (double x : prod) m += 0.5 * (1.0 - x);
    return m;
}

// Admission of batches to the GPU: shared batches run together, an exclusive batch runs
// alone.  Batches are admitted in the order they reach the gate: a waiting batch is
// admitted once every batch that arrived before it has been, an exclusive one when nothing
// is running, a shared one when no exclusive batch is running.  So neither kind starves
// the other, and the pieces of a heavy request interleave with what arrived between them.
class GpuGate {
public:
    void lock_shared() { enter(false); }
    void unlock_shared() { leave(false); }
    void lock() { enter(true); }
    void unlock() { leave(true); }

private:
    void enter(bool excl) {
        std::unique_lock<std::mutex> lk(m_);
        const uint64_t me = next_++;
        waiting_.push_back(me);
        cv_.wait(lk, [&] { return waiting_.front() == me && (excl ? inside_ == 0 : !excl_inside_); });
        waiting_.pop_front();
        ++inside_;
        excl_inside_ = excl;
        cv_.notify_all();  // the next waiter may be compatible
    }
    void leave(bool excl) {
        std::lock_guard<std::mutex> lk(m_);
        --inside_;
        if (excl) excl_inside_ = false;
        cv_.notify_all();
    }
    std::mutex m_;
    std::condition_variable cv_;
    std::deque<uint64_t> waiting_;
    uint64_t next_ = 0;
    int inside_ = 0;
    bool excl_inside_ = false;
};

// Holds the gate for one batch (exclusive or shared) until it goes out of scope.
struct GateHold {
    GpuGate& g;
    bool excl;
    GateHold(GpuGate& g_, bool excl_) : g(g_), excl(excl_) {
        if (excl)
            g.lock();
        else
            g.lock_shared();
    }
    ~GateHold() {
        if (excl)
            g.unlock();
        else
            g.unlock_shared();
    }
};

bool same_batch(const SrvRequest& a, const SrvRequest& b) {
    return a.graph == b.graph && a.iters == b.iters && a.opts.precision == b.opts.precision &&
           a.opts.early_exit == b.opts.early_exit && a.opts.decoder == b.opts.decoder &&
           a.opts.alpha == b.opts.alpha && a.opts.type == b.opts.type && a.opts.forced == b.opts.forced &&
           a.opts.stream_cluster == b.opts.stream_cluster && a.opts.tile_form == b.opts.tile_form;
}

}  // namespace

struct bp4m_server {
    std::vector<bp4m_graph*> graphs;
    // per graph: its shots average more unsatisfied detectors than the shared-memory tiers
    // hold, so a batch runs in the streaming tier and fills the GPU by itself
    std::vector<char> heavy;
    // heavy batches run alone: concurrent streaming-tier launches of several slots were
    // measured to lose up to 3x of the throughput of running them one after another, so a
    // heavy batch holds this gate exclusively and every other batch holds it shared
    GpuGate gate;
    int device = -1;
    int64_t max_batch = 4096;
    int64_t budget = 0;
    std::atomic<int64_t> used{0};
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<SrvRequest*> pending;
    std::unordered_map<int64_t, SrvRequest*> reqs;
    int64_t next_id = 0;
    bool stop = false;
    std::vector<SrvSlot*> slots;
    // statistics
    int64_t n_batches = 0, n_merged = 0, shots_done = 0, evictions = 0, max_inflight = 0;
    int inflight = 0;
};

namespace {

// Device bytes that admission keeps free when the service has no explicit budget.
size_t srv_reserve_bytes(size_t total) { return std::max<size_t>((size_t)1 << 30, total / 32); }

int srv_run_batch(bp4m_server* S, SrvSlot& sl, std::vector<SrvPiece>& batch, int64_t n, int64_t stamp) {
    SrvRequest& h = *batch[0].r;
    bp4m_graph* g = nullptr;
    bool heavy = false;
    {
        std::lock_guard<std::mutex> lk(S->mu);  // bp4m_server_add_graph may grow the list
        g = S->graphs[h.graph];
        heavy = S->heavy[h.graph] != 0;
    }
    GateHold hold(S->gate, heavy);
    const int ty = g->host.n_types == 2 ? h.opts.type : 0;
    const int nw = n_words_of(g, ty);
    cudaStream_t st = sl.st;
    // workspace of this graph in this slot, within the device-memory budget
    auto it = sl.ws.find(h.graph);
    const size_t before = it == sl.ws.end() ? 0 : ws_bytes(it->second);
    Workspace& w = sl.ws[h.graph];
    sl.last_use[h.graph] = stamp;
    // per-shot buffers are sized for a full batch at once: a workspace that grew request by
    // request would free and reallocate device memory (a device-wide synchronisation that
    // stalls every other slot) each time a larger request arrived
    const int64_t cap = std::max<int64_t>(n, S->max_batch);
    if (w.cap < cap) {
        // admission: bytes of the per-shot buffers at that capacity (ensure_ws) beyond what
        // this workspace holds must fit the caller's budget, or with no budget leave at
        // least srv_reserve_bytes() of the device free; least recently used workspaces of
        // this slot are freed until they do
        size_t words = 0;
        for (int t = 0; t < g->host.n_types; ++t) words += n_words_of(g, t);
        const int64_t need = (int64_t)((size_t)cap * (words * 4 + 5 * g->host.n_types + kTiers * 4)) - (int64_t)before;
        auto fits = [&]() -> bool {
            if (S->budget > 0) return S->used.load() + need <= S->budget;
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return false;
            return (int64_t)free_b - need >= (int64_t)srv_reserve_bytes(total_b);
        };
        while (!fits()) {
            int victim = -1;
            int64_t oldest = INT64_MAX;
            for (auto& kv : sl.ws)
                if (kv.first != h.graph && sl.last_use[kv.first] < oldest) {
                    oldest = sl.last_use[kv.first];
                    victim = kv.first;
                }
            if (victim < 0)
                return fail(BP4M_ENOMEM, S->budget > 0 ? "the batch's workspace does not fit the device budget"
                                                       : "the batch's workspace does not fit the free device memory");
            S->used -= (int64_t)ws_bytes(sl.ws[victim]);
            free_ws(sl.ws[victim]);
            sl.ws.erase(victim);
            sl.last_use.erase(victim);
            std::lock_guard<std::mutex> lk(S->mu);
            ++S->evictions;
        }
    }
    int rc = ensure_ws(g, w, std::max<int64_t>(cap, w.cap));
    if (rc) return rc;
    // pinned staging, sized for the widest syndrome row of the server's graphs
    if (sl.h_cap < n || sl.h_words < nw) {
        cudaFreeHost(sl.h_in);
        cudaFreeHost(sl.h_out);
        sl.h_in = nullptr;
        sl.h_out = nullptr;
        sl.h_cap = 0;
        int64_t words = std::max<int64_t>(nw, sl.h_words);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (bp4m_graph* gg : S->graphs)
                for (int t = 0; t < gg->host.n_types; ++t) words = std::max<int64_t>(words, n_words_of(gg, t));
        }
        CK(cudaMallocHost(reinterpret_cast<void**>(&sl.h_in), (size_t)cap * words * 4));
        CK(cudaMallocHost(reinterpret_cast<void**>(&sl.h_out), (size_t)cap * 2));
        sl.h_cap = cap;
        sl.h_words = words;
    }
    int64_t off = 0;
    for (const SrvPiece& pc : batch) {
        std::memcpy(sl.h_in + (size_t)off * nw, pc.r->synd.data() + (size_t)pc.off * nw, (size_t)pc.cnt * nw * 4);
        off += pc.cnt;
    }
    CK(cudaMemcpyAsync(w.synd, sl.h_in, (size_t)n * nw * 4, cudaMemcpyHostToDevice, st));
    rc = decode_device(g, w, ty, w.synd, n, h.iters, &h.opts, w.obs_pred, w.flags, w.iters, nullptr, st);
    if (rc) return rc;
    CK(cudaMemcpyAsync(sl.h_out, w.obs_pred, (size_t)n, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(sl.h_out + n, w.flags, (size_t)n, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    S->used += (int64_t)ws_bytes(w) - (int64_t)before;
    off = 0;
    for (const SrvPiece& pc : batch) {
        std::memcpy(pc.r->out_obs + pc.off, sl.h_out + off, (size_t)pc.cnt);
        if (pc.r->out_conv)
            for (int64_t k = 0; k < pc.cnt; ++k)
                pc.r->out_conv[pc.off + k] = (uint8_t)(sl.h_out[n + off + k] & F_CONVERGED);
        off += pc.cnt;
    }
    return BP4M_OK;
}

void srv_worker(bp4m_server* S, SrvSlot* sl) {
    tl_no_prof = true;
    cudaSetDevice(S->device);
    int64_t stamp = 0;
    for (;;) {
        std::vector<SrvPiece> batch;
        int64_t n = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->pending.empty(); });
            if (S->pending.empty()) return;  // stop requested and nothing left
            SrvRequest* h = S->pending.front();
            S->pending.pop_front();
            // a heavy graph's batch is at most one piece; the rest of its request goes to the
            // back of the queue, behind what arrived meanwhile
            const int64_t limit = S->heavy[h->graph] ? std::min<int64_t>(kHeavyPiece, S->max_batch) : S->max_batch;
            const int64_t cnt = std::min<int64_t>(limit, h->shots - h->taken);
            batch.push_back(SrvPiece{h, h->taken, cnt});
            h->taken += cnt;
            n = cnt;
            if (h->taken < h->shots) S->pending.push_back(h);
            for (auto it = S->pending.begin(); it != S->pending.end();) {
                SrvRequest* r = *it;
                if (r != h && r->taken == 0 && same_batch(*h, *r) && n + r->shots <= limit) {
                    batch.push_back(SrvPiece{r, 0, r->shots});
                    r->taken = r->shots;
                    n += r->shots;
                    it = S->pending.erase(it);
                } else {
                    ++it;
                }
            }
            ++S->inflight;
            S->max_inflight = std::max<int64_t>(S->max_inflight, S->inflight);
        }
        const double t0 = now_s();
        for (const SrvPiece& pc : batch)
            if (pc.off == 0) pc.r->t_start = t0;
        const int rc = srv_run_batch(S, *sl, batch, n, ++stamp);
        const double t1 = now_s();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            --S->inflight;
            ++S->n_batches;
            S->n_merged += (int64_t)batch.size() - 1;
            if (rc == BP4M_OK) S->shots_done += n;
            for (const SrvPiece& pc : batch) {
                SrvRequest* r = pc.r;
                r->finished += pc.cnt;
                r->batch_shots = std::max<int64_t>(r->batch_shots, n);
                r->slot = sl->index;
                if (rc && !r->rc) {
                    r->rc = rc;
                    r->err = g_last_error;
                }
                if (r->finished == r->shots) {
                    r->t_done = t1;
                    r->done = true;
                    std::vector<uint32_t>().swap(r->synd);
                }
            }
        }
        S->done_cv.notify_all();
    }
}

}  // namespace

// ------------------------------------------------------------------ fused multi-graph decode
//
// Several graphs (or Pauli types of one graph) decoded together: each graph's syndromes are
// classified into shared tier lists whose items name the graph (entry << kMultiShift |
// shot), and every decode tier is one persistent launch over the shots of all graphs.
// With a fixed shot vector the whole sequence (host-to-device copies from the plan's
// pinned staging, classification, the tier launches, the streaming tier, device-to-host
// copies) has no host synchronisation, so it is captured once in a CUDA graph and
// replayed.  The tier plan (which row counts each tier takes) is chosen by timing the
// candidates on the first run (the autotuner).

struct bp4m_multi;

namespace {

struct MultiHostEntry {
    bp4m_graph* g = nullptr;
    int type = 0;
    int n_words = 0;
    int64_t cap = 0;
    uint32_t* d_synd = nullptr;
    uint8_t* d_obs = nullptr;
    uint8_t* d_flags = nullptr;
    int16_t* d_iters = nullptr;
    uint32_t* h_synd = nullptr;   // pinned
    uint8_t* h_out = nullptr;     // pinned [2][cap]: obs, flags
};

// Candidate tier plans of the autotuner, as the largest row count each FP32 tier takes;
// a tier whose bound equals the previous one's is never populated.
constexpr int kPlanCount = 3;
const int kPlanSmax[kPlanCount][kGlobalTier] = {
    {0, 32, 64, 96, 112, 128, 144, 160},   // every tier (finest padding)
    {0, 32, 64, 96, 96, 128, 128, 160},    // 32-row steps above 64
    {0, 32, 64, 64, 112, 112, 144, 160},   // 48/32-row steps
};

}  // namespace

struct bp4m_multi {
    std::vector<MultiHostEntry> e;
    int device = -1;
    int num_sms = 0;
    int iters = 0;
    bp4m_opts opts{};
    int pio = 1;
    int max_defects = 256;
    int64_t total_cap = 0;
    MultiEntry* d_entries = nullptr;
    int32_t* lists = nullptr;
    int32_t* small = nullptr;          // counts[kTiers], next[kTiers], max_s
    unsigned long long* ctr = nullptr;
    unsigned long long* h_ctr = nullptr;
    void* gscratch = nullptr;
    int32_t* sub = nullptr;       // [kMaxGlobalClasses][total_cap]
    int32_t* subctr = nullptr;
    cudaStream_t st = nullptr;
    int plan = 0;
    bool tuned = false;
    double plan_ms[kPlanCount] = {0, 0, 0};
    int stream_cl = 1;                 // streaming tier's cluster size (autotuner or opts)
    double stream_ms[2] = {0, 0};      // chosen plan with one block per shot / cluster form
    bool use_graph = true;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> graph_shots;  // shot vector the captured graph was made for
    int64_t runs = 0, replays = 0;
};

namespace {

void multi_free(bp4m_multi* m) {
    for (auto& x : m->e) {
        cudaFree(x.d_synd);
        cudaFree(x.d_obs);
        cudaFree(x.d_flags);
        cudaFree(x.d_iters);
        cudaFreeHost(x.h_synd);
        cudaFreeHost(x.h_out);
    }
    cudaFree(m->d_entries);
    cudaFree(m->lists);
    cudaFree(m->small);
    cudaFree(m->ctr);
    cudaFreeHost(m->h_ctr);
    cudaFree(m->gscratch);
    cudaFree(m->sub);
    cudaFree(m->subctr);
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->st) cudaStreamDestroy(m->st);
    delete m;
}

// Everything of one run after the host staging is filled; no host synchronisation.
int multi_enqueue(bp4m_multi* m, const std::vector<int64_t>& shots, int plan, int stream_cl) {
    cudaStream_t st = m->st;
    const int n = (int)m->e.size();
    for (int k = 0; k < n; ++k) {
        const MultiHostEntry& x = m->e[k];
        if (shots[k] > 0)
            CK(cudaMemcpyAsync(x.d_synd, x.h_synd, (size_t)shots[k] * x.n_words * 4, cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemsetAsync(m->small, 0, (2 * kTiers + 1) * sizeof(int32_t), st));
    CK(cudaMemsetAsync(m->ctr, 0, C_NUM * sizeof(unsigned long long), st));
    TierPlan tp{};
    for (int t = 0; t < kGlobalTier; ++t) tp.smax[t] = m->pio == 0 ? tier_plan(0).smax[t] : kPlanSmax[plan][t];
    tp.smax[kGlobalTier] = 0x7fffffff;
    for (int k = 0; k < n; ++k) {
        const MultiHostEntry& x = m->e[k];
        CK(launch_classify(x.d_synd, shots[k], x.n_words, tp, m->lists, m->small, m->small + 2 * kTiers, x.d_obs,
                           x.d_flags, x.d_iters, nullptr, nullptr, nullptr, nullptr, st, m->total_cap,
                           (int32_t)((int64_t)k << kMultiShift)));
    }
    DecodeArgs a;
    a.multi = m->d_entries;
    a.T = m->iters;
    a.early_exit = m->opts.early_exit ? 1 : 0;
    a.decoder = m->opts.decoder;
    a.forced_static = m->opts.forced == BP4M_FORCED_STATIC ? 1 : 0;
    a.tile_form = m->opts.tile_form;
    a.stream_cl = stream_cl;
    a.alpha = m->opts.alpha;
    a.ctr = m->ctr;
    for (int tier = 1; tier < kGlobalTier; ++tier) {
        if (m->pio != 0 && tier > 1 && kPlanSmax[plan][tier] == kPlanSmax[plan][tier - 1]) continue;
        a.list = m->lists + (size_t)tier * m->total_cap;
        a.count = m->small + tier;
        a.next = m->small + kTiers + tier;
        a.tier = tier;
        CK(launch_decode_tier(m->pio, tier, a, m->num_sms, st));
    }
    a.list = m->lists + (size_t)kGlobalTier * m->total_cap;
    a.count = m->small + kGlobalTier;
    a.tier = kGlobalTier;
    a.gscratch = m->gscratch;
    {
        // every width class up to max_defects: the counts stay on the device
        const GlobalPlan p = global_plan(m->pio, m->max_defects, m->num_sms);
        const int rc = launch_global_classes(a, p, m->pio, m->total_cap, m->sub, m->subctr, m->total_cap,
                                             m->small + kTiers + kGlobalTier, m->num_sms, st);
        if (rc) return rc;
    }
    for (int k = 0; k < n; ++k) {
        const MultiHostEntry& x = m->e[k];
        if (shots[k] <= 0) continue;
        CK(cudaMemcpyAsync(x.h_out, x.d_obs, (size_t)shots[k], cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(x.h_out + x.cap, x.d_flags, (size_t)shots[k], cudaMemcpyDeviceToHost, st));
    }
    CK(cudaMemcpyAsync(m->h_ctr, m->ctr, C_NUM * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    return BP4M_OK;
}

}  // namespace

extern "C" {

bp4m_server* bp4m_server_create(int n_slots, int64_t max_batch_shots, int64_t device_budget_bytes) {
    if (n_slots < 1 || n_slots > 64) {
        fail(BP4M_EINVAL, "n_slots must be in [1, 64]");
        return nullptr;
    }
    if (max_batch_shots < 1 || max_batch_shots > kBatch) {
        fail(BP4M_EINVAL, "max_batch_shots must be in [1, 2^20]");
        return nullptr;
    }
    if (device_budget_bytes < 0) {
        fail(BP4M_EINVAL, "device_budget_bytes must be >= 0 (0: admission by free device memory)");
        return nullptr;
    }
    bp4m_server* S = new (std::nothrow) bp4m_server();
    if (!S) {
        fail(BP4M_ENOMEM, "out of host memory");
        return nullptr;
    }
    S->max_batch = max_batch_shots;
    S->budget = device_budget_bytes;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        fail(BP4M_ECUDA, "no CUDA device");
        return nullptr;
    }
    for (int k = 0; k < n_slots; ++k) {
        SrvSlot* sl = new SrvSlot();
        sl->index = k;
        if (cudaStreamCreateWithFlags(&sl->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete sl;
            bp4m_server_destroy(S);
            fail(BP4M_ECUDA, "cudaStreamCreate failed");
            return nullptr;
        }
        S->slots.push_back(sl);
    }
    for (SrvSlot* sl : S->slots) sl->th = std::thread(srv_worker, S, sl);
    return S;
}

int bp4m_server_add_graph(bp4m_server* S, bp4m_graph* g) {
    if (!S || !g) return fail(BP4M_EINVAL, "null argument");
    int rc = ensure_uploaded(g);
    if (rc) return rc;
    if (g->device != S->device) return fail(BP4M_EINVAL, "graph lives on another device");
    for (int prec = 0; prec < 4; ++prec)
        if (!g->prepared[prec]) {
            CK(prepare_decode_kernels(prec));
            g->prepared[prec] = true;
        }
    double m = 0.0;
    for (int ty = 0; ty < g->host.n_types; ++ty) m = std::max(m, expected_defects(g, ty));
    std::lock_guard<std::mutex> lk(S->mu);
    S->graphs.push_back(g);
    S->heavy.push_back(m > 160.0 ? 1 : 0);
    return (int)S->graphs.size() - 1;
}

int64_t bp4m_server_submit(bp4m_server* S, int graph_id, const uint32_t* syndromes, int64_t shots, int iters,
                           const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* converged) {
    if (!S || !syndromes || !obs_pred) return fail(BP4M_EINVAL, "null argument");
    bp4m_graph* g;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (graph_id < 0 || graph_id >= (int)S->graphs.size()) return fail(BP4M_EINVAL, "unknown graph id");
        g = S->graphs[graph_id];
    }
    int rc = check_opts(g, opts, iters);
    if (rc) return rc;
    if (opts->decoder == BP4M_DEC_BBP4MF) return fail(BP4M_EUNSUPPORTED, "the service decodes BP4M and BP4MF");
    if (shots < 1 || shots > kBatch) return fail(BP4M_EINVAL, "shots must be in [1, 2^20]");
    if (is_device_ptr(syndromes) || is_device_ptr(obs_pred) || (converged && is_device_ptr(converged)))
        return fail(BP4M_EINVAL, "the service takes host buffers");
    const int ty = g->host.n_types == 2 ? opts->type : 0;
    const int nw = n_words_of(g, ty);
    SrvRequest* r = new (std::nothrow) SrvRequest();
    if (!r) return fail(BP4M_ENOMEM, "out of host memory");
    r->graph = graph_id;
    r->iters = iters;
    r->opts = *opts;
    r->shots = shots;
    r->synd.assign(syndromes, syndromes + (size_t)shots * nw);
    r->out_obs = obs_pred;
    r->out_conv = converged;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return fail(BP4M_EINVAL, "server is shutting down");
        }
        r->id = S->next_id++;
        S->reqs[r->id] = r;
        S->pending.push_back(r);
    }
    S->cv.notify_one();
    return r->id;
}

int bp4m_server_wait(bp4m_server* S, int64_t request, double timeout_s, bp4m_request_info* info) {
    if (!S) return fail(BP4M_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request);
    if (it == S->reqs.end()) return fail(BP4M_EINVAL, "unknown or already collected request");
    SrvRequest* r = it->second;
    const auto pred = [&] { return r->done; };
    if (timeout_s < 0)
        S->done_cv.wait(lk, pred);
    else if (!S->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), pred))
        return fail(BP4M_ETIMEOUT, "request not finished");
    if (info) {
        info->t_submit = r->t_submit;
        info->t_start = r->t_start;
        info->t_done = r->t_done;
        info->latency_s = r->t_done - r->t_submit;
        info->batch_shots = r->batch_shots;
        info->slot = r->slot;
    }
    const int rc = r->rc;
    const std::string err = r->err;
    S->reqs.erase(it);
    delete r;
    return rc ? fail(rc, err) : BP4M_OK;
}

int bp4m_server_stats(bp4m_server* S, bp4m_server_stats_t* out) {
    if (!S || !out) return fail(BP4M_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    out->batches = S->n_batches;
    out->merged_requests = S->n_merged;
    out->shots = S->shots_done;
    out->evictions = S->evictions;
    out->max_inflight_batches = S->max_inflight;
    out->pending = (int64_t)S->pending.size();
    out->device_bytes = S->used.load();
    return BP4M_OK;
}

int bp4m_server_destroy(bp4m_server* S) {
    if (!S) return BP4M_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    for (SrvSlot* sl : S->slots)
        if (sl->th.joinable()) sl->th.join();
    for (SrvSlot* sl : S->slots) {
        for (auto& kv : sl->ws) free_ws(kv.second);
        cudaFreeHost(sl->h_in);
        cudaFreeHost(sl->h_out);
        if (sl->st) cudaStreamDestroy(sl->st);
        delete sl;
    }
    for (auto& kv : S->reqs) delete kv.second;
    delete S;
    return BP4M_OK;
}

bp4m_multi* bp4m_multi_create(int n, bp4m_graph* const* graphs, const int* types, const int64_t* max_shots,
                              int iters, const bp4m_opts* opts, int max_defects, int use_cuda_graph) {
    if (n < 1 || n > 1000 || !graphs || !max_shots) {
        fail(BP4M_EINVAL, "need 1..1000 graphs and their capacities");
        return nullptr;
    }
    if (!opts || (opts->precision != BP4M_FP32 && opts->precision != BP4M_FP16 && opts->precision != BP4M_BF16)) {
        fail(BP4M_EINVAL, "the fused decode runs in FP32, FP16 or BF16");
        return nullptr;
    }
    if (opts->decoder != BP4M_DEC_BP4M && opts->decoder != BP4M_DEC_BP4MF) {
        fail(BP4M_EUNSUPPORTED, "the fused decode runs BP4M and BP4MF");
        return nullptr;
    }
    if (max_defects < 161 || max_defects > 1024) {
        fail(BP4M_EINVAL, "max_defects must be in [161, 1024]");
        return nullptr;
    }
    bp4m_multi* m = new (std::nothrow) bp4m_multi();
    if (!m) {
        fail(BP4M_ENOMEM, "out of host memory");
        return nullptr;
    }
    m->iters = iters;
    m->opts = *opts;
    m->pio = opts->precision;
    m->max_defects = max_defects;
    m->use_graph = use_cuda_graph != 0;
    std::vector<MultiEntry> host(n);
    auto bad = [&](int rc) -> bp4m_multi* {
        multi_free(m);
        (void)rc;
        return nullptr;
    };
    for (int k = 0; k < n; ++k) {
        bp4m_graph* g = graphs[k];
        if (!g) return bad(fail(BP4M_EINVAL, "null graph"));
        int rc = ensure_uploaded(g);
        if (rc) return bad(rc);
        if (k == 0) {
            m->device = g->device;
            m->num_sms = g->num_sms;
        } else if (g->device != m->device) {
            return bad(fail(BP4M_EINVAL, "graphs on different devices"));
        }
        rc = check_opts(g, opts, iters);
        if (rc) return bad(rc);
        if (max_shots[k] < 1 || max_shots[k] > kMultiMask) return bad(fail(BP4M_EINVAL, "max_shots must be in [1, 2^21)"));
        MultiHostEntry x;
        x.g = g;
        x.type = g->host.n_types == 2 ? (types ? types[k] : 0) : 0;
        if (x.type < 0 || x.type >= g->host.n_types) return bad(fail(BP4M_EINVAL, "bad Pauli type"));
        x.n_words = n_words_of(g, x.type);
        x.cap = max_shots[k];
        m->e.push_back(x);
        MultiHostEntry& y = m->e.back();
        if (dalloc(&y.d_synd, (size_t)y.cap * y.n_words) != cudaSuccess || dalloc(&y.d_obs, (size_t)y.cap) != cudaSuccess ||
            dalloc(&y.d_flags, (size_t)y.cap) != cudaSuccess || dalloc(&y.d_iters, (size_t)y.cap) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&y.h_synd), (size_t)y.cap * y.n_words * 4) != cudaSuccess ||
            cudaMallocHost(reinterpret_cast<void**>(&y.h_out), (size_t)y.cap * 2) != cudaSuccess)
            return bad(fail(BP4M_ENOMEM, "out of memory for the fused decode's buffers"));
        host[k].tb = dev_tables(g, y.type);
        host[k].synd = y.d_synd;
        host[k].obs_pred = y.d_obs;
        host[k].flags = y.d_flags;
        host[k].iters = y.d_iters;
        m->total_cap += y.cap;
        if (!g->prepared[m->pio]) {
            if (prepare_decode_kernels(m->pio) != cudaSuccess) return bad(fail(BP4M_ECUDA, "kernel set-up failed"));
            g->prepared[m->pio] = true;
        }
    }
    if (dalloc(&m->d_entries, (size_t)n) != cudaSuccess || dalloc(&m->lists, (size_t)m->total_cap * kTiers) != cudaSuccess ||
        dalloc(&m->small, 2 * kTiers + 1) != cudaSuccess || dalloc(&m->ctr, C_NUM) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&m->h_ctr), C_NUM * sizeof(unsigned long long)) != cudaSuccess)
        return bad(fail(BP4M_ENOMEM, "out of memory for the fused decode's lists"));
    if (cudaMemcpy(m->d_entries, host.data(), sizeof(MultiEntry) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return bad(fail(BP4M_ECUDA, "upload of the entries failed"));
    // streaming tier: per width class up to max_defects one slot per resident block
    {
        const GlobalPlan p = global_plan(m->pio, max_defects, m->num_sms);
        if (cudaMalloc(&m->gscratch, p.need) != cudaSuccess)
            return bad(fail(BP4M_ENOMEM, "out of memory for the streaming tier's scratch"));
        if (dalloc(&m->sub, (size_t)kMaxGlobalClasses * m->total_cap) != cudaSuccess ||
            dalloc(&m->subctr, 2 * kMaxGlobalClasses) != cudaSuccess)
            return bad(fail(BP4M_ENOMEM, "out of memory for the streaming tier's lists"));
    }
    if (cudaStreamCreateWithFlags(&m->st, cudaStreamNonBlocking) != cudaSuccess)
        return bad(fail(BP4M_ECUDA, "cudaStreamCreate failed"));
    return m;
}

int bp4m_multi_run(bp4m_multi* m, const uint32_t* const* syndromes, const int64_t* shots, uint8_t* const* obs_pred,
                   uint8_t* const* converged) {
    if (!m || !syndromes || !shots || !obs_pred) return fail(BP4M_EINVAL, "null argument");
    const int n = (int)m->e.size();
    std::vector<int64_t> sh(shots, shots + n);
    for (int k = 0; k < n; ++k) {
        if (sh[k] < 0 || sh[k] > m->e[k].cap) return fail(BP4M_EINVAL, "shots exceed the entry's capacity");
        if (sh[k] > 0 && (!syndromes[k] || !obs_pred[k])) return fail(BP4M_EINVAL, "null buffer");
        if (sh[k] > 0) std::memcpy(m->e[k].h_synd, syndromes[k], (size_t)sh[k] * m->e[k].n_words * 4);
    }
    if (cudaSetDevice(m->device) != cudaSuccess) return fail(BP4M_ECUDA, "cudaSetDevice failed");
    if (!m->tuned) {
        // autotuner: time every candidate tier plan on this run's shots, keep the fastest
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        // time one plan: a warm run (first use of its kernels), then a timed one
        auto time_plan = [&](int pl, int cl, double* ms_out) -> int {
            int rc = multi_enqueue(m, sh, pl, cl);
            if (rc) return rc;
            CK(cudaEventRecord(e0, m->st));
            rc = multi_enqueue(m, sh, pl, cl);
            if (rc) return rc;
            CK(cudaEventRecord(e1, m->st));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            *ms_out = ms;
            return BP4M_OK;
        };
        const int cl_opt = m->opts.stream_cluster;
        const int cl0 = cl_opt > 1 ? cl_opt : 1;
        for (int pl = 0; pl < kPlanCount; ++pl) {
            const int rc = time_plan(pl, cl0, &m->plan_ms[pl]);
            if (rc) return rc;
        }
        m->plan = (int)(std::min_element(m->plan_ms, m->plan_ms + kPlanCount) - m->plan_ms);
        m->stream_cl = cl0;
        // the streaming tier's block shape: with the automatic choice, the chosen plan once
        // more with the cluster form (each width's default size), kept if faster
        if (cl_opt == 0 && m->pio != 0 && m->max_defects > tier_plan(m->pio).smax[kGlobalTier - 1]) {
            m->stream_ms[0] = m->plan_ms[m->plan];
            const int rc = time_plan(m->plan, 16, &m->stream_ms[1]);
            if (rc) return rc;
            if (m->stream_ms[1] < m->stream_ms[0]) m->stream_cl = 16;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        m->tuned = true;
    } else if (m->use_graph) {
        if (!m->exec || m->graph_shots != sh) {
            if (m->exec) cudaGraphExecDestroy(m->exec);
            m->exec = nullptr;
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(m->st, cudaStreamCaptureModeThreadLocal));
            const int rc = multi_enqueue(m, sh, m->plan, m->stream_cl);
            const cudaError_t ce = cudaStreamEndCapture(m->st, &graph);
            if (rc) return rc;
            CK(ce);
            const cudaError_t ie = cudaGraphInstantiate(&m->exec, graph, 0);
            cudaGraphDestroy(graph);
            CK(ie);
            m->graph_shots = sh;
        }
        CK(cudaGraphLaunch(m->exec, m->st));
        ++m->replays;
    } else {
        const int rc = multi_enqueue(m, sh, m->plan, m->stream_cl);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(m->st));
    ++m->runs;
    for (int k = 0; k < n; ++k) {
        if (sh[k] <= 0) continue;
        const MultiHostEntry& x = m->e[k];
        std::memcpy(obs_pred[k], x.h_out, (size_t)sh[k]);
        if (converged && converged[k])
            for (int64_t j = 0; j < sh[k]; ++j) converged[k][j] = (uint8_t)(x.h_out[x.cap + j] & F_CONVERGED);
    }
    if (m->h_ctr[C_ERRORS])
        return fail(BP4M_EUNSUPPORTED, std::to_string(m->h_ctr[C_ERRORS]) + " shots exceed max_defects unsatisfied detectors");
    return BP4M_OK;
}

int bp4m_multi_info(const bp4m_multi* m, bp4m_multi_info_t* out) {
    if (!m || !out) return fail(BP4M_EINVAL, "null argument");
    out->plan = m->plan;
    for (int k = 0; k < 3; ++k) out->plan_ms[k] = m->plan_ms[k];
    out->runs = m->runs;
    out->graph_replays = m->replays;
    out->msg_updates = m->h_ctr ? m->h_ctr[C_MSGS] : 0;
    out->stream_cluster = m->stream_cl;
    out->stream_ms[0] = m->stream_ms[0];
    out->stream_ms[1] = m->stream_ms[1];
    return BP4M_OK;
}

void bp4m_multi_destroy(bp4m_multi* m) {
    if (m) multi_free(m);
}

const char* bp4m_last_error(void) { return g_last_error.c_str(); }

const char* bp4m_version(void) { return "bp4m-gb300 0.1 (sm_103a)"; }

int bp4m_build_graph(const bp4m_code* code, const bp4m_noise* noise, bp4m_graph** out) {
    if (!code || !noise || !out) return fail(BP4M_EINVAL, "null argument");
    *out = nullptr;
    bp4m_graph* g = new (std::nothrow) bp4m_graph();
    if (!g) return fail(BP4M_ENOMEM, "host allocation failed");
    std::string err;
    int rc;
    try {
        rc = build_host_graph(*code, *noise, g->host, err);
    } catch (const std::bad_alloc&) {
        rc = BP4M_ENOMEM;
        err = "host allocation failed while building the graph";
    }
    if (rc != BP4M_OK) {
        delete g;
        return fail(rc, err);
    }
    *out = g;
    return BP4M_OK;
}

int bp4m_graph_info(const bp4m_graph* g, bp4m_graph_info_t* out) {
    if (!g || !out) return fail(BP4M_EINVAL, "null argument");
    std::memset(out, 0, sizeof(*out));
    const HostGraph& h = g->host;
    out->n_types = h.n_types;
    for (int ty = 0; ty < h.n_types; ++ty) {
        out->n_det[ty] = h.t[ty].n_det;
        out->n_words[ty] = (h.t[ty].n_det + 31) / 32;
        out->n_edges[ty] = (int)h.t[ty].edges.size();
    }
    out->n_units = h.n_units;
    out->model = h.model;
    out->d = h.d;
    out->rounds = h.rounds;
    out->p = h.p;
    int64_t tb = 0;
    for (int ty = 0; ty < h.n_types; ++ty)
        tb += (int64_t)h.t[ty].n_det * h.t[ty].n_det * (int64_t)(sizeof(float) + 2 * sizeof(double) + 1);
    tb += h.model == BP4M_CIRCUIT ? (int64_t)h.n_units * 8 : (int64_t)h.n_units * 8;
    out->table_bytes = tb;
    for (int ty = 0; ty < h.n_types; ++ty) out->mean_defects[ty] = expected_defects(g, ty);
    return BP4M_OK;
}

int bp4m_graph_export(const bp4m_graph* g, int type, int what, void* out, size_t bytes) {
    if (!g || !out) return fail(BP4M_EINVAL, "null argument");
    const HostGraph& h = g->host;
    if (type < 0 || type >= h.n_types) return fail(BP4M_EINVAL, "type out of range");
    const TypeTables& t = h.t[type];
    const size_t nn = (size_t)t.n_det * t.n_det;
    switch (what) {
        case BP4M_EXPORT_W:
            if (bytes < nn * 8) return fail(BP4M_EINVAL, "buffer too small");
            std::memcpy(out, t.W.data(), nn * 8);
            return BP4M_OK;
        case BP4M_EXPORT_L:
            if (bytes < nn * 8) return fail(BP4M_EINVAL, "buffer too small");
            std::memcpy(out, t.L.data(), nn * 8);
            return BP4M_OK;
        case BP4M_EXPORT_PARITY:
            if (bytes < nn) return fail(BP4M_EINVAL, "buffer too small");
            std::memcpy(out, t.P.data(), nn);
            return BP4M_OK;
        case BP4M_EXPORT_EDGES: {
            if (bytes < t.edges.size() * sizeof(bp4m_edge)) return fail(BP4M_EINVAL, "buffer too small");
            bp4m_edge* e = static_cast<bp4m_edge*>(out);
            for (size_t k = 0; k < t.edges.size(); ++k)
                e[k] = bp4m_edge{t.edges[k].u, t.edges[k].v, t.edges[k].obs, 0, t.edges[k].q};
            return BP4M_OK;
        }
        case BP4M_EXPORT_THRESH:
            if (h.model == BP4M_CIRCUIT) {
                if (bytes < h.thr.size() * 4) return fail(BP4M_EINVAL, "buffer too small");
                std::memcpy(out, h.thr.data(), h.thr.size() * 4);
            } else {
                if (bytes < 12) return fail(BP4M_EINVAL, "buffer too small");
                std::memcpy(out, h.cc_thr, 12);
            }
            return BP4M_OK;
        default:
            return fail(BP4M_EINVAL, "unknown export");
    }
}

int bp4m_sample(bp4m_graph* g, uint64_t first_shot, int64_t shots, uint64_t seed,
                uint32_t stream_id, uint32_t* syndromes, uint8_t* obs_true, void* stream) {
    if (!g || !syndromes || !obs_true) return fail(BP4M_EINVAL, "null argument");
    if (shots < 0 || shots > ((int64_t)1 << 31)) return fail(BP4M_EINVAL, "shots out of range");
    if (shots == 0) return BP4M_OK;
    int rc = ensure_uploaded(g);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool dev_s = is_device_ptr(syndromes), dev_o = is_device_ptr(obs_true);
    const int nt = g->host.n_types;
    size_t words = 0;
    for (int ty = 0; ty < nt; ++ty) words += n_words_of(g, ty);
    for (int64_t off = 0; off < shots; off += kBatch) {
        const int64_t nb = std::min(kBatch, shots - off);
        // layout per batch is [types][nb][words]; assemble the caller's [types][shots] layout
        uint32_t* sd;
        uint8_t* od;
        const bool direct = dev_s && dev_o && nb == shots;
        if (direct) {
            sd = syndromes;
            od = obs_true;
        } else {
            rc = ensure_ws(g, std::max<int64_t>(nb, g->ws.cap));
            if (rc) return rc;
            sd = g->ws.synd;
            od = g->ws.obs_true;
        }
        rc = sample_into(g, first_shot + (uint64_t)off, nb, seed, stream_id, sd, od, st);
        if (rc) return rc;
        if (!direct) {
            size_t woff = 0;
            for (int ty = 0; ty < nt; ++ty) {
                const int nw = n_words_of(g, ty);
                uint32_t* dst = syndromes + (size_t)shots * woff + (size_t)off * nw;
                CK(cudaMemcpyAsync(dst, sd + (size_t)nb * woff, (size_t)nb * nw * 4,
                                   cudaMemcpyDefault, st));
                CK(cudaMemcpyAsync(obs_true + (size_t)ty * shots + off, od + (size_t)ty * nb, nb,
                                   cudaMemcpyDefault, st));
                woff += nw;
            }
            CK(cudaStreamSynchronize(st));
        }
    }
    CK(cudaStreamSynchronize(st));
    return BP4M_OK;
}

static int decode_common(bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                         const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* converged,
                         int16_t* iters_used, const bp4m_trace* tr, void* stream) {
    if (!g || !syndromes) return fail(BP4M_EINVAL, "null argument");
    if (shots < 0 || shots > ((int64_t)1 << 31)) return fail(BP4M_EINVAL, "shots out of range");
    int rc = check_opts(g, opts, iters);
    if (rc) return rc;
    if (tr && (tr->s_cap < 1 || tr->s_cap > 4096)) return fail(BP4M_EINVAL, "trace s_cap out of range");
    if (opts->decoder == BP4M_DEC_BBP4MF)
        return fail(BP4M_EINVAL, "B-BP4MF decodes both Pauli types together: use bp4m_decode_bbp4mf");
    if (shots == 0) return BP4M_OK;
    rc = ensure_uploaded(g);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ty = g->host.n_types == 2 ? opts->type : 0;
    const int nw = n_words_of(g, ty);
    const bool dev_in = is_device_ptr(syndromes);
    if (tr) {
        if ((tr->lambda && !is_device_ptr(tr->lambda)) || (tr->partner && !is_device_ptr(tr->partner)) ||
            (tr->defects && !is_device_ptr(tr->defects)) || (tr->flags && !is_device_ptr(tr->flags)))
            return fail(BP4M_EINVAL, "trace buffers must be device memory");
        if (shots > kBatch) return fail(BP4M_EINVAL, "traced decodes take at most 2^20 shots");
    }
    rc = ensure_ws(g, std::max<int64_t>(std::min(kBatch, shots), g->ws.cap));
    if (rc) return rc;
    CK(cudaMemsetAsync(g->ws.ctr, 0, C_NUM * sizeof(unsigned long long), st));
    for (int64_t off = 0; off < shots; off += kBatch) {
        const int64_t nb = std::min(kBatch, shots - off);
        Workspace& w = g->ws;
        const uint32_t* sd = syndromes + (size_t)off * nw;
        if (!dev_in) {
            CK(cudaMemcpyAsync(w.synd, sd, (size_t)nb * nw * 4, cudaMemcpyHostToDevice, st));
            sd = w.synd;
        }
        rc = decode_device(g, w, ty, sd, nb, iters, opts, w.obs_pred, w.flags, w.iters, tr, st);
        if (rc) return rc;
        if (tr && tr->flags) CK(cudaMemcpyAsync(tr->flags, w.flags, nb, cudaMemcpyDeviceToDevice, st));
        if (obs_pred) CK(cudaMemcpyAsync(obs_pred + off, w.obs_pred, nb, cudaMemcpyDefault, st));
        if (iters_used) CK(cudaMemcpyAsync(iters_used + off, w.iters, nb * 2, cudaMemcpyDefault, st));
        if (converged) {
            if (is_device_ptr(converged)) {
                finalize_kernel<<<(int)std::min<int64_t>((nb + 255) / 256, 4096), 256, 0, st>>>(
                    w.flags, nb, converged + off);
                CK(cudaGetLastError());
            } else {
                std::vector<uint8_t> fl(nb);
                CK(cudaMemcpyAsync(fl.data(), w.flags, nb, cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                for (int64_t k = 0; k < nb; ++k) converged[off + k] = (fl[k] & F_CONVERGED) ? 1 : 0;
            }
        }
        CK(cudaStreamSynchronize(st));
    }
    Workspace& w = g->ws;
    CK(cudaMemcpyAsync(w.host_ctr, w.ctr, C_NUM * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (w.host_ctr[C_ERRORS]) return fail(BP4M_ECUDA, "decoder kernels rejected shots (internal size check)");
    prof_add_counters(g, w.host_ctr);
    return BP4M_OK;
}

int bp4m_decode_batch(bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                      const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* converged,
                      int16_t* iters_used, void* stream) {
    return decode_common(g, syndromes, shots, iters, opts, obs_pred, converged, iters_used, nullptr,
                         stream);
}

int bp4m_decode_trace(bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                      const bp4m_opts* opts, uint8_t* obs_pred, const bp4m_trace* trace,
                      void* stream) {
    if (!trace) return fail(BP4M_EINVAL, "trace is NULL");
    return decode_common(g, syndromes, shots, iters, opts, obs_pred, nullptr, nullptr, trace, stream);
}

int bp4m_sample_and_decode_range(bp4m_graph* g, uint64_t first_shot, int64_t shots, uint64_t seed,
                                 uint32_t stream_id, int iters, const bp4m_opts* opts,
                                 bp4m_counts* out, void* stream) {
    if (!g || !out) return fail(BP4M_EINVAL, "null argument");
    if (shots < 0) return fail(BP4M_EINVAL, "shots must be non-negative");
    int rc = check_opts(g, opts, iters);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    if (shots == 0) return BP4M_OK;
    rc = ensure_uploaded(g);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool bbp = opts->decoder == BP4M_DEC_BBP4MF;
    const int64_t cap = std::min(bbp ? kBbpBatch : kBatch, shots);
    rc = ensure_ws(g, std::max<int64_t>(cap, g->ws.cap));
    if (rc) return rc;
    Workspace& w = g->ws;
    const int nt = g->host.n_types;
    CK(cudaMemsetAsync(w.ctr, 0, C_NUM * sizeof(unsigned long long), st));
    for (int64_t off = 0; off < shots; off += cap) {
        const int64_t nb = std::min(cap, shots - off);
        rc = sample_into(g, first_shot + (uint64_t)off, nb, seed, stream_id, w.synd, w.obs_true, st);
        if (rc) return rc;
        if (bbp) {
            rc = bbp4mf_device(g, w, w.synd, w.synd + (size_t)nb * n_words_of(g, 0), nb, iters, opts, w.obs_pred,
                               w.flags, w.iters, st);
            if (rc) return rc;
            ProfScope ps(g, PROF_COUNT, st);
            CK(launch_count(w.obs_true, w.obs_pred, w.flags, nb, nt, w.ctr, st));
            ps.end();
            continue;
        }
        size_t woff = 0;
        for (int ty = 0; ty < nt; ++ty) {
            bp4m_opts o = *opts;
            o.type = ty;
            rc = decode_device(g, w, ty, w.synd + (size_t)nb * woff, nb, iters, &o, w.obs_pred + (size_t)ty * nb,
                               w.flags + (size_t)ty * nb, w.iters + (size_t)ty * nb, nullptr, st);
            if (rc) return rc;
            woff += n_words_of(g, ty);
        }
        ProfScope ps(g, PROF_COUNT, st);
        CK(launch_count(w.obs_true, w.obs_pred, w.flags, nb, nt, w.ctr, st));
        ps.end();
    }
    CK(cudaMemcpyAsync(w.host_ctr, w.ctr, C_NUM * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (w.host_ctr[C_ERRORS]) return fail(BP4M_ECUDA, "decoder kernels rejected shots (internal size check)");
    prof_add_counters(g, w.host_ctr);
    fill_counts(w.host_ctr, nt, out);
    return BP4M_OK;
}

int bp4m_sample_and_decode(bp4m_graph* g, double p, int64_t shots, uint64_t seed, int iters,
                           const bp4m_opts* opts, bp4m_counts* out, void* stream) {
    if (!g) return fail(BP4M_EINVAL, "null graph");
    if (p == g->host.p) return bp4m_sample_and_decode_range(g, 0, shots, seed, 0, iters, opts, out, stream);
    if (!(p > 0.0 && p < 0.5)) return fail(BP4M_EINVAL, "p must lie in (0, 0.5)");
    // another p: the priors (and for circuits the merged edge probabilities and every
    // shortest path) depend on it, so the graph is re-derived from the same code and noise
    // options, cached per p and uploaded on its first decoding call
    bp4m_graph* dg = nullptr;
    for (size_t k = 0; k < g->derived.size(); ++k)
        if (g->derived[k]->host.p == p) {
            dg = g->derived[k];
            g->derived.erase(g->derived.begin() + (std::ptrdiff_t)k);
            break;
        }
    if (!dg) {
        const HostGraph& h = g->host;
        bp4m_code code{h.family, h.d, h.model == BP4M_CIRCUIT ? h.rounds : 0, BP4M_MEMORY_Z};
        bp4m_noise noise{h.model, p, h.prior_conv, h.through_boundary};
        int rc = bp4m_build_graph(&code, &noise, &dg);
        if (rc != BP4M_OK) return rc;
        if (g->derived.size() >= kMaxDerived) {
            bp4m_free_graph(g->derived.front());
            g->derived.erase(g->derived.begin());
        }
    }
    g->derived.push_back(dg);
    if (dg->prof_on != g->prof_on) {
        prof_clear(dg);
        dg->prof_on = g->prof_on;
    }
    return bp4m_sample_and_decode_range(dg, 0, shots, seed, 0, iters, opts, out, stream);
}

int bp4m_decode_bbp4mf(bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                       const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* flags, void* stream) {
    if (!g || !syndromes || !obs_pred) return fail(BP4M_EINVAL, "null argument");
    if (g->host.model != BP4M_CODE_CAPACITY) return fail(BP4M_EUNSUPPORTED, "B-BP4MF is implemented for code-capacity noise");
    if (shots < 0 || shots > ((int64_t)1 << 31)) return fail(BP4M_EINVAL, "shots out of range");
    if (!opts) return fail(BP4M_EINVAL, "opts is NULL");
    bp4m_opts o = *opts;
    o.decoder = BP4M_DEC_BBP4MF;
    int rc = check_opts(g, &o, iters);
    if (rc) return rc;
    if (shots == 0) return BP4M_OK;
    rc = ensure_uploaded(g);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nw0 = n_words_of(g, 0), nw1 = n_words_of(g, 1);
    for (int64_t off = 0; off < shots; off += kBbpBatch) {
        const int64_t nb = std::min(kBbpBatch, shots - off);
        rc = ensure_ws(g, std::max<int64_t>(nb, g->ws.cap));
        if (rc) return rc;
        Workspace& w = g->ws;
        CK(cudaMemcpyAsync(w.synd, syndromes + (size_t)off * nw0, (size_t)nb * nw0 * 4, cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(w.synd + (size_t)nb * nw0, syndromes + (size_t)shots * nw0 + (size_t)off * nw1,
                           (size_t)nb * nw1 * 4, cudaMemcpyDefault, st));
        CK(cudaMemsetAsync(w.ctr, 0, C_NUM * sizeof(unsigned long long), st));
        rc = bbp4mf_device(g, w, w.synd, w.synd + (size_t)nb * nw0, nb, iters, &o, w.obs_pred, w.flags, w.iters, st);
        if (rc) return rc;
        for (int ty = 0; ty < 2; ++ty) {
            CK(cudaMemcpyAsync(obs_pred + (size_t)ty * shots + off, w.obs_pred + (size_t)ty * nb, nb,
                               cudaMemcpyDefault, st));
            if (flags)
                CK(cudaMemcpyAsync(flags + (size_t)ty * shots + off, w.flags + (size_t)ty * nb, nb, cudaMemcpyDefault, st));
        }
        CK(cudaStreamSynchronize(st));
    }
    return BP4M_OK;
}

int bp4m_decode_noalloc(const bp4m_graph* g, const uint32_t* syndromes, int64_t shots, int iters,
                        const bp4m_opts* opts, uint8_t* obs_pred, uint8_t* converged,
                        int16_t* iters_used, void* stream) {
    // No allocation on any path of this function: it reads the graph's resident tables
    // and uses the library's static scratch array (see launch_decode_noalloc).
    if (!g || !syndromes) return fail(BP4M_EINVAL, "null argument");
    // the kernel's work counter is a 32-bit int that every block bumps once past the last
    // shot: keep it clear of overflow
    if (shots < 0 || shots > noalloc_max_shots()) return fail(BP4M_EINVAL, "shots out of range");
    int rc = check_opts(g, opts, iters);
    if (rc) return rc;
    if (opts->precision == BP4M_FP16 || opts->precision == BP4M_BF16)
        return fail(BP4M_EUNSUPPORTED, "bp4m_decode_noalloc runs in FP32 or FP64");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (!g->uploaded || g->device != dev)
        return fail(BP4M_EINVAL, "the graph's tables are not on this device: run one bp4m_decode_batch on it "
                                 "during set-up first");
    if (!is_device_ptr(syndromes) || (obs_pred && !is_device_ptr(obs_pred)) ||
        (converged && !is_device_ptr(converged)) || (iters_used && !is_device_ptr(iters_used)))
        return fail(BP4M_EINVAL, "bp4m_decode_noalloc takes device buffers only");
    if (shots == 0) return BP4M_OK;
    const int ty = g->host.n_types == 2 ? opts->type : 0;
    DecodeArgs a;
    a.tb = dev_tables(g, ty);
    a.synd = syndromes;
    a.shots = shots;
    a.T = iters;
    a.early_exit = opts->early_exit ? 1 : 0;
    a.decoder = opts->decoder;
    a.forced_static = opts->forced == BP4M_FORCED_STATIC ? 1 : 0;
    a.stream_cl = opts->stream_cluster;
    a.tile_form = opts->tile_form;
    a.alpha = opts->alpha;
    a.obs_pred = obs_pred;
    a.flags = converged;
    a.flags_mode = 1;
    a.iters = iters_used;
    a.ctr = nullptr;
    int too_many = 0;
    cudaError_t e = launch_decode_noalloc(opts->precision == BP4M_FP64 ? 0 : 1, a, shots,
                                          static_cast<cudaStream_t>(stream), &too_many);
    if (too_many)
        return fail(BP4M_EINVAL, "a shot has more than " + std::to_string(noalloc_max_defects()) +
                                     " unsatisfied detectors, the limit of bp4m_decode_noalloc");
    if (e != cudaSuccess) return cuda_fail(e, "bp4m_decode_noalloc");
    return BP4M_OK;
}

int bp4m_profile_enable(bp4m_graph* g, int on) {
    if (!g) return fail(BP4M_EINVAL, "null graph");
    for (bp4m_graph* x : g->derived) {
        prof_clear(x);
        x->prof_on = on != 0;
    }
    prof_clear(g);
    g->prof_on = on != 0;
    return BP4M_OK;
}

namespace {
int prof_collect(bp4m_graph* g) {
    for (auto& e : g->prof_events) {
        CK(cudaEventSynchronize(e.b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e.a, e.b));
        g->prof.ms[e.slot] += ms;
        g->prof.launches[e.slot] += 1;
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    g->prof_events.clear();
    return BP4M_OK;
}
}  // namespace

int bp4m_profile_read(bp4m_graph* g, bp4m_profile_t* out) {
    if (!g || !out) return fail(BP4M_EINVAL, "null argument");
    int rc = prof_collect(g);
    if (rc) return rc;
    *out = g->prof;
    // launches made through graphs re-derived for another p count as this graph's
    for (bp4m_graph* x : g->derived) {
        rc = prof_collect(x);
        if (rc) return rc;
        for (int k = 0; k < BP4M_PROF_SLOTS; ++k) {
            out->launches[k] += x->prof.launches[k];
            out->ms[k] += x->prof.ms[k];
            out->msg_updates[k] += x->prof.msg_updates[k];
            out->shots[k] += x->prof.shots[k];
        }
    }
    return BP4M_OK;
}

int bp4m_probe_mufu(int steps, double* out, void* stream) {
    if (!out || steps < 1 || steps > (1 << 20)) return fail(BP4M_EINVAL, "null output or steps outside 1..2^20");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    long long* cyc = nullptr;
    float* sink = nullptr;
    CK(dalloc(&cyc, (size_t)sms));
    cudaError_t e = dalloc(&sink, (size_t)sms * 1024);
    if (e != cudaSuccess) {
        cudaFree(cyc);
        return cuda_fail(e, "bp4m_probe_mufu");
    }
    std::vector<long long> h((size_t)sms);
    int rc = BP4M_OK;
    for (int mode = 0; mode < 3 && rc == BP4M_OK; ++mode) {
        // one untimed launch to load the kernel and warm the clocks, then the measured one
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) e = launch_mufu_probe(mode, sms, steps, cyc, sink, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * (size_t)sms, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "bp4m_probe_mufu");
            break;
        }
        std::sort(h.begin(), h.end());
        const double ops = 1024.0 * mufu_probe_ops_per_thread(mode, steps);
        out[mode] = ops / (double)std::max<long long>(h[(size_t)sms / 2], 1);
    }
    if (rc == BP4M_OK) out[3] = sms;
    cudaFree(cyc);
    cudaFree(sink);
    return rc;
}

void bp4m_free_graph(bp4m_graph* g) {
    if (!g) return;
    for (bp4m_graph* x : g->derived) bp4m_free_graph(x);
    g->derived.clear();
    if (g->uploaded) prof_clear(g);
    if (g->uploaded) {
        for (int ty = 0; ty < 2; ++ty) {
            cudaFree(g->L32[ty]);
            cudaFree(g->L64[ty]);
            cudaFree(g->W64[ty]);
            cudaFree(g->P[ty]);
        }
        cudaFree(g->thr);
        cudaFree(g->uvo);
        cudaFree(g->cc_uvo);
        cudaFree(g->chk_q);
        cudaFree(g->q_edge);
        cudaFree(g->in_zl);
        cudaFree(g->in_xl);
        for (int ty = 0; ty < 2; ++ty) {
            cudaFree(g->rw_off[ty]);
            cudaFree(g->rw_adj[ty]);
        }
        free_ws(g->ws);
    }
    delete g;
}

}  // extern "C"
