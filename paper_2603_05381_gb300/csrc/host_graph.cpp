// Static graph construction on the host.
//
// Code capacity (Sec. "MWPM on the surface code"): the decoding graph of one Pauli type
// has a node per check of the matching type and an edge per data qubit between its one
// or two checks (one check: an edge to the boundary).
//
// Circuit level (Sec. "Numerical Results"): the memory-Z circuit with d rounds,
// depolarizing noise of strength p after every gate, on the data before every round and on
// idle qubits of every gate layer, and flips of probability p after resets and before
// measurements.  Every non-identity Pauli of a channel is an independent mechanism.  Its
// effect on the Z-detectors and the observable is found by FORWARD Pauli-frame simulation,
// 64 mechanisms at a time in the bits of a machine word.  Mechanisms with equal effect are
// merged (odd-parity probability, folded over the probabilities in ascending order).
//
// Priors (Eq. (two-syn var factors) and Eq. (priorllr)): W_ij is the shortest path between
// detectors i and j with edge weights ln((1-q)/q) (code capacity: hops times
// ln((1-p)/p)), W_ii the shortest path to the boundary; l = -W - log1p(-exp(-W)).
// Parallel edges keep the smaller weight (ties: observable bit 0); pair paths do not pass
// through the boundary unless requested; Dijkstra finalises nodes in (distance, index)
// order and changes a predecessor only on a strict improvement, and the parity of a path
// is accumulated along its predecessor tree.
//
// This file must be compiled without floating-point contraction so that the merged
// probabilities and path sums are the plain IEEE results of the expressions written here.
#include "host_graph.h"

#include <algorithm>
#include <cmath>
#include <functional>
#include <limits>
#include <map>
#include <queue>
#include <thread>
#include <tuple>
#include <utility>

namespace bp4m {
namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

struct Check {
    int row, col;               // position (rotated: north-west corner of the plaquette)
    std::vector<int> qubits;    // data qubits, ascending
    int sched[4];               // data qubit met in each CNOT step, -1 for none
};

struct CodeLayout {
    int n = 0;                  // data qubits
    std::vector<Check> xs, zs;  // X- and Z-checks in (row, col) order
    std::vector<char> in_zl;    // data qubit in supp(Z_L)
    std::vector<char> in_xl;    // data qubit in supp(X_L)
};

// Rotated code.  Data (r, c) in [0, d)^2, index r*d + c.  Plaquette (pr, pc) covers data
// (pr..pr+1, pc..pc+1); X-type iff pr+pc is even.  Kept: every weight-4 plaquette;
// weight-2 ones on the top/bottom edges if Z-type and on the left/right edges if X-type.
// Z_L = column 0, X_L = row 0.  CNOT order: X-checks NW, SW, NE, SE; Z-checks NW, NE,
// SW, SE.
CodeLayout rotated_layout(int d) {
    CodeLayout L;
    L.n = d * d;
    const int xo[4][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}};
    const int zo[4][2] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}};
    auto at = [d](int r, int c) { return (r >= 0 && r < d && c >= 0 && c < d) ? r * d + c : -1; };
    for (int pr = -1; pr < d; ++pr) {
        for (int pc = -1; pc < d; ++pc) {
            Check ch{pr, pc, {}, {-1, -1, -1, -1}};
            for (int dr = 0; dr < 2; ++dr)
                for (int dc = 0; dc < 2; ++dc) {
                    const int q = at(pr + dr, pc + dc);
                    if (q >= 0) ch.qubits.push_back(q);
                }
            const bool x_type = (((pr + pc) % 2) + 2) % 2 == 0;
            bool keep;
            if (ch.qubits.size() == 4) {
                keep = true;
            } else if (ch.qubits.size() == 2) {
                const bool top_bottom = (pr == -1 || pr == d - 1);
                keep = top_bottom ? !x_type : x_type;
            } else {
                keep = false;
            }
            if (!keep) continue;
            const int(*o)[2] = x_type ? xo : zo;
            for (int k = 0; k < 4; ++k) ch.sched[k] = at(pr + o[k][0], pc + o[k][1]);
            std::sort(ch.qubits.begin(), ch.qubits.end());
            (x_type ? L.xs : L.zs).push_back(ch);
        }
    }
    L.in_zl.assign(L.n, 0);
    L.in_xl.assign(L.n, 0);
    for (int r = 0; r < d; ++r) L.in_zl[r * d] = 1;
    for (int c = 0; c < d; ++c) L.in_xl[c] = 1;
    return L;
}

// Unrotated code.  A (2d-1) x (2d-1) grid; data at (r, c) with r + c even, numbered
// row-major; Z-checks at (r odd, c even), X-checks at (r even, c odd), each acting on its
// N, S, W, E neighbours.  Z_L = data row 0, X_L = data column 0.  CNOT order: X-checks
// N, W, E, S; Z-checks N, E, W, S.
CodeLayout unrotated_layout(int d) {
    CodeLayout L;
    const int G = 2 * d - 1;
    std::vector<int> index(G * G, -1);
    for (int r = 0; r < G; ++r)
        for (int c = 0; c < G; ++c)
            if ((r + c) % 2 == 0) index[r * G + c] = L.n++;
    auto at = [&](int r, int c) { return (r >= 0 && r < G && c >= 0 && c < G) ? index[r * G + c] : -1; };
    const int N[2] = {-1, 0}, S[2] = {1, 0}, W[2] = {0, -1}, E[2] = {0, 1};
    const int* xo[4] = {N, W, E, S};
    const int* zo[4] = {N, E, W, S};
    for (int r = 0; r < G; ++r)
        for (int c = 0; c < G; ++c) {
            if ((r + c) % 2 == 0) continue;
            const bool z_type = r % 2 == 1;
            Check ch{r, c, {}, {-1, -1, -1, -1}};
            const int* const* o = z_type ? zo : xo;
            for (int k = 0; k < 4; ++k) {
                ch.sched[k] = at(r + o[k][0], c + o[k][1]);
                if (ch.sched[k] >= 0) ch.qubits.push_back(ch.sched[k]);
            }
            std::sort(ch.qubits.begin(), ch.qubits.end());
            (z_type ? L.zs : L.xs).push_back(ch);
        }
    L.in_zl.assign(L.n, 0);
    L.in_xl.assign(L.n, 0);
    for (int c = 0; c < G; c += 2) L.in_zl[at(0, c)] = 1;
    for (int r = 0; r < G; r += 2) L.in_xl[at(r, 0)] = 1;
    return L;
}

// ---------------------------------------------------------------- circuit model

enum class OpK { Reset, Had, Cnot, MeasReset, Meas, Dep1, Dep2, Flip };

struct Op {
    OpK k;
    std::vector<int> a;  // qubits, or first element of each pair
    std::vector<int> b;  // second element of each pair (Cnot: target, Dep2: second qubit)
    double p = 0.0;
    int rec0 = 0;        // first measurement record of this op
};

struct Circuit {
    int nq = 0;
    int n_records = 0;
    std::vector<Op> ops;
    std::vector<std::vector<int>> zdet;  // record lists, canonical order
    std::vector<int> obs;
};

Circuit memory_z(const CodeLayout& lay, int d, double p) {
    const int n = lay.n, nx = (int)lay.xs.size(), nz = (int)lay.zs.size();
    const std::vector<Check>& zs = lay.zs;
    Circuit c;
    c.nq = n + nx + nz;
    std::vector<int> data(n), xa(nx), za(nz), anc, all(c.nq);
    for (int i = 0; i < n; ++i) data[i] = i;
    for (int i = 0; i < nx; ++i) xa[i] = n + i;
    for (int i = 0; i < nz; ++i) za[i] = n + nx + i;
    anc = xa;
    anc.insert(anc.end(), za.begin(), za.end());
    for (int i = 0; i < c.nq; ++i) all[i] = i;
    std::vector<int> idle_h = data;
    idle_h.insert(idle_h.end(), za.begin(), za.end());

    // CNOT layers in the checks' schedule: the ancilla controls for X-checks, the data
    // qubit controls for Z-checks.
    std::vector<Op> cx_layers(4);
    std::vector<std::vector<int>> idle_cx(4);
    for (int k = 0; k < 4; ++k) {
        Op op{OpK::Cnot, {}, {}, 0.0, 0};
        std::vector<char> busy(c.nq, 0);
        for (int a = 0; a < nx; ++a) {
            const int q = lay.xs[a].sched[k];
            if (q >= 0) {
                op.a.push_back(xa[a]);
                op.b.push_back(q);
            }
        }
        for (int a = 0; a < nz; ++a) {
            const int q = zs[a].sched[k];
            if (q >= 0) {
                op.a.push_back(q);
                op.b.push_back(za[a]);
            }
        }
        for (size_t e = 0; e < op.a.size(); ++e) busy[op.a[e]] = busy[op.b[e]] = 1;
        for (int q = 0; q < c.nq; ++q)
            if (!busy[q]) idle_cx[k].push_back(q);
        cx_layers[k] = op;
    }

    auto noise1 = [&](OpK k, const std::vector<int>& qs) {
        if (p > 0.0 && !qs.empty()) c.ops.push_back(Op{k, qs, {}, p, 0});
    };
    int rec = 0;
    std::vector<std::vector<int>> zrec(d, std::vector<int>(nz));
    c.ops.push_back(Op{OpK::Reset, all, {}, 0.0, 0});
    noise1(OpK::Flip, all);
    for (int rnd = 0; rnd < d; ++rnd) {
        noise1(OpK::Dep1, data);
        c.ops.push_back(Op{OpK::Had, xa, {}, 0.0, 0});
        noise1(OpK::Dep1, xa);
        noise1(OpK::Dep1, idle_h);
        for (int k = 0; k < 4; ++k) {
            c.ops.push_back(cx_layers[k]);
            if (p > 0.0) {
                Op dn{OpK::Dep2, cx_layers[k].a, cx_layers[k].b, p, 0};
                c.ops.push_back(dn);
            }
            noise1(OpK::Dep1, idle_cx[k]);
        }
        c.ops.push_back(Op{OpK::Had, xa, {}, 0.0, 0});
        noise1(OpK::Dep1, xa);
        noise1(OpK::Dep1, idle_h);
        noise1(OpK::Flip, anc);
        Op m{OpK::MeasReset, anc, {}, 0.0, rec};
        c.ops.push_back(m);
        for (int a = 0; a < nz; ++a) zrec[rnd][a] = rec + nx + a;
        rec += nx + nz;
        noise1(OpK::Flip, anc);
    }
    noise1(OpK::Flip, data);
    c.ops.push_back(Op{OpK::Meas, data, {}, 0.0, rec});
    const int drec = rec;
    rec += n;
    c.n_records = rec;

    for (int rnd = 0; rnd < d; ++rnd)
        for (int a = 0; a < nz; ++a) {
            if (rnd == 0)
                c.zdet.push_back({zrec[0][a]});
            else
                c.zdet.push_back({zrec[rnd][a], zrec[rnd - 1][a]});
        }
    for (int a = 0; a < nz; ++a) {
        std::vector<int> det{zrec[d - 1][a]};
        for (int q : zs[a].qubits) det.push_back(drec + q);
        c.zdet.push_back(det);
    }
    for (int q = 0; q < n; ++q)
        if (lay.in_zl[q]) c.obs.push_back(drec + q);
    return c;
}

struct Fault {
    int op;
    int idx;      // target (or pair) index inside the op
    uint8_t pa;   // Pauli on the first qubit: bit0 = X, bit1 = Z
    uint8_t pb;   // Pauli on the second qubit (two-qubit channels)
    double prob;
};

std::vector<Fault> enumerate_faults(const Circuit& c) {
    std::vector<Fault> f;
    for (int o = 0; o < (int)c.ops.size(); ++o) {
        const Op& op = c.ops[o];
        if (op.k == OpK::Dep1) {
            for (int i = 0; i < (int)op.a.size(); ++i)
                for (uint8_t pa = 1; pa < 4; ++pa) f.push_back(Fault{o, i, pa, 0, op.p / 3.0});
        } else if (op.k == OpK::Dep2) {
            for (int i = 0; i < (int)op.a.size(); ++i)
                for (uint8_t pa = 0; pa < 4; ++pa)
                    for (uint8_t pb = 0; pb < 4; ++pb)
                        if (pa | pb) f.push_back(Fault{o, i, pa, pb, op.p / 15.0});
        } else if (op.k == OpK::Flip) {
            for (int i = 0; i < (int)op.a.size(); ++i) f.push_back(Fault{o, i, 1, 0, op.p});
        }
    }
    return f;
}

// Effects of every fault: a list of Z-detectors (sorted) and the observable bit.
struct Effect {
    std::vector<int> dets;
    int obs;
};

std::vector<Effect> simulate_faults(const Circuit& c, const std::vector<Fault>& faults) {
    const int nf = (int)faults.size();
    std::vector<Effect> out(nf);
    std::vector<uint64_t> X(c.nq), Z(c.nq), rec(c.n_records);
    const int ndet = (int)c.zdet.size();
    std::vector<uint64_t> detw(ndet);
    for (int f0 = 0; f0 < nf; f0 += 64) {
        const int f1 = std::min(nf, f0 + 64);
        std::fill(X.begin(), X.end(), 0);
        std::fill(Z.begin(), Z.end(), 0);
        std::fill(rec.begin(), rec.end(), 0);
        int ptr = f0;
        for (int o = faults[f0].op; o < (int)c.ops.size(); ++o) {
            const Op& op = c.ops[o];
            switch (op.k) {
                case OpK::Reset:
                    for (int q : op.a) X[q] = Z[q] = 0;
                    break;
                case OpK::Had:
                    for (int q : op.a) std::swap(X[q], Z[q]);
                    break;
                case OpK::Cnot:
                    for (size_t e = 0; e < op.a.size(); ++e) {
                        X[op.b[e]] ^= X[op.a[e]];
                        Z[op.a[e]] ^= Z[op.b[e]];
                    }
                    break;
                case OpK::MeasReset:
                    for (size_t e = 0; e < op.a.size(); ++e) {
                        int q = op.a[e];
                        rec[op.rec0 + e] = X[q];
                        X[q] = Z[q] = 0;
                    }
                    break;
                case OpK::Meas:
                    for (size_t e = 0; e < op.a.size(); ++e) rec[op.rec0 + e] = X[op.a[e]];
                    break;
                default:
                    while (ptr < f1 && faults[ptr].op == o) {
                        const Fault& ft = faults[ptr];
                        const uint64_t bit = 1ull << (ptr - f0);
                        int q1 = op.a[ft.idx];
                        if (ft.pa & 1) X[q1] ^= bit;
                        if (ft.pa & 2) Z[q1] ^= bit;
                        if (op.k == OpK::Dep2) {
                            int q2 = op.b[ft.idx];
                            if (ft.pb & 1) X[q2] ^= bit;
                            if (ft.pb & 2) Z[q2] ^= bit;
                        }
                        ++ptr;
                    }
                    break;
            }
        }
        for (int j = 0; j < ndet; ++j) {
            uint64_t w = 0;
            for (int m : c.zdet[j]) w ^= rec[m];
            detw[j] = w;
        }
        uint64_t ow = 0;
        for (int m : c.obs) ow ^= rec[m];
        for (int j = 0; j < ndet; ++j) {
            uint64_t w = detw[j];
            while (w) {
                int b = __builtin_ctzll(w);
                w &= w - 1;
                out[f0 + b].dets.push_back(j);
            }
        }
        for (int b = 0; b < f1 - f0; ++b) out[f0 + b].obs = (int)((ow >> b) & 1ull);
    }
    return out;
}

double odd_parity_merge(std::vector<double> qs) {
    std::sort(qs.begin(), qs.end());
    double acc = 0.0;
    for (double q2 : qs) acc = acc * (1.0 - q2) + q2 * (1.0 - acc);
    return acc;
}

// ---------------------------------------------------------------- shortest paths

struct Arc {
    int v;
    double w;
    int obs;
};

std::vector<std::vector<Arc>> build_adjacency(int n_det, const std::vector<Edge>& edges,
                                              const std::vector<double>& w) {
    std::map<std::pair<int, int>, std::pair<double, int>> best;
    for (size_t e = 0; e < edges.size(); ++e) {
        auto key = std::make_pair(edges[e].u, edges[e].v);
        auto cand = std::make_pair(w[e], edges[e].obs);
        auto it = best.find(key);
        if (it == best.end() || cand < it->second) best[key] = cand;
    }
    std::vector<std::vector<Arc>> adj(n_det + 1);
    for (auto& kv : best) {
        adj[kv.first.first].push_back(Arc{kv.first.second, kv.second.first, kv.second.second});
        adj[kv.first.second].push_back(Arc{kv.first.first, kv.second.first, kv.second.second});
    }
    return adj;
}

void all_pairs(int n_det, const std::vector<std::vector<Arc>>& adj, bool through_boundary,
               double scale, TypeTables& t) {
    const int n = n_det;
    t.W.assign((size_t)n * n, kInf);
    t.P.assign((size_t)n * n, 0);
    auto worker = [&](int lo, int hi) {
        std::vector<double> dist(n + 1);
        std::vector<uint8_t> par(n + 1), done(n + 1);
        using Item = std::pair<double, int>;
        for (int src = lo; src < hi; ++src) {
            std::fill(dist.begin(), dist.end(), kInf);
            std::fill(par.begin(), par.end(), 0);
            std::fill(done.begin(), done.end(), 0);
            std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
            dist[src] = 0.0;
            heap.push(Item(0.0, src));
            while (!heap.empty()) {
                Item it = heap.top();
                heap.pop();
                const int u = it.second;
                if (done[u]) continue;
                done[u] = 1;
                if (u == n && !through_boundary) continue;
                for (const Arc& a : adj[u]) {
                    const double nd = it.first + a.w;
                    if (nd < dist[a.v]) {
                        dist[a.v] = nd;
                        par[a.v] = (uint8_t)(par[u] ^ a.obs);
                        heap.push(Item(nd, a.v));
                    }
                }
            }
            t.W[(size_t)src * n + src] = dist[n] * scale;
            t.P[(size_t)src * n + src] = par[n];
            for (int j = src + 1; j < n; ++j) {
                t.W[(size_t)src * n + j] = dist[j] * scale;
                t.P[(size_t)src * n + j] = par[j];
            }
        }
    };
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    int nthreads = (int)std::min<unsigned>(hw, 64u);
    if (n < 64) nthreads = 1;
    std::vector<std::thread> pool;
    // interleave rows so that long (small index) and short rows spread across threads
    std::vector<int> order;
    for (int r = 0; r < nthreads; ++r) pool.emplace_back([&, r]() {
        for (int src = r; src < n; src += nthreads) worker(src, src + 1);
    });
    for (auto& th : pool) th.join();
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            t.W[(size_t)j * n + i] = t.W[(size_t)i * n + j];
            t.P[(size_t)j * n + i] = t.P[(size_t)i * n + j];
        }
    t.L.resize((size_t)n * n);
    for (size_t k = 0; k < t.W.size(); ++k) {
        const double W = t.W[k];
        t.L[k] = std::isinf(W) ? -kInf : -W - std::log1p(-std::exp(-W));
    }
}

}  // namespace

int build_host_graph(const bp4m_code& code, const bp4m_noise& noise, HostGraph& g,
                     std::string& err) {
    if (code.family != BP4M_ROTATED && code.family != BP4M_UNROTATED) {
        err = "unknown code family";
        return BP4M_EINVAL;
    }
    if (code.basis != BP4M_MEMORY_Z) {
        err = "only the memory-Z experiment is implemented";
        return BP4M_EUNSUPPORTED;
    }
    if (code.d < 3 || code.d % 2 == 0 || code.d > 41) {
        err = "distance must be odd and in [3, 41]";
        return BP4M_EINVAL;
    }
    if (!(noise.p > 0.0 && noise.p < 0.5)) {
        err = "p must lie in (0, 0.5)";
        return BP4M_EINVAL;
    }
    if (noise.prior_conv != BP4M_PRIOR_P && noise.prior_conv != BP4M_PRIOR_2P3) {
        err = "unknown prior convention";
        return BP4M_EINVAL;
    }
    const int d = code.d;
    g.model = noise.model;
    g.d = d;
    g.p = noise.p;
    g.prior_conv = noise.prior_conv;
    g.through_boundary = noise.pair_through_boundary ? 1 : 0;
    const CodeLayout lay = code.family == BP4M_ROTATED ? rotated_layout(d) : unrotated_layout(d);
    g.family = code.family;

    if (noise.model == BP4M_CODE_CAPACITY) {
        if (code.rounds != 0) {
            err = "code capacity takes rounds = 0";
            return BP4M_EINVAL;
        }
        g.rounds = 0;
        g.n_types = 2;
        g.n_units = lay.n;
        for (int k = 1; k <= 3; ++k)
            g.cc_thr[k - 1] = (uint32_t)std::floor((double)k * noise.p / 3.0 * 4294967296.0);
        const double pp = noise.prior_conv == BP4M_PRIOR_P ? noise.p : 2.0 * noise.p / 3.0;
        const double c = std::log((1.0 - pp) / pp);
        for (int ty = 0; ty < 2; ++ty) {
            // type 0: X errors on the Z-checks, obs = qubit in supp(Z_L);
            // type 1: Z errors on the X-checks, obs = qubit in supp(X_L)
            const std::vector<Check>& chk = ty == 0 ? lay.zs : lay.xs;
            TypeTables& t = g.t[ty];
            t.n_det = (int)chk.size();
            std::vector<std::vector<int>> touch(lay.n);
            for (int a = 0; a < t.n_det; ++a)
                for (int q : chk[a].qubits) touch[q].push_back(a);
            g.cc_u[ty].resize(lay.n);
            g.cc_v[ty].resize(lay.n);
            g.cc_obs[ty].resize(lay.n);
            for (int q = 0; q < lay.n; ++q) {
                std::vector<int> ts = touch[q];
                std::sort(ts.begin(), ts.end());
                int u, v;
                if (ts.size() == 1) {
                    u = ts[0];
                    v = t.n_det;
                } else if (ts.size() == 2) {
                    u = ts[0];
                    v = ts[1];
                } else {
                    err = "geometry error: a qubit touches 0 or >2 checks of one type";
                    return BP4M_EINVAL;
                }
                const int obs = ty == 0 ? lay.in_zl[q] : lay.in_xl[q];
                g.cc_u[ty][q] = u;
                g.cc_v[ty][q] = v;
                g.cc_obs[ty][q] = (uint8_t)obs;
                t.edges.push_back(Edge{u, v, obs, 0.0});
            }
            std::vector<double> w(t.edges.size(), 1.0);
            auto adj = build_adjacency(t.n_det, t.edges, w);
            all_pairs(t.n_det, adj, g.through_boundary != 0, c, t);
        }
        return BP4M_OK;
    }
    if (noise.model != BP4M_CIRCUIT) {
        err = "unknown noise model";
        return BP4M_EINVAL;
    }
    if (code.rounds != 0 && code.rounds != d) {
        err = "circuit experiments use rounds = d (pass 0 or d)";
        return BP4M_EUNSUPPORTED;
    }
    g.rounds = d;
    g.n_types = 1;
    Circuit c = memory_z(lay, d, noise.p);
    std::vector<Fault> faults = enumerate_faults(c);
    std::vector<Effect> eff = simulate_faults(c, faults);
    const int n_det = (int)c.zdet.size();
    std::map<std::tuple<int, int, int>, std::vector<double>> groups;
    for (size_t f = 0; f < faults.size(); ++f) {
        const Effect& e = eff[f];
        if (e.dets.empty()) {
            if (e.obs) {
                err = "circuit has an undetectable logical mechanism";
                return BP4M_EUNSUPPORTED;
            }
            continue;
        }
        if (e.dets.size() > 2) {
            err = "non-graphlike Z-part in the circuit model";
            return BP4M_EUNSUPPORTED;
        }
        int u = e.dets[0];
        int v = e.dets.size() == 2 ? e.dets[1] : n_det;
        groups[std::make_tuple(u, v, e.obs)].push_back(faults[f].prob);
    }
    TypeTables& t = g.t[0];
    t.n_det = n_det;
    for (auto& kv : groups)
        t.edges.push_back(Edge{std::get<0>(kv.first), std::get<1>(kv.first),
                               std::get<2>(kv.first), odd_parity_merge(kv.second)});
    g.n_units = (int)t.edges.size();
    g.thr.resize(t.edges.size());
    std::vector<double> w(t.edges.size());
    for (size_t e = 0; e < t.edges.size(); ++e) {
        const double q = t.edges[e].q;
        g.thr[e] = (uint32_t)std::floor(q * 4294967296.0);
        w[e] = std::log((1.0 - q) / q);
    }
    auto adj = build_adjacency(n_det, t.edges, w);
    all_pairs(n_det, adj, g.through_boundary != 0, 1.0, t);
    return BP4M_OK;
}

}  // namespace bp4m
