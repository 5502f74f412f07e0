// Host-side static graph construction: rotated surface code geometry, the memory-Z
// circuit's detector error model, the merged detector graph and the per-pair tables
// (shortest-path weight W, prior LLR l of Eq. (priorllr), observable parity).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "bp4m.h"

namespace bp4m {

struct Edge {
    int u;       // detector, u < v
    int v;       // detector or n_det (boundary)
    int obs;     // observable bit
    double q;    // merged flip probability (circuit); 0 for code capacity edges
};

struct TypeTables {
    int n_det = 0;
    std::vector<Edge> edges;      // canonical order
    std::vector<double> W;        // n_det * n_det, row-major, diagonal = boundary
    std::vector<double> L;        // prior LLR, same layout
    std::vector<uint8_t> P;       // observable parity, same layout
};

struct HostGraph {
    int model = 0;
    int family = 0;
    int d = 0;
    int rounds = 0;
    double p = 0.0;
    int prior_conv = 0;
    int through_boundary = 0;
    int n_types = 1;
    TypeTables t[2];
    // code capacity sampler data: per data qubit and type, the edge endpoints and obs bit
    std::vector<int32_t> cc_u[2], cc_v[2];
    std::vector<uint8_t> cc_obs[2];
    uint32_t cc_thr[3] = {0, 0, 0};
    // circuit sampler data: one threshold per canonical edge of type 0
    std::vector<uint32_t> thr;
    int n_units = 0;
};

// Returns BP4M_OK or a negative code with `err` set.
int build_host_graph(const bp4m_code& code, const bp4m_noise& noise, HostGraph& g,
                     std::string& err);

}  // namespace bp4m
