// Host-side template topology and relaxed state (see topology.cpp).
#pragma once

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

namespace lbib {

struct Topology {
    int nn = 0, nt = 0, ne = 0;
    std::vector<double> x;                    // stretched rest coordinates [nn][3]
    std::vector<int> tri;                     // [nt][3] as given
    std::vector<int> edges;                   // [ne][2], i < j, lexicographic
    std::vector<int> quads;                   // [ne][4] (a, b, c, d)
    std::vector<double> L0, theta0, S0;       // [ne], [ne], [nt]
    double Sg0 = 0.0, V0 = 0.0;
    // device evaluation order of each element list: consecutive groups of 32
    // elements touch pairwise-different nodes where possible, so the lanes of
    // a warp add to different nodes' force sums
    std::vector<int> edge_order, quad_order, tri_order;
};

// Greedy packing of elements (node lists of `arity` ids each) into groups of
// `width` with disjoint nodes; returns the evaluation order.
std::vector<int> conflict_free_order(const std::vector<int> &nodes, int arity, int width);

bool build_template(const double *xyz, int nn, const int32_t *tris, int nt, const double stretch[3],
                    Topology &out, std::string &err);

}  // namespace lbib
