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
    std::vector<int> quads;                   // [ne][4] (a, b, c, d); edge e is (b, c) of quad e
    std::vector<double> L0, theta0, S0;       // [ne], [ne], [nt]
    double Sg0 = 0.0, V0 = 0.0;
    // device evaluation order of each element list (edges go with their
    // quads): consecutive groups of 32 elements touch pairwise-different
    // nodes where possible, so the lanes of a warp add to different nodes'
    // force sums
    std::vector<int> quad_order, tri_order;
};

// Greedy packing of elements (node lists of `arity` ids each) into groups of
// `width` with disjoint nodes; returns the evaluation order.
std::vector<int> conflict_free_order(const std::vector<int> &nodes, int arity, int width);

bool build_template(const double *xyz, int nn, const int32_t *tris, int nt, const double stretch[3],
                    Topology &out, std::string &err);

// Mesh orientation (Sec. 5, mesh analysis).  mode 0: report the triangles
// that a repair would turn; 1: repair; 2: flip every triangle.  The repair
// makes the orientation consistent across shared edges (breadth-first from
// triangle 0 over each connected component) and then turns a component
// whose divergence-theorem volume is negative, so that AB x AC points
// inside; unlike a per-triangle test against the centroid this also holds
// for concave meshes.  out: the resulting triangles (may alias nothing);
// changed: number of triangles turned.  Returns false with err for a mesh
// that is not a closed orientable 2-manifold.
bool orient_mesh(const double *xyz, int nn, const int32_t *tris, int nt, int mode, int32_t *out, int &changed,
                 std::string &err);

}  // namespace lbib
