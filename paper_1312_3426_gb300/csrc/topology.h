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

// Evaluation order of elements (node lists of `arity` ids each) for the
// membrane kernel, whose warps take `width` (32) consecutive elements, one
// per lane, and for each node slot k load the staged positions (16 bytes per
// node, 8 lanes per shared-memory wavefront) and add forces (4 bytes per node
// and component, 32 banks).  Greedy, lane by lane: each lane takes, among the
// first `window` remaining elements, the first of least cost, where a node
// already in the group costs most, then each slot's node index sharing its
// residue mod 32 with an earlier lane of the group (an atomic bank
// conflict), then mod 8 with an earlier lane of the same quarter (a 16-byte
// load conflict).
std::vector<int> conflict_free_order(const std::vector<int> &nodes, int arity, int width, int window = 1024);

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
