// Host-side template builder (Sec. 5, template creation; Sec. 4 relaxed
// state).  From a triangle list it derives, by sorting directed edges:
//   - the undirected edges (i < j) in lexicographic order,
//   - for every edge (b,c) its bending pair (a,b,c,d): a is the third node
//     of the triangle that runs b->c, d that of the triangle that runs c->b,
//   - the relaxed lengths L0, inner angles theta0, triangle areas S0, total
//     area S_g0 and volume V0 of the (stretched) template geometry, in FP64.
// It rejects meshes that are not closed, consistently ordered 2-manifolds,
// meshes with unused nodes or degenerate triangles, and meshes whose
// triangles point outward (the library requires AB x AC to point inside).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "topology.h"

namespace lbib {

namespace {

struct V3 {
    double x, y, z;
};
V3 at(const std::vector<double> &x, int i) { return {x[3 * i], x[3 * i + 1], x[3 * i + 2]}; }
V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
double dotp(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 crossp(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double len(V3 a) { return std::sqrt(dotp(a, a)); }
V3 unit(V3 a) {
    const double l = len(a);
    return {a.x / l, a.y / l, a.z / l};
}

// Inner angle at edge (b,c) between the inward-ordered triangles (a,b,c)
// and (d,c,b): pi minus the angle between their inward normals when d lies
// on the inner side of the first triangle's plane, pi plus it otherwise.
double inner_angle(V3 a, V3 b, V3 c, V3 d) {
    const V3 n1 = unit(crossp(sub(b, a), sub(c, a)));
    const V3 n2 = unit(crossp(sub(c, d), sub(b, d)));
    const double alpha = std::atan2(len(crossp(n1, n2)), dotp(n1, n2));
    const double pi = 3.14159265358979323846;
    return dotp(sub(d, b), n1) > 0.0 ? pi - alpha : pi + alpha;
}

}  // namespace

bool build_template(const double *xyz, int nn, const int32_t *tris, int nt, const double stretch[3],
                    Topology &T, std::string &err) {
    if (nn < 4 || nt < 4) {
        err = "a closed mesh needs at least 4 nodes and 4 triangles";
        return false;
    }
    T.nn = nn;
    T.nt = nt;
    T.x.resize(3 * (size_t)nn);
    for (int i = 0; i < nn; ++i)
        for (int k = 0; k < 3; ++k) T.x[3 * i + k] = xyz[3 * i + k] * (stretch ? stretch[k] : 1.0);
    T.tri.assign(tris, tris + 3 * (size_t)nt);
    std::vector<int> used(nn, 0);
    for (size_t i = 0; i < T.tri.size(); ++i) {
        if (T.tri[i] < 0 || T.tri[i] >= nn) {
            err = "triangle refers to a node id outside [0, n_nodes)";
            return false;
        }
        used[T.tri[i]] = 1;
    }
    for (int t = 0; t < nt; ++t) {
        const int a = T.tri[3 * t], b = T.tri[3 * t + 1], c = T.tri[3 * t + 2];
        if (a == b || b == c || a == c) {
            err = "triangle " + std::to_string(t) + " repeats a node";
            return false;
        }
    }
    for (int i = 0; i < nn; ++i)
        if (!used[i]) {
            err = "node " + std::to_string(i) + " belongs to no triangle";
            return false;
        }

    // directed edges (from, to) -> apex, sorted by key
    struct DE {
        uint64_t key;
        int apex;
    };
    std::vector<DE> de;
    de.reserve(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            const uint32_t i = (uint32_t)T.tri[3 * t + k], j = (uint32_t)T.tri[3 * t + (k + 1) % 3];
            de.push_back({((uint64_t)i << 32) | j, T.tri[3 * t + (k + 2) % 3]});
        }
    std::sort(de.begin(), de.end(), [](const DE &p, const DE &q) { return p.key < q.key; });
    for (size_t k = 1; k < de.size(); ++k)
        if (de[k].key == de[k - 1].key) {
            err = "directed edge used twice: the mesh is non-manifold or inconsistently ordered";
            return false;
        }
    auto find = [&](uint64_t key) -> int {
        auto it = std::lower_bound(de.begin(), de.end(), key, [](const DE &p, uint64_t k) { return p.key < k; });
        return (it != de.end() && it->key == key) ? it->apex : -1;
    };
    T.edges.clear();
    T.quads.clear();
    for (const DE &e : de) {
        const int b = (int)(e.key >> 32), c = (int)(e.key & 0xffffffffu);
        const int d = find(((uint64_t)(uint32_t)c << 32) | (uint32_t)b);
        if (d < 0) {
            err = "edge " + std::to_string(b) + "-" + std::to_string(c) + " has no opposite triangle (open mesh)";
            return false;
        }
        if (b < c) {
            T.edges.push_back(b);
            T.edges.push_back(c);
            T.quads.push_back(e.apex);
            T.quads.push_back(b);
            T.quads.push_back(c);
            T.quads.push_back(d);
        }
    }
    T.ne = (int)(T.edges.size() / 2);
    if (2 * (size_t)T.ne != de.size()) {
        err = "edge count inconsistent with a closed mesh";
        return false;
    }

    // relaxed state
    T.L0.resize(T.ne);
    T.theta0.resize(T.ne);
    for (int e = 0; e < T.ne; ++e) {
        const int *q = &T.quads[4 * e];
        T.L0[e] = len(sub(at(T.x, T.edges[2 * e + 1]), at(T.x, T.edges[2 * e])));
        T.theta0[e] = inner_angle(at(T.x, q[0]), at(T.x, q[1]), at(T.x, q[2]), at(T.x, q[3]));
        if (!(T.L0[e] > 0.0)) {
            err = "zero-length edge";
            return false;
        }
    }
    T.S0.resize(nt);
    double sg = 0.0, v6 = 0.0;
    const V3 o = at(T.x, 0);
    for (int t = 0; t < nt; ++t) {
        const V3 a = sub(at(T.x, T.tri[3 * t]), o), b = sub(at(T.x, T.tri[3 * t + 1]), o),
                 c = sub(at(T.x, T.tri[3 * t + 2]), o);
        const double s = 0.5 * len(crossp(sub(b, a), sub(c, a)));
        if (!(s > 0.0)) {
            err = "degenerate triangle " + std::to_string(t);
            return false;
        }
        T.S0[t] = s;
        sg += s;
        v6 += dotp(a, crossp(b, c));
    }
    T.Sg0 = sg;
    T.V0 = -v6 / 6.0;
    if (!(T.V0 > 0.0)) {
        err = "triangles are ordered outward (AB x AC must point inside the object)";
        return false;
    }

    T.quad_order = conflict_free_order(T.quads, 4, 32);
    T.tri_order = conflict_free_order(T.tri, 3, 32);
    return true;
}

bool orient_mesh(const double *xyz, int nn, const int32_t *tris, int nt, int mode, int32_t *out, int &changed,
                 std::string &err) {
    changed = 0;
    std::vector<int> t(tris, tris + 3 * (size_t)nt);
    for (int v : t)
        if (v < 0 || v >= nn) {
            err = "triangle refers to a node id outside [0, n_nodes)";
            return false;
        }
    std::vector<char> flip(nt, 0);
    if (mode == 2) {
        std::fill(flip.begin(), flip.end(), 1);
    } else {
        // undirected edge -> the (at most two) triangles using it
        struct E {
            uint64_t key;
            int tri;
        };
        std::vector<E> es;
        es.reserve(3 * (size_t)nt);
        for (int i = 0; i < nt; ++i)
            for (int k = 0; k < 3; ++k) {
                uint32_t a = (uint32_t)t[3 * i + k], b = (uint32_t)t[3 * i + (k + 1) % 3];
                if (a > b) std::swap(a, b);
                es.push_back({((uint64_t)a << 32) | b, i});
            }
        std::sort(es.begin(), es.end(), [](const E &p, const E &q) { return p.key < q.key || (p.key == q.key && p.tri < q.tri); });
        std::vector<std::vector<int>> nb(nt);
        for (size_t k = 0; k < es.size();) {
            size_t j = k;
            while (j < es.size() && es[j].key == es[k].key) ++j;
            if (j - k != 2) {
                err = "an edge is not shared by exactly two triangles: the mesh is not a closed 2-manifold";
                return false;
            }
            nb[es[k].tri].push_back(es[k + 1].tri);
            nb[es[k + 1].tri].push_back(es[k].tri);
            k = j;
        }
        // does triangle i (with its flip) traverse edge (a, b) in that order?
        auto runs = [&](int i, int a, int b) {
            for (int k = 0; k < 3; ++k) {
                int p = t[3 * i + k], q = t[3 * i + (k + 1) % 3];
                if (flip[i]) std::swap(p, q);
                if (p == a && q == b) return true;
            }
            return false;
        };
        std::vector<char> seen(nt, 0);
        for (int root = 0; root < nt; ++root) {
            if (seen[root]) continue;
            std::vector<int> comp{root}, queue{root};
            seen[root] = 1;
            for (size_t h = 0; h < queue.size(); ++h) {
                const int i = queue[h];
                for (int j : nb[i]) {
                    // the shared edge must run in opposite directions
                    int a = -1, b = -1;
                    for (int k = 0; k < 3 && a < 0; ++k) {
                        int p = t[3 * i + k], q = t[3 * i + (k + 1) % 3];
                        if (flip[i]) std::swap(p, q);
                        for (int m = 0; m < 3; ++m)
                            if ((t[3 * j + m] == p || t[3 * j + m] == q) &&
                                (t[3 * j + (m + 1) % 3] == p || t[3 * j + (m + 1) % 3] == q)) {
                                a = p;
                                b = q;
                            }
                    }
                    if (!seen[j]) {
                        seen[j] = 1;
                        if (runs(j, a, b)) flip[j] ^= 1;
                        comp.push_back(j);
                        queue.push_back(j);
                    } else if (runs(j, a, b)) {
                        err = "the mesh is not orientable";
                        return false;
                    }
                }
            }
            // inward: -(1/6) sum A.(B x C) > 0 with the first node of the component as origin
            double v6 = 0.0;
            const int o = t[3 * comp[0]];
            for (int i : comp) {
                int a = t[3 * i], b = t[3 * i + 1], c = t[3 * i + 2];
                if (flip[i]) std::swap(b, c);
                double A[3], B[3], Cc[3];
                for (int k = 0; k < 3; ++k) {
                    A[k] = xyz[3 * a + k] - xyz[3 * o + k];
                    B[k] = xyz[3 * b + k] - xyz[3 * o + k];
                    Cc[k] = xyz[3 * c + k] - xyz[3 * o + k];
                }
                v6 += A[0] * (B[1] * Cc[2] - B[2] * Cc[1]) + A[1] * (B[2] * Cc[0] - B[0] * Cc[2]) +
                      A[2] * (B[0] * Cc[1] - B[1] * Cc[0]);
            }
            if (v6 > 0.0)
                for (int i : comp) flip[i] ^= 1;
        }
    }
    for (int i = 0; i < nt; ++i) {
        changed += flip[i];
        if (out) {
            out[3 * i] = t[3 * i];
            out[3 * i + 1] = flip[i] ? t[3 * i + 2] : t[3 * i + 1];
            out[3 * i + 2] = flip[i] ? t[3 * i + 1] : t[3 * i + 2];
        }
    }
    return true;
}

std::vector<int> conflict_free_order(const std::vector<int> &nodes, int arity, int width, int window) {
    const int n = (int)(nodes.size() / arity);
    int max_node = 0;
    for (int v : nodes) max_node = std::max(max_node, v);
    std::vector<int> stamp(max_node + 1, -1), order, remaining(n);
    for (int i = 0; i < n; ++i) remaining[i] = i;
    order.reserve(n);
    std::vector<int> res32(32 * arity), res8(8 * arity);
    constexpr int NODE_TAKEN = 1 << 20;
    for (int group = 0; !remaining.empty(); ++group) {
        std::fill(res32.begin(), res32.end(), 0);
        for (int lane = 0; lane < width && !remaining.empty(); ++lane) {
            if (lane % 8 == 0) std::fill(res8.begin(), res8.end(), 0);
            const int scan = std::min((int)remaining.size(), window);
            int best = 0, best_cost = -1;
            for (int j = 0; j < scan; ++j) {
                const int *e = &nodes[(size_t)arity * remaining[j]];
                int c = 0;
                for (int k = 0; k < arity; ++k) {
                    if (stamp[e[k]] == group) c += NODE_TAKEN;
                    c += 3 * res32[32 * k + (e[k] & 31)] + 2 * res8[8 * k + (e[k] & 7)];
                }
                if (best_cost < 0 || c < best_cost) {
                    best_cost = c;
                    best = j;
                    if (c == 0) break;
                }
            }
            const int eb = remaining[best];
            remaining.erase(remaining.begin() + best);
            const int *e = &nodes[(size_t)arity * eb];
            for (int k = 0; k < arity; ++k) {
                stamp[e[k]] = group;
                ++res32[32 * k + (e[k] & 31)];
                ++res8[8 * k + (e[k] & 7)];
            }
            order.push_back(eb);
        }
    }
    return order;
}

}  // namespace lbib
