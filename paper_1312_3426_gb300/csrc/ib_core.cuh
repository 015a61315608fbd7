// Device-side bodies of the immersed-boundary update (Sec. 2 and Sec. 4 of
// arXiv:1312.3426), shared by the single-simulation kernels (ib.cu) and the
// batched persistent kernel (batch.cu).  The update has two parts.
//
// Membrane part, one thread-block cluster of C blocks per object; it needs
// only the node positions, so it can run while the fluid step that precedes
// it is still in progress:
//   1. every block stages the positions of all the object's nodes, relative
//      to its first node, as hi + lo FP32 pairs in shared memory, and clears
//      its own force array;
//   2. every block sums the area and divergence-theorem volume terms of its
//      share of the triangles (error-free FP32 pair sums); after a cluster
//      barrier one thread per block reads the C partial sums through
//      distributed shared memory in a fixed order and forms the object's
//      total area S_g and volume V in FP64 (Sec. 4, global area and volume
//      conservation);
//   3. every block evaluates its share of the elements and adds each
//      contribution to its own shared-memory force array:
//        edge       stretching (Eq. stretching) ks kappa(lambda) (L-L0)/L0
//                   along the edge, +f on one node, -f on the other;
//        edge pair  bending: theta is the inner angle between the triangles
//                   (a,b,c) and (d,c,b), s = kb (theta-theta0)/theta0, the
//                   apices take s n1 and s n2 (inward unit normals), the edge
//                   nodes minus half of their sum;
//        triangle   local area -kal (S-S0)/S w_v and global area
//                   -kag (S_g-S_g0)/S_g w_v, w_v the unit vector from the
//                   centroid to vertex v, and volume kv (V-V0)/V0 S n_in / 3;
//      a pair of opposite contributions is the same FP32 value with both
//      signs, so internal forces cancel up to the rounding of the sums;
//   4. after a cluster barrier every block sums, for its share of the
//      nodes, the C partial force arrays through distributed shared memory in
//      a fixed order and writes the membrane force of each node.
// Coupling part, one thread per node: interpolates the fluid velocity
//   trilinearly from the 8 surrounding lattice nodes (u = 0 on solid rows),
//   applies the drag F_d = xi (u - v), spreads -F_d with the same weights
//   (one 16-byte vector atomic per corner) and advances
//   v += (F + F_d + F_ext)/m, X += v (Eq. newton, unit time step); when the
//   node's lower lattice corner changes, the 4x4x4 cells around the new
//   position are marked active (see lbib_internal.h).
// Node state is kept as hi + lo FP32 pairs (error-free two-sum arithmetic);
// FP64 is used only for the per-object area and volume totals.
#pragma once

#include <cooperative_groups.h>

#include "lattice_index.h"
#include "lbib_internal.h"

namespace lbib {

struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ f3 xyz(float4 v) { return {v.x, v.y, v.z}; }
__device__ __forceinline__ float4 f4(f3 v, float w) { return make_float4(v.x, v.y, v.z, w); }

// Error-free FP32 transformations (Knuth's two-sum and its fast variant):
// a pair (hi, lo) holds the unevaluated sum hi + lo.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add_f(df a, float b) {
    df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    const df t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, s.lo + t.hi);
    return fast_two_sum(s.hi, s.lo + t.lo);
}

// Staged positions of one object: node q relative to the object's first
// node is hi[q].xyz + lo[q].xyz (float4 for 16-byte shared-memory loads).
struct Stage {
    const float4 *hi, *lo;
    // position of node q relative to node p; the difference of the hi parts
    // is exact for the nearby nodes of one element
    __device__ __forceinline__ f3 rel(int q, int p) const {
        const float4 a = hi[q], b = hi[p], c = lo[q], d = lo[p];
        return {(a.x - b.x) + (c.x - d.x), (a.y - b.y) + (c.y - d.y), (a.z - b.z) + (c.z - d.z)};
    }
    __device__ __forceinline__ f3 pos(int q) const {
        const float4 a = hi[q], c = lo[q];
        return {a.x + c.x, a.y + c.y, a.z + c.z};
    }
};

struct Corners {
    int f[8];
    float w[8];
};

// The 8 interpolation corners of a node (lattice_index.h); a corner on an
// obstacle cell counts as solid.
__device__ __forceinline__ void corners(const SimDev &s, df x, df y, df z, Corners &c) {
    corner_cells(s, x.hi, x.lo, y.hi, y.lo, z.hi, z.lo, c.f, c.w);
    if (s.solid) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (c.f[k] >= 0 && solid_bit(s, c.f[k])) c.f[k] = -1;
    }
}

namespace cg = cooperative_groups;

__device__ __forceinline__ void mark(uint32_t *mask, int f) { atomicOr(mask + (f >> 5), 1u << (f & 31)); }

// Marks the 4x4x4 lattice nodes (i0-1 .. i0+2, ...) around lower corner
// (ix, iy, iz) as active.
__device__ __forceinline__ void mark_halo(const SimDev &s, int ix, int iy, int iz) {
    for_each_halo(s, ix, iy, iz, [&](int f) { mark(s.amask, f); });
}

// mark_halo for the lanes of the calling converged threads that pass
// `need`: the threads take each such lane's 64 halo nodes together (one
// or a few nodes per thread), instead of one lane walking 64 nodes while
// the others of its warp wait.
__device__ __forceinline__ void mark_halo_coalesced(const SimDev &s, bool need, int3 lc) {
    cg::coalesced_group g = cg::coalesced_threads();
    unsigned m = g.ballot(need);
    const int n = (int)g.size(), r = (int)g.thread_rank();
    while (m) {
        const int src = __ffs(m) - 1;  // rank in g
        m &= m - 1;
        const int ix = g.shfl(lc.x, src), iy = g.shfl(lc.y, src), iz = g.shfl(lc.z, src);
        for (int j = r; j < 64; j += n) {
            const int f = halo_cell(s, ix, iy, iz, j);
            if (f >= 0) mark(s.amask, f);
        }
    }
}

// G[f] += (x, y, z, 0) as one vector reduction: no value comes back, so
// nothing waits for it.
__device__ __forceinline__ void red_add_v4(float4 *p, float x, float y, float z) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(0.f)
                 : "memory");
}

// Lower lattice corner of a position.
__device__ __forceinline__ int3 lower_corner(df x, df y, df z) {
    int3 c;
    float w;
    lattice_coord(x.hi, x.lo, c.x, w);
    lattice_coord(y.hi, y.lo, c.y, w);
    lattice_coord(z.hi, z.lo, c.z, w);
    return c;
}

// Shared memory per object team: per node of the largest template the
// staged position (two float4) and the force (3 floats), plus a fixed tail
// (area / volume partials and factors, the per-warp partial sums of the
// reductions).  A multiple of 16 bytes, so teams can sit side by side.
constexpr int IB_SMEM_PER_NODE = 11 * sizeof(float);
constexpr int IB_SMEM_TAIL = 512;
constexpr int IB_TAIL_WPART = 16;                         // float offset: df [2][IB_THREADS / 32]
constexpr int IB_TAIL_BOX = IB_TAIL_WPART + 4 * IB_THREADS / 32;  // float [6][IB_THREADS / 32]
static_assert((IB_TAIL_BOX + 6 * IB_THREADS / 32) * 4 <= IB_SMEM_TAIL, "tail layout");

// The threads that update one object's membrane together: every block of a
// thread-block cluster (ClusterTeam), or a group of whole warps inside one
// block (GroupTeam, several objects per block, a named barrier each).
struct ClusterTeam {
    cg::cluster_group cl;
    __device__ __forceinline__ ClusterTeam() : cl(cg::this_cluster()) {}
    __device__ __forceinline__ int tid() const { return (int)threadIdx.x; }
    __device__ __forceinline__ int size() const { return (int)blockDim.x; }
    __device__ __forceinline__ int rank() const { return (int)cl.block_rank(); }
    __device__ __forceinline__ int ranks() const { return (int)cl.num_blocks(); }
    __device__ __forceinline__ void sync_block() const { __syncthreads(); }
    __device__ __forceinline__ void sync_all() const { cl.sync(); }
    __device__ __forceinline__ float *peer(float *p, int j) const { return cl.map_shared_rank(p, j); }
};
struct GroupTeam {
    int t, n, bar;  // thread index in the group, group size (a multiple of 32), named barrier (1..15)
    __device__ __forceinline__ int tid() const { return t; }
    __device__ __forceinline__ int size() const { return n; }
    __device__ __forceinline__ int rank() const { return 0; }
    __device__ __forceinline__ int ranks() const { return 1; }
    __device__ __forceinline__ void sync_block() const {
        asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(n) : "memory");
    }
    __device__ __forceinline__ void sync_all() const { sync_block(); }
    __device__ __forceinline__ float *peer(float *p, int) const { return p; }
};

__host__ __device__ inline size_t ib_smem_bytes(int max_nodes) {
    return ((size_t)IB_SMEM_PER_NODE * max_nodes + IB_SMEM_TAIL + 15) & ~(size_t)15;
}

// Sum over a warp of FP32 values as an unevaluated hi + lo pair.
__device__ __forceinline__ df warp_sum_df(df a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const df b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = df_add(a, b);
    }
    return a;
}

struct Forces {
    float *x, *y, *z;
    __device__ __forceinline__ void add(int p, f3 v) const {
        atomicAdd(x + p, v.x);
        atomicAdd(y + p, v.y);
        atomicAdd(z + p, v.z);
    }
};

// The two forces that live on edge e = (b, c) of the hinge (a, b, c, d)
// (triangles (a, b, c) and (d, c, b)): the stretching of the edge and the
// bending between the two triangles.  One pass over the edges serves both:
// they share the record, the staged positions of b and c and the vector
// c - b, and their forces on b and c are summed before the shared-memory
// reductions (the order of FP32 additions into a node is not fixed anyway).
template <bool AV>
__device__ __forceinline__ void hinge_force(const TplDev &T, const Stage &P, int e, const Forces &F, df &area,
                                            df &vol) {
    const int4 q = __ldg(T.quad + e);
    const float4 h = __ldg(T.hinge + e);  // (L0, 1/L0, 1/theta0, 0)
    const f3 C = P.rel(q.z, q.y);         // c - b
    f3 fb = mk(0.f, 0.f, 0.f), fc = fb;
    if (T.ks != 0.f) {  // stretching along c - b
        const float il = rsqrtf(dot(C, C));
        const float L = dot(C, C) * il;
        const float lam = L * h.y;
        float kap = 1.f;
        if (T.nonlinear) {  // (lambda^0.5 + lambda^-2.5) / (lambda + lambda^-3)
            // lambda stays near 1: the fast reciprocal and quotient are within 2 ulp
            const float sl = sqrtf(lam), il3 = __fdividef(1.f, lam * lam * lam);
            kap = __fdividef(sl + il3 * sl, lam + il3);
        }
        fb = (T.ks * kap * (L - h.x) * h.y * il) * C;
        fc = -1.f * fb;
    }
    if (T.kb != 0.f) {  // bending: the angle between the two triangles' normals
        const f3 A = P.rel(q.x, q.y), D = P.rel(q.w, q.y);  // relative to b
        f3 n1 = cross(-1.f * A, C - A);  // (b-a) x (c-a)
        f3 n2 = cross(C - D, -1.f * D);  // (c-d) x (b-d)
        if constexpr (AV) {  // each triangle is in three hinges: a third of its area and volume term each
            area = df_add_f(area, 0.5f * (sqrtf(dot(n1, n1)) + sqrtf(dot(n2, n2))));
            vol = df_add_f(vol, dot(P.pos(q.x), n1) + dot(P.pos(q.w), n2));
        }
        n1 = rsqrtf(dot(n1, n1)) * n1;
        n2 = rsqrtf(dot(n2, n2)) * n2;
        const f3 cr = cross(n1, n2);
        const float alpha = atan2f(sqrtf(dot(cr, cr)), dot(n1, n2));
        const float PI_F = 3.14159265358979f;
        const float theta = dot(D, n1) > 0.f ? PI_F - alpha : PI_F + alpha;
        const float sb = T.kb * (theta * h.z - 1.f);
        const f3 fa = sb * n1, fd = sb * n2;
        const f3 fe = -0.5f * (fa + fd);
        F.add(q.x, fa);
        F.add(q.w, fd);
        fb = fb + fe;
        fc = fc + fe;
    }
    F.add(q.y, fb);
    F.add(q.z, fc);
}

__device__ __forceinline__ void triangle_force(const TplDev &T, const Stage &P, int t, float dSg, float dV,
                                               const Forces &F) {
    const int4 tr = __ldg(T.tri + t);  // (a, b, c, S0 bits), inward
    const float S0 = __int_as_float(tr.w);
    const f3 B = P.rel(tr.y, tr.x), C = P.rel(tr.z, tr.x);  // relative to a
    const f3 N = cross(B, C);
    const float inl = rsqrtf(dot(N, N));
    const float S = 0.5f * dot(N, N) * inl;
    const f3 G = (1.f / 3.f) * (B + C);  // centroid relative to a
    const f3 fv = (T.kv * dV * S * inl * (1.f / 3.f)) * N;  // volume, a third per vertex
    const f3 wa = -1.f * G, wb = B - G, wc = C - G;
    const float iS = 2.f * inl;  // 1/S
    if (!T.kal_altitude) {
        const float cw = -T.kal * (S - S0) * iS - T.kag * dSg;  // local + global area
        F.add(tr.x, (cw * rsqrtf(dot(wa, wa))) * wa + fv);
        F.add(tr.y, (cw * rsqrtf(dot(wb, wb))) * wb + fv);
        F.add(tr.z, (cw * rsqrtf(dot(wc, wc))) * wc + fv);
        return;
    }
    // local area along each vertex's altitude (from the foot on the opposite
    // edge to the vertex), global area along centroid -> vertex
    const float cl = -T.kal * (S - S0) * iS, cg = -T.kag * dSg;
    const f3 Z = mk(0.f, 0.f, 0.f);
    auto alt = [](f3 p, f3 q, f3 r) {  // component of p - q orthogonal to r - q
        const f3 e = r - q, d = p - q;
        return d - (dot(d, e) / dot(e, e)) * e;
    };
    const f3 ha = alt(Z, B, C), hb = alt(B, C, Z), hc = alt(C, Z, B);
    F.add(tr.x, (cl * rsqrtf(dot(ha, ha))) * ha + (cg * rsqrtf(dot(wa, wa))) * wa + fv);
    F.add(tr.y, (cl * rsqrtf(dot(hb, hb))) * hb + (cg * rsqrtf(dot(wb, wb))) * wb + fv);
    F.add(tr.z, (cl * rsqrtf(dot(hc, hc))) * hc + (cg * rsqrtf(dot(wc, wc))) * wc + fv);
}

// Coupling and Newton update of node i (global index) of object o.  EARLY
// (the kernel may be launched early, by programmatic dependent launch):
// before dep_wait() it reads only the node state and the object tables
// (written by no kernel that can still be running when a node kernel starts
// early); the membrane force, the external force, the velocity field, the
// coupling buffer and the mask come after it.  Otherwise the membrane force
// is read first.
template <bool EARLY>
__device__ __forceinline__ void node_update(const SimDev &s, int o, int i, float inv_mass, int par) {
    const int NN = s.nn_total;
    f3 F;
    if constexpr (!EARLY) F = mk(s.Fel[i], s.Fel[NN + i], s.Fel[2 * NN + i]);
    float *Xh = s.Xh, *Xl = s.Xl, *Vh = s.Vh, *Vl = s.Vl;
    df x{Xh[i], Xl[i]}, y{Xh[NN + i], Xl[NN + i]}, z{Xh[2 * NN + i], Xl[2 * NN + i]};
    if (!isfinite(x.hi) || !isfinite(y.hi) || !isfinite(z.hi)) {
        // a failed simulation (already flagged): no coupling, so that its
        // nodes do not pile reductions onto one cell
        atomicOr(s.status, ST_NODE_NAN);
        return;
    }
    df vx{Vh[i], Vl[i]}, vy{Vh[NN + i], Vl[NN + i]}, vz{Vh[2 * NN + i], Vl[2 * NN + i]};
    Corners c;
    corners(s, x, y, z, c);
    const int3 c0 = lower_corner(x, y, z);
    if constexpr (EARLY) {
        dep_wait();
        dep_release();
        F = mk(s.Fel[i], s.Fel[NN + i], s.Fel[2 * NN + i]);
    }
    float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (c.f[k] >= 0) {
            const float4 u = s.ufield[c.f[k]];
            ux += c.w[k] * u.x;
            uy += c.w[k] * u.y;
            uz += c.w[k] * u.z;
        }
    }
    const float xi = s.xi;
    const float fdx = xi * ((ux - vx.hi) - vx.lo);
    const float fdy = xi * ((uy - vy.hi) - vy.lo);
    const float fdz = xi * ((uz - vz.hi) - vz.lo);
    float dropx = 0.f, dropy = 0.f, dropz = 0.f;
    float4 *G = s.G[par];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float w = c.w[k];
        if (c.f[k] >= 0) {
            red_add_v4(G + c.f[k], -w * fdx, -w * fdy, -w * fdz);
        } else {
            dropx -= w * fdx;
            dropy -= w * fdy;
            dropz -= w * fdz;
        }
    }
    if (dropx != 0.f || dropy != 0.f || dropz != 0.f) {
        atomicAdd(s.dropped, (double)dropx);
        atomicAdd(s.dropped + 1, (double)dropy);
        atomicAdd(s.dropped + 2, (double)dropz);
    }
    const float *fe = s.fext + 3 * o;
    vx = df_add_f(vx, (F.x + fdx + fe[0]) * inv_mass);
    vy = df_add_f(vy, (F.y + fdy + fe[1]) * inv_mass);
    vz = df_add_f(vz, (F.z + fdz + fe[2]) * inv_mass);
    x = df_add(x, vx);
    y = df_add(y, vy);
    z = df_add(z, vz);
    Vh[i] = vx.hi;
    Vl[i] = vx.lo;
    Vh[NN + i] = vy.hi;
    Vl[NN + i] = vy.lo;
    Vh[2 * NN + i] = vz.hi;
    Vl[2 * NN + i] = vz.lo;
    Xh[i] = x.hi;
    Xl[i] = x.lo;
    Xh[NN + i] = y.hi;
    Xl[NN + i] = y.lo;
    Xh[2 * NN + i] = z.hi;
    Xl[2 * NN + i] = z.lo;
    const bool fin = isfinite(x.hi) && isfinite(y.hi) && isfinite(z.hi);
    if (!fin) atomicOr(s.status, ST_NODE_NAN);
    const int3 lc = lower_corner(x, y, z);
    mark_halo_coalesced(s, fin && (lc.x != c0.x || lc.y != c0.y || lc.z != c0.z), lc);
}

// Share [r n / C, (r+1) n / C) of n items for cluster rank r.
__device__ __forceinline__ int share_lo(int n, int r, int C) { return (int)(((long long)n * r) / C); }

// The same split on multiples of 32, so that a warp's 32 consecutive
// elements are one group of the template's conflict-free order.
__device__ __forceinline__ int share_lo32(int n, int r, int C) {
    return r >= C ? n : (int)((((long long)n * r) / C) & ~31LL);
}

// Soft-sphere force magnitude a n r^-(n+1) (the repulsion reading; see
// lbib.h lbib_set_repulsion).
__device__ __forceinline__ float soft_force(float a, float n, float r) { return a * n * powf(r, -(n + 1.0f)); }

// Wall term of the repulsion for a node at height y (hi + lo): pushed away
// from the planes y = 1 and y = ny - 1 when closer than the cutoff.
__device__ __forceinline__ float wall_force(const SimDev &s, float yh, float yl) {
    const float dlo = (yh - 1.0f) + yl;
    const float dhi = ((float)(s.ny - 1) - yh) - yl;
    float f = 0.f;
    if (dlo < s.rep_wrc) f += soft_force(s.rep_wa, s.rep_wn, fmaxf(dlo, 1e-3f));
    if (dhi < s.rep_wrc) f -= soft_force(s.rep_wa, s.rep_wn, fmaxf(dhi, 1e-3f));
    return f;
}

// Bounding box of object o from its staged relative positions plus the
// first node's position (FP32: a broad-phase filter, widened by the
// cutoff where it is used).  Every thread of the team calls it.
template <class Team>
__device__ __forceinline__ void object_box(const SimDev &s, int o, const Stage &P, int nn, int f0, float *tail,
                                           const Team &tm) {
    float mn[3] = {3.0e38f, 3.0e38f, 3.0e38f}, mx[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    for (int p = tm.tid(); p < nn; p += tm.size()) {
        const float4 h = P.hi[p];
        mn[0] = fminf(mn[0], h.x), mn[1] = fminf(mn[1], h.y), mn[2] = fminf(mn[2], h.z);
        mx[0] = fmaxf(mx[0], h.x), mx[1] = fmaxf(mx[1], h.y), mx[2] = fmaxf(mx[2], h.z);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], off));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], off));
        }
    float *box_part = tail + IB_TAIL_BOX;  // [6][IB_THREADS / 32]
    constexpr int W = IB_THREADS / 32;
    if ((tm.tid() & 31) == 0)
        for (int k = 0; k < 3; ++k) {
            box_part[k * W + (tm.tid() >> 5)] = mn[k];
            box_part[(3 + k) * W + (tm.tid() >> 5)] = mx[k];
        }
    tm.sync_block();
    if (tm.tid() < 6) {
        const int k = tm.tid();
        float v = box_part[k * W];
        for (int w = 1; w < (tm.size() >> 5); ++w)
            v = k < 3 ? fminf(v, box_part[k * W + w]) : fmaxf(v, box_part[k * W + w]);
        const int c = k % 3;
        s.aabb[8 * o + k] = v + s.Xh[c * s.nn_total + f0];
    }
}

// The membrane part of object o by the calling team (every thread of all
// its C blocks calls it; sh: the team's shared memory in each block):
// writes the membrane force of each of its nodes to s.Fel (plus the wall
// repulsion, when set).
template <class Team>
__device__ __forceinline__ void membrane_object(const SimDev &s, int o, float *sh, const Team &tm) {
    const int C = tm.ranks(), r = tm.rank(), tid = tm.tid(), nthr = tm.size();
    const ObjDev ob = s.obj[o];
    const TplDev &T = s.tpl[ob.tid];
    const int nn = ob.nn, f0 = ob.first, NN = s.nn_total;

    float4 *hi = (float4 *)sh, *lo = hi + nn;
    float *Fx = sh + 8 * nn, *Fy = sh + 9 * nn, *Fz = sh + 10 * nn;
    float *tail = sh + 11 * nn;  // [0..3] this block's area / volume partials, [4..5] factors
    const Stage P{hi, lo};
    const Forces F{Fx, Fy, Fz};

    // 1. stage positions relative to the first node, clear the forces
    for (int p = tid; p < nn; p += nthr) {
        df d[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const df a{s.Xh[k * NN + f0 + p], s.Xl[k * NN + f0 + p]};
            const df b{s.Xh[k * NN + f0], s.Xl[k * NN + f0]};
            d[k] = df_add(a, {-b.hi, -b.lo});
        }
        hi[p] = make_float4(d[0].hi, d[1].hi, d[2].hi, 0.f);
        lo[p] = make_float4(d[0].lo, d[1].lo, d[2].lo, 0.f);
        Fx[p] = 0.f;
        Fy[p] = 0.f;
        Fz[p] = 0.f;
    }
    tm.sync_block();

    // 1b. bounding box of the object's nodes (broad phase of the repulsion)
    if (s.rep_on && r == 0) object_box(s, o, P, nn, f0, tail, tm);

    // 2. this block's share of the area and volume sums: with bending on,
    //    from the hinge pass (each triangle three times), else by triangle
    df area{0.f, 0.f}, vol{0.f, 0.f};
    const bool need_av = T.kag != 0.f || T.kv != 0.f;
    const bool av_in_hinges = need_av && T.kb != 0.f;
    if (T.ks != 0.f || T.kb != 0.f) {
        const int e1 = share_lo32(T.ne, r + 1, C);
        if (av_in_hinges) {
#pragma unroll 2
            for (int e = share_lo32(T.ne, r, C) + tid; e < e1; e += nthr) hinge_force<true>(T, P, e, F, area, vol);
        } else {
#pragma unroll 2
            for (int e = share_lo32(T.ne, r, C) + tid; e < e1; e += nthr) hinge_force<false>(T, P, e, F, area, vol);
        }
    }
    if (need_av && !av_in_hinges) {
        for (int t = share_lo(T.nt, r, C) + tid; t < share_lo(T.nt, r + 1, C); t += nthr) {
            const int4 tr = __ldg(T.tri + t);
            const f3 N = cross(P.rel(tr.y, tr.x), P.rel(tr.z, tr.x));
            area = df_add_f(area, 0.5f * sqrtf(dot(N, N)));
            vol = df_add_f(vol, dot(P.pos(tr.x), N));
        }
    }
    df *wpart = (df *)(tail + IB_TAIL_WPART);  // [2][IB_THREADS / 32]
    constexpr int W = IB_THREADS / 32;
    area = warp_sum_df(area);
    vol = warp_sum_df(vol);
    if ((tid & 31) == 0) {
        wpart[tid >> 5] = area;
        wpart[W + (tid >> 5)] = vol;
    }
    tm.sync_block();
    if (tid < 2) {
        df t = wpart[tid * W];
        for (int w = 1; w < (nthr >> 5); ++w) t = df_add(t, wpart[tid * W + w]);
        tail[2 * tid] = t.hi;
        tail[2 * tid + 1] = t.lo;
    }
    tm.sync_all();  // staging, cleared forces and partial sums visible to the team

    // totals of the object in FP64, partials taken in rank order
    if (tid == 0) {
        double Sg = 0.0, V6 = 0.0;
        for (int j = 0; j < C; ++j) {
            const float *pj = tm.peer(tail, j);
            Sg += (double)pj[0] + (double)pj[1];
            V6 += (double)pj[2] + (double)pj[3];
        }
        if (av_in_hinges) {  // every triangle was summed three times
            Sg *= 1.0 / 3.0;
            V6 *= 1.0 / 3.0;
        }
        // differences to the relaxed state in FP64, ratios in FP32
        const float dS = (float)(Sg - T.Sg0), dVol = (float)(V6 * (-1.0 / 6.0) - T.V0);
        tail[4] = (T.kag != 0.f) ? dS / (float)Sg : 0.f;
        tail[5] = (T.kv != 0.f) ? dVol / (float)T.V0 : 0.f;
    }
    tm.sync_block();
    const float dSg = tail[4], dV = tail[5];

    // 3. this block's share of each kind of element; one loop per kind so
    //    that independent iterations overlap
    if (T.kal != 0.f || T.kag != 0.f || T.kv != 0.f) {
        const int t1 = share_lo32(T.nt, r + 1, C);
#pragma unroll 2
        for (int t = share_lo32(T.nt, r, C) + tid; t < t1; t += nthr)
            triangle_force(T, P, t, dSg, dV, F);
    }
    tm.sync_all();  // every block's partial forces complete

    // 4. this block's share of the nodes: forces summed over the cluster in
    //    rank order
    for (int p = share_lo(nn, r, C) + tid; p < share_lo(nn, r + 1, C); p += nthr) {
        f3 Fp = mk(0.f, 0.f, 0.f);
        for (int j = 0; j < C; ++j) {
            const float *Fj = tm.peer(sh, j) + 8 * nn;
            Fp = Fp + mk(Fj[p], Fj[nn + p], Fj[2 * nn + p]);
        }
        if (s.rep_wall_on) Fp.y += wall_force(s, s.Xh[NN + f0 + p], s.Xl[NN + f0 + p]);
        s.Fel[f0 + p] = Fp.x;
        s.Fel[NN + f0 + p] = Fp.y;
        s.Fel[2 * NN + f0 + p] = Fp.z;
    }
    tm.sync_all();  // remote reads complete before any block reuses its shared memory
}

// Coupling part for global node i.
template <bool EARLY>
__device__ __forceinline__ void node_step(const SimDev &s, int i, int par) {
    const int o = s.node_obj[i];
    node_update<EARLY>(s, o, i, s.obj[o].inv_mass, par);
}

}  // namespace lbib
