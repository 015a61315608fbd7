// Immersed-boundary kernels: one thread block per object.
//
// Per step and object (Sec. 4 and Sec. 2 of arXiv:1312.3426):
//   1. positions relative to the object's first node are split into a
//      float "hi" part and a float remainder "lo" and staged in shared
//      memory, so that differences of nearby nodes are formed in FP32 with
//      FP64-like accuracy ((hi_q - hi_p) is exact for nearby values);
//   2. total area S_g and volume V (Sec. 4, global area and volume
//      conservation): per-triangle terms in FP32, accumulated in FP64 with
//      warp shuffles and one shared-memory pass;
//   3. every node gathers the forces acting on it from its incidence
//      records (node-centric: no atomics, deterministic order):
//        stretching (Eq. stretching)  ks kappa(lambda) (L-L0)/L0 along the edge,
//        bending                      kb (theta-theta0)/theta0 along the
//                                     inward normal on the apex, minus half
//                                     of each triangle's term on the edge nodes,
//        local area                   -kal (S-S0)/S w,
//        global area                  -kag (S_g-S_g0)/S_g w,
//        volume                       kv (V-V0)/V0 S n_in / 3 per triangle,
//      with w the unit vector from the triangle centroid to the node;
//   4. the fluid velocity is interpolated trilinearly from the 8 lattice
//      nodes around the node (u = 0 on solid rows), the drag
//      F_d = xi (u - v) acts on the node and -F_d is added with the same
//      weights to the coupling force field (one 16-byte vector atomic per
//      corner, plus a bit in the live-entry mask);
//   5. Newton's law (Eq. newton) with unit time step: v += (F + F_d +
//      F_ext)/m, X += v in FP64; the 8 lattice nodes around the new position
//      are marked so that the next fluid step writes their velocity.
// FP64 is used only for the node state, the reductions and the drag
// difference: the FP64 rate of this GPU is a small fraction of FP32.
#include "ib_core.cuh"

namespace lbib {

extern __shared__ float ib_smem[];

__global__ void __launch_bounds__(IB_THREADS) k_ib(SimDev s, int par) {
    ib_object(s, blockIdx.x, par, ib_smem);
}

cudaError_t ib_configure(int max_nodes) {
    const int bytes = 6 * (int)sizeof(float) * max_nodes;
    return cudaFuncSetAttribute(k_ib, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes > 48 * 1024 ? bytes : 48 * 1024);
}

cudaError_t launch_ib(const SimDev &s, int par, int max_nodes, cudaStream_t st) {
    if (s.nobj == 0) return cudaSuccess;
    const size_t smem = 6 * sizeof(float) * (size_t)max_nodes;
    k_ib<<<s.nobj, IB_THREADS, smem, st>>>(s, par);
    return cudaGetLastError();
}

// Object analysis (Sec. 5): mean position, bounds, volume, area, mean
// velocity of one object, all in FP64 (a read-out, not part of the step).
__global__ void k_analyze(SimDev s, int oid, double *out) {
    if (oid < 0) {
        oid = blockIdx.x;
        out += 14 * (size_t)oid;
    }
    const ObjDev ob = s.obj[oid];
    const TplDev T = s.tpl[ob.tid];
    const int NN = s.nn_total;
    const double *Xx = s.X, *Xy = s.X + NN, *Xz = s.X + 2 * NN;
    const double *Vx = s.V, *Vy = s.V + NN, *Vz = s.V + 2 * NN;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // sx sy sz vx vy vz S V
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int p = threadIdx.x; p < ob.nn; p += blockDim.x) {
        const int i = ob.first + p;
        const double q[3] = {Xx[i], Xy[i], Xz[i]};
        for (int k = 0; k < 3; ++k) {
            acc[k] += q[k];
            mn[k] = fmin(mn[k], q[k]);
            mx[k] = fmax(mx[k], q[k]);
        }
        acc[3] += Vx[i];
        acc[4] += Vy[i];
        acc[5] += Vz[i];
    }
    const int f0 = ob.first;
    for (int t = threadIdx.x; t < T.nt; t += blockDim.x) {
        const int4 tr = T.tri[t];
        double a[3] = {Xx[f0 + tr.x] - Xx[f0], Xy[f0 + tr.x] - Xy[f0], Xz[f0 + tr.x] - Xz[f0]};
        double b[3] = {Xx[f0 + tr.y] - Xx[f0], Xy[f0 + tr.y] - Xy[f0], Xz[f0 + tr.y] - Xz[f0]};
        double c[3] = {Xx[f0 + tr.z] - Xx[f0], Xy[f0 + tr.z] - Xy[f0], Xz[f0 + tr.z] - Xz[f0]};
        const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        acc[6] += 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        acc[7] += -(a[0] * n[0] + a[1] * n[1] + a[2] * n[2]) / 6.0;
    }
    __shared__ double sacc[8][256];
    __shared__ double smn[3][256], smx[3][256];
    for (int k = 0; k < 8; ++k) sacc[k][threadIdx.x] = acc[k];
    for (int k = 0; k < 3; ++k) {
        smn[k][threadIdx.x] = mn[k];
        smx[k][threadIdx.x] = mx[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int t = 1; t < blockDim.x; ++t) {
            for (int k = 0; k < 8; ++k) sacc[k][0] += sacc[k][t];
            for (int k = 0; k < 3; ++k) {
                smn[k][0] = fmin(smn[k][0], smn[k][t]);
                smx[k][0] = fmax(smx[k][0], smx[k][t]);
            }
        }
        const double inv = 1.0 / ob.nn;
        for (int k = 0; k < 3; ++k) out[k] = sacc[k][0] * inv;
        for (int k = 0; k < 3; ++k) {
            out[3 + 2 * k] = smn[k][0];
            out[4 + 2 * k] = smx[k][0];
        }
        out[9] = sacc[7][0];
        out[10] = sacc[6][0];
        for (int k = 0; k < 3; ++k) out[11 + k] = sacc[3 + k][0] * inv;
    }
}

cudaError_t launch_analyze(const SimDev &s, int oid, double *out, cudaStream_t st) {
    if (oid < 0 && s.nobj == 0) return cudaSuccess;
    k_analyze<<<oid < 0 ? s.nobj : 1, 256, 0, st>>>(s, oid, out);
    return cudaGetLastError();
}

}  // namespace lbib
