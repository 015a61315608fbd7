// Immersed-boundary kernels of one simulation: the membrane part (one
// thread-block cluster per object) and the coupling part (one thread per
// node), as described in ib_core.cuh.
#include "ib_core.cuh"

namespace lbib {

extern __shared__ float ib_smem[];

// Cluster c takes objects c, c + n_clusters, ... (a grid smaller than the
// object count leaves SMs to the fluid kernel that runs beside it).
__global__ void __launch_bounds__(IB_THREADS, 4) k_membrane(SimDev s) {
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int n_clusters = (int)(gridDim.x / C);
    for (int o = (int)(blockIdx.x / C); o < s.nobj; o += n_clusters) membrane_object(s, o, ib_smem);
}

__global__ void __launch_bounds__(IB_THREADS, 4) k_nodes(SimDev s, int par) {
    const int i = blockIdx.x * IB_THREADS + threadIdx.x;
    if (i < s.nn_total) node_step(s, i, par);
}

cudaError_t launch_membrane(const SimDev &s, int max_nodes, int cluster, int max_clusters, cudaStream_t st) {
    if (s.nobj == 0) return cudaSuccess;
    const size_t smem = ib_smem_bytes(max_nodes);
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(k_membrane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_membrane, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    cudaLaunchConfig_t cfg = {};
    const int n_clusters = (max_clusters > 0 && max_clusters < s.nobj) ? max_clusters : s.nobj;
    cfg.gridDim = dim3((unsigned)(n_clusters * cluster));
    cfg.blockDim = dim3(IB_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_membrane, s);
}

cudaError_t launch_nodes(const SimDev &s, int par, cudaStream_t st) {
    if (s.nn_total == 0) return cudaSuccess;
    k_nodes<<<(s.nn_total + IB_THREADS - 1) / IB_THREADS, IB_THREADS, 0, st>>>(s, par);
    return cudaGetLastError();
}

// Marks the cells around every node as active (after the mask was cleared).
__global__ void k_mark_all(SimDev s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= s.nn_total) return;
    const int NN = s.nn_total;
    const df x{s.Xh[i], s.Xl[i]}, y{s.Xh[NN + i], s.Xl[NN + i]}, z{s.Xh[2 * NN + i], s.Xl[2 * NN + i]};
    if (!isfinite(x.hi) || !isfinite(y.hi) || !isfinite(z.hi)) return;
    const int3 c = lower_corner(x, y, z);
    mark_halo(s, c.x, c.y, c.z);
}

cudaError_t launch_mark_all(const SimDev &s, cudaStream_t st) {
    if (s.nn_total == 0) return cudaSuccess;
    k_mark_all<<<(s.nn_total + 255) / 256, 256, 0, st>>>(s);
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
    auto X = [&](int k, int i) { return (double)s.Xh[k * NN + i] + (double)s.Xl[k * NN + i]; };
    auto V = [&](int k, int i) { return (double)s.Vh[k * NN + i] + (double)s.Vl[k * NN + i]; };
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // sx sy sz vx vy vz S V
    double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
    for (int p = threadIdx.x; p < ob.nn; p += blockDim.x) {
        const int i = ob.first + p;
        for (int k = 0; k < 3; ++k) {
            const double q = X(k, i);
            acc[k] += q;
            mn[k] = fmin(mn[k], q);
            mx[k] = fmax(mx[k], q);
            acc[3 + k] += V(k, i);
        }
    }
    const int f0 = ob.first;
    for (int t = threadIdx.x; t < T.nt; t += blockDim.x) {
        const int4 tr = T.tri[t];
        double a[3], b[3], c[3];
        for (int k = 0; k < 3; ++k) {
            const double o = X(k, f0);
            a[k] = X(k, f0 + tr.x) - o;
            b[k] = X(k, f0 + tr.y) - o;
            c[k] = X(k, f0 + tr.z) - o;
        }
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
