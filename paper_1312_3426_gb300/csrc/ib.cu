// Immersed-boundary kernels of one simulation: the membrane part (one
// thread-block cluster per object) and the coupling part (one thread per
// node), as described in ib_core.cuh.
#include "ib_core.cuh"

namespace lbib {

extern __shared__ float ib_smem[];

// Cluster c takes objects c, c + n_clusters, ... (a grid smaller than the
// object count leaves SMs to the fluid kernel that runs beside it).
__global__ void __launch_bounds__(IB_THREADS, 4) k_membrane(SimDev s) {
    const ClusterTeam tm;
    const int C = tm.ranks();
    const int n_clusters = (int)(gridDim.x / C);
    for (int o = (int)(blockIdx.x / C); o < s.nobj; o += n_clusters) membrane_object(s, o, ib_smem, tm);
}

// Several objects per block: group g (threads [g T, (g + 1) T)) of block b
// takes object b G + g with its own shared memory and named barrier g + 1.
// A few dense blocks hold a few SMs for a short time, where one block per
// object would hold a slot on almost every SM while the fluid kernel runs.
__global__ void __launch_bounds__(1024, 1) k_membrane_groups(SimDev s, int T, int group_floats) {
    const int g = (int)threadIdx.x / T, G = (int)blockDim.x / T;
    const int o = (int)blockIdx.x * G + g;
    if (o >= s.nobj) return;  // whole groups only: no barrier is shared with another group
    const GroupTeam tm{(int)threadIdx.x - g * T, T, g + 1};
    membrane_object(s, o, ib_smem + (size_t)g * group_floats, tm);
}

// NT nodes per block (LBIB_TUNE_NODE_THREADS: 32, 64, 128 or 256); EARLY:
// the instantiation for an early (programmatic dependent) launch
template <int NT, bool EARLY>
__global__ void __launch_bounds__(NT, 1024 / NT) k_nodes(SimDev s, int par) {
    const int i = blockIdx.x * NT + threadIdx.x;
    if (i < s.nn_total) node_step<EARLY>(s, i, par);
}

cudaError_t launch_membrane(const SimDev &s, int max_nodes, int cluster, int max_clusters, int threads, int group,
                            cudaStream_t st) {
    if (s.nobj == 0) return cudaSuccess;
    // as many objects per block as fit (threads and shared memory), at most `group`
    const size_t per = ib_smem_bytes(max_nodes);  // a multiple of 16 bytes
    while (group > 1 && (group * threads > 1024 || group > 15 || per * (size_t)group > 227 * 1024)) --group;
    if (group > 1) {  // several objects per block (cluster size and cluster count do not apply)
        const size_t smem = per * (size_t)group;
        static SmemAttr gattr;
        cudaError_t eg = gattr.ensure((const void *)k_membrane_groups, smem, false);
        if (eg != cudaSuccess) return eg;
        const int blocks = (s.nobj + group - 1) / group;
        k_membrane_groups<<<blocks, group * threads, smem, st>>>(s, threads, (int)(per / sizeof(float)));
        return cudaGetLastError();
    }
    const size_t smem = per;
    static SmemAttr attr;
    cudaError_t ea = attr.ensure((const void *)k_membrane, smem, true);
    if (ea != cudaSuccess) return ea;
    cudaLaunchConfig_t cfg = {};
    const int n_clusters = (max_clusters > 0 && max_clusters < s.nobj) ? max_clusters : s.nobj;
    cfg.gridDim = dim3((unsigned)(n_clusters * cluster));
    cfg.blockDim = dim3((unsigned)threads);
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

cudaError_t launch_nodes(const SimDev &s, int par, int threads, cudaStream_t st, bool pdl) {
    if (s.nn_total == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((s.nn_total + threads - 1) / threads);
    switch (threads * 2 + (pdl ? 1 : 0)) {
        case 64: return launch_dep(k_nodes<32, false>, blocks, 32, st, false, s, par);
        case 65: return launch_dep(k_nodes<32, true>, blocks, 32, st, true, s, par);
        case 128: return launch_dep(k_nodes<64, false>, blocks, 64, st, false, s, par);
        case 129: return launch_dep(k_nodes<64, true>, blocks, 64, st, true, s, par);
        case 256: return launch_dep(k_nodes<128, false>, blocks, 128, st, false, s, par);
        case 257: return launch_dep(k_nodes<128, true>, blocks, 128, st, true, s, par);
        case 512: return launch_dep(k_nodes<256, false>, blocks, 256, st, false, s, par);
        case 513: return launch_dep(k_nodes<256, true>, blocks, 256, st, true, s, par);
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------ repulsion
// Object-object soft-sphere repulsion, in two launches after the membrane
// kernel (which wrote each object's bounding box):
//   k_rep_pairs   one thread per object pair (i < j): the periodic image of
//                 j nearest to i (minimum image of the box centres; the box
//                 is taken larger than twice an object plus the cutoff), and
//                 whether the boxes widened by the cutoff overlap; close
//                 pairs go to a list
//   k_rep_forces  one block per listed pair: j's nodes (shifted to the
//                 image) are staged in shared memory as hi + lo pairs; each
//                 thread takes nodes of i inside j's widened box and tests
//                 all of j's nodes; the pair force goes to i's node directly
//                 and to j's node through a shared-memory sum, both added
//                 to Fel with global atomics.
// Separations are formed as (hi_i - hi_j) + (lo_i - lo_j), exact in the
// leading part for nearby nodes, so the force does not lose digits at
// large coordinates.

__device__ __forceinline__ int image_shift(float ci, float cj, int L) {
    return (int)rintf((ci - cj) / (float)L);  // j + shift * L is the image nearest to i
}

__global__ void __launch_bounds__(256) k_rep_pairs(SimDev s) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j <= i || j >= s.nobj) return;
    const float *A = s.aabb + 8 * i, *B = s.aabb + 8 * j;
    const int L[3] = {s.nx, s.ny, s.nz};
    int k3[3];
    bool close = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const bool periodic = k != 1 || !s.walls;
        k3[k] = periodic ? image_shift(0.5f * (A[k] + A[3 + k]), 0.5f * (B[k] + B[3 + k]), L[k]) : 0;
        const float sh = (float)(k3[k] * L[k]);
        close = close && (B[k] + sh < A[3 + k] + s.rep_rc) && (A[k] < B[3 + k] + sh + s.rep_rc);
    }
    if (!close) return;
    const unsigned slot = atomicAdd(s.npairs, 1u);
    if (slot < (unsigned)s.pair_cap)
        s.pairs[slot] = make_int4(i | (j << 16), k3[0], k3[1], k3[2]);  // nobj <= 65535
    else
        atomicOr(s.status, ST_PAIRS);
}

extern __shared__ float rep_smem[];

__global__ void __launch_bounds__(256) k_rep_forces(SimDev s) {
    const unsigned np = min(*s.npairs, (unsigned)s.pair_cap);
    const int NN = s.nn_total;
    const float rc2 = s.rep_rc * s.rep_rc;
    for (unsigned p = blockIdx.x; p < np; p += gridDim.x) {
        const int4 pr = s.pairs[p];
        const int oi = pr.x & 0xffff, oj = (int)((unsigned)pr.x >> 16);
        const ObjDev A = s.obj[oi], B = s.obj[oj];
        const float sh[3] = {(float)(pr.y * s.nx), (float)(pr.z * s.ny), (float)(pr.w * s.nz)};
        float *bh = rep_smem, *bl = bh + 3 * B.nn, *bf = bl + 3 * B.nn;
        for (int q = threadIdx.x; q < B.nn; q += blockDim.x)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                // (hi + shift) as an unevaluated pair: the shift is an integer
                const df t = two_sum(s.Xh[k * NN + B.first + q], sh[k]);
                bh[3 * q + k] = t.hi;
                bl[3 * q + k] = t.lo + s.Xl[k * NN + B.first + q];
                bf[3 * q + k] = 0.f;
            }
        __syncthreads();
        const float *bb = s.aabb + 8 * oj;
        for (int a = threadIdx.x; a < A.nn; a += blockDim.x) {
            float xh[3], xl[3];
            bool inside = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                xh[k] = s.Xh[k * NN + A.first + a];
                xl[k] = s.Xl[k * NN + A.first + a];
                inside = inside && xh[k] > bb[k] + sh[k] - s.rep_rc - 1e-3f && xh[k] < bb[3 + k] + sh[k] + s.rep_rc + 1e-3f;
            }
            if (!inside) continue;
            float F[3] = {0.f, 0.f, 0.f};
            for (int q = 0; q < B.nn; ++q) {
                const float dx = (xh[0] - bh[3 * q]) + (xl[0] - bl[3 * q]);
                const float dy = (xh[1] - bh[3 * q + 1]) + (xl[1] - bl[3 * q + 1]);
                const float dz = (xh[2] - bh[3 * q + 2]) + (xl[2] - bl[3 * q + 2]);
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < rc2 && r2 > 0.f) {
                    const float rr = sqrtf(r2);
                    const float f = soft_force(s.rep_a, s.rep_n, rr) / rr;
                    F[0] += f * dx;
                    F[1] += f * dy;
                    F[2] += f * dz;
                    atomicAdd(bf + 3 * q, -f * dx);
                    atomicAdd(bf + 3 * q + 1, -f * dy);
                    atomicAdd(bf + 3 * q + 2, -f * dz);
                }
            }
            if (F[0] != 0.f || F[1] != 0.f || F[2] != 0.f)
#pragma unroll
                for (int k = 0; k < 3; ++k) atomicAdd(s.Fel + k * NN + A.first + a, F[k]);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < B.nn; q += blockDim.x)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (bf[3 * q + k] != 0.f) atomicAdd(s.Fel + k * NN + B.first + q, bf[3 * q + k]);
        __syncthreads();  // shared memory is restaged for the next pair
    }
}

cudaError_t launch_repulsion(const SimDev &s, int max_nodes, cudaStream_t st) {
    if (!s.rep_on || s.nobj < 2) return cudaSuccess;
    if (s.nobj > 65535) return cudaErrorInvalidValue;  // grid rows and the pair encoding
    cudaError_t e = cudaMemsetAsync(s.npairs, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    k_rep_pairs<<<dim3((s.nobj + 255) / 256, s.nobj), 256, 0, st>>>(s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = (size_t)9 * max_nodes * sizeof(float);
    static SmemAttr attr;
    if ((e = attr.ensure((const void *)k_rep_forces, smem, false)) != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_rep_forces<<<2 * sms, 256, smem, st>>>(s);
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
// velocity of one object (a read-out, not part of the step).  One block per
// object.  Sums are taken as error-free FP32 pairs over
// positions relative to the object's first node (hi + lo differences),
// reduced in a fixed order (so one object's analysis is bit-identical
// alone and in the all-objects launch) and finished in FP64.
__global__ void __launch_bounds__(256) k_analyze(SimDev s, int oid, double *out) {
    if (oid < 0) {
        oid = blockIdx.x;
        out += 14 * (size_t)oid;
    }
    const ObjDev ob = s.obj[oid];
    const TplDev &T = s.tpl[ob.tid];
    const int NN = s.nn_total, f0 = ob.first;
    const float bh[3] = {s.Xh[f0], s.Xh[NN + f0], s.Xh[2 * NN + f0]};
    const float bl[3] = {s.Xl[f0], s.Xl[NN + f0], s.Xl[2 * NN + f0]};
    auto rel = [&](int k, int p) {  // node p relative to the first node
        return (s.Xh[k * NN + f0 + p] - bh[k]) + (s.Xl[k * NN + f0 + p] - bl[k]);
    };
    df acc[8] = {};  // sum of relative x, y, z; of v x, y, z; area; 6 x volume
    float mn[3] = {3.0e38f, 3.0e38f, 3.0e38f}, mx[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    for (int p = threadIdx.x; p < ob.nn; p += blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float q = rel(k, p);
            acc[k] = df_add_f(acc[k], q);
            mn[k] = fminf(mn[k], q);
            mx[k] = fmaxf(mx[k], q);
            acc[3 + k] = df_add(acc[3 + k], df{s.Vh[k * NN + f0 + p], s.Vl[k * NN + f0 + p]});
        }
    }
    for (int t = threadIdx.x; t < T.nt; t += blockDim.x) {
        const int4 tr = T.tri[t];
        const f3 A = mk(rel(0, tr.x), rel(1, tr.x), rel(2, tr.x));
        const f3 B = mk(rel(0, tr.y), rel(1, tr.y), rel(2, tr.y)) - A;
        const f3 Cc = mk(rel(0, tr.z), rel(1, tr.z), rel(2, tr.z)) - A;
        const f3 N = cross(B, Cc);
        acc[6] = df_add_f(acc[6], 0.5f * sqrtf(dot(N, N)));
        acc[7] = df_add_f(acc[7], dot(A, N));
    }
    // fixed-order reduction: warp shuffles, then warp 0 over the warps
    __shared__ df wacc[8][8];
    __shared__ float wmn[3][8], wmx[3][8];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = warp_sum_df(acc[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
        }
    if (lane == 0) {
        for (int k = 0; k < 8; ++k) wacc[k][w] = acc[k];
        for (int k = 0; k < 3; ++k) {
            wmn[k][w] = mn[k];
            wmx[k][w] = mx[k];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (int)(blockDim.x >> 5);
        double tot[8];
        for (int k = 0; k < 8; ++k) {
            df t = wacc[k][0];
            for (int j = 1; j < nw; ++j) t = df_add(t, wacc[k][j]);
            tot[k] = (double)t.hi + (double)t.lo;
        }
        const double inv = 1.0 / ob.nn;
        for (int k = 0; k < 3; ++k) {
            const double base = (double)bh[k] + (double)bl[k];
            float lo = wmn[k][0], hi = wmx[k][0];
            for (int j = 1; j < nw; ++j) {
                lo = fminf(lo, wmn[k][j]);
                hi = fmaxf(hi, wmx[k][j]);
            }
            out[k] = base + tot[k] * inv;
            out[3 + 2 * k] = base + (double)lo;
            out[4 + 2 * k] = base + (double)hi;
            out[11 + k] = tot[3 + k] * inv;
        }
        out[9] = -tot[7] / 6.0;
        out[10] = tot[6];
    }
}

cudaError_t launch_analyze(const SimDev &s, int oid, double *out, cudaStream_t st) {
    if (oid < 0 && s.nobj == 0) return cudaSuccess;
    k_analyze<<<oid < 0 ? s.nobj : 1, 256, 0, st>>>(s, oid, out);
    return cudaGetLastError();
}

}  // namespace lbib
