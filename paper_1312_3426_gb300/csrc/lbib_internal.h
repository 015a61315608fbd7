// Internal declarations shared by the translation units of the CUDA library.
//
// Device data layout (one simulation):
//   fluid cells      only the fluid rows are stored; fluid index
//                    f = x + nx * (y' + nyf * z), y' = y - 1 with walls
//                    (nyf = ny - 2), y' = y without (nyf = ny).
//   populations      pop[2][19][nfp] of the storage type, direction-major
//                    (plane stride nfp = nf rounded up to 64 elements), the
//                    deviation h_i = f_i - w_i rho0 (times 2^s for FP16/BF16).
//                    Step t pulls from pop[t&1] and writes pop[(t+1)&1].
//   active cells     bit f of amask[nwords] marks the cells near objects: the
//                    4x4x4 lattice nodes around every node (its 8
//                    interpolation corners and a one-cell halo).  A node
//                    marks them when its lower corner changes; marks persist
//                    until a periodic reset, after which all nodes re-mark.
//                    Nodes move less than one cell per step, so a node's
//                    corners at the next step are always active already.
//   coupling force   G[2][nf] float4, dense, non-zero only at active cells.
//                    Step t spreads into G[t&1]; the fluid step t adds
//                    G[t&1] at active cells and zeroes G[(t+1)&1] there (the
//                    buffer step t+1 spreads into), so after step t the
//                    buffer of step t is still readable.
//   velocity samples ufield[nf] float4 (u, rho) written by the fluid step at
//                    active cells and read at the node corners by the next
//                    step.
//   nodes            positions and velocities as unevaluated sums of two
//                    FP32 numbers (hi + lo, about 48 significant bits):
//                    Xh, Xl, Vh, Vl each [3][nn_total], structure of arrays,
//                    objects contiguous in id order.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <stdint.h>

#include "lbib.h"

namespace lbib {

constexpr int NQ = 19;
constexpr int FLUID_THREADS = 256;
constexpr int IB_THREADS = 256;          // largest block of the object kernels
constexpr int IB_THREADS_DEFAULT = 256;  // node kernel block (LBIB_TUNE_NODE_THREADS)
constexpr int MAX_TEMPLATE_NODES = 5120;  // 11 floats of shared memory per node
constexpr int ACTIVE_RESET_STEPS = 128;    // period of the active-cell re-marking

// D3Q19 directions of this library: rest, the 6 axis directions in +/- pairs,
// then the 12 face diagonals in +/- pairs; opposite(q) = q+1 for odd q,
// q-1 for even q > 0.
__host__ __device__ constexpr int d3q19_ex(int q) {
    constexpr int t[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[q];
}
__host__ __device__ constexpr int d3q19_ey(int q) {
    constexpr int t[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return t[q];
}
__host__ __device__ constexpr int d3q19_ez(int q) {
    constexpr int t[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return t[q];
}
__host__ __device__ constexpr int d3q19_opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr double d3q19_w(int q) { return q == 0 ? 1.0 / 3.0 : (q < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }

// Device status bits (sticky per simulation).
enum : uint32_t {
    ST_UNSTABLE = 1u,     // NaN or |u|^2 > 0.09 in a fluid cell
    ST_NODE_NAN = 2u,     // non-finite node position
    ST_TIMEOUT = 4u,      // a bounded device-side wait gave up
    ST_PAIRS = 8u,        // more close object pairs than the repulsion pair list holds
};

// Element lists of one template (device), all node ids local to an object,
// each in the bank-aware evaluation order of topology.cpp:
//   tri:        (a, b, c, rest area S0 as float bits), inward-ordered as given
//   quad:       per edge (b, c), b < c: (a, b, c, d), where (a,b,c) and
//               (d,c,b) are the inward cyclic orders of the two triangles
//               sharing it
//   hinge:      per edge, (rest length L0, 1/L0, 1/rest inner angle, 0)
struct TplDev {
    int nn, nt, ne;
    float ks, kb, kal, kag, kv;
    int nonlinear;
    int kal_altitude;  // local-area force along the altitudes (else centroid -> vertex)
    double Sg0, V0;
    const int4 *tri;
    const int4 *quad;
    const float4 *hinge;
};

// One object: its template, first global node, node count and 1/m.
struct ObjDev {
    int tid, first, nn;
    float inv_mass;
};

// Division by a fixed divisor d >= 1 of any 32-bit unsigned n with one
// multiply-high (Granlund and Montgomery, "Division by invariant integers
// using multiplication", PLDI 1994): l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((n - t) >> 1)) >> (l - 1)
// with t = mulhi(n, m); l = 0 (d = 1) gives q = n.
struct FastDiv {
    uint32_t m;
    int l;
    void init(uint32_t d) {
        l = 0;
        while ((1ull << l) < d) ++l;
        m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    }
#ifdef __CUDACC__
    __device__ __forceinline__ uint32_t div(uint32_t n) const {
        if (l == 0) return n;
        const uint32_t t = __umulhi(n, m);
        return (t + ((n - t) >> 1)) >> (l - 1);
    }
#endif
};

// Everything a kernel needs to know about one simulation (POD, passed by
// value to single-simulation kernels and stored in an array for batches).
struct SimDev {
    int nx, ny, nz, walls;
    FastDiv div_nx, div_nyf;  // cell index -> (x, row), row -> (y, z)
    int nyf, nf, nfp, nwords;
    int prec;                 // lbib_precision
    float omega, fpre, rho0;  // 1/tau, 1 - 1/(2 tau), rest density
    float gx, gy, gz;         // body force
    float scale, inv_scale;   // 2^s, 2^-s
    float xi;
    void *pop[2];
    float4 *G[2];
    uint32_t *amask;
    float4 *ufield;
    float *Xh, *Xl, *Vh, *Vl; // [3][nn_total] each
    float *Fel;               // [3][nn_total] membrane force of the current step
    const int *node_obj;      // [nn_total] object of each node
    int nn_total, nobj;
    const ObjDev *obj;
    const float *fext;        // [nobj][3] external force per node of each object
    const TplDev *tpl;
    uint32_t *status;
    double *dropped;          // [3]
    // soft-sphere repulsion (a, n, cutoff): object-object and object-wall
    float rep_a, rep_n, rep_rc;
    float rep_wa, rep_wn, rep_wrc;
    int rep_on, rep_wall_on;
    float *aabb;              // [nobj][8]: min x,y,z, max x,y,z of each object's nodes
    int4 *pairs;              // close object pairs (i | j << 16, image shift x, y, z)
    unsigned *npairs;
    int pair_cap;
    // velocity inlet: cells x in [in_box[0], in_box[1]), y (lattice row, walls
    // included) in [in_box[2], in_box[3]), z in [in_box[4], in_box[5])
    int in_on;
    int in_box[6];
    float in_u[3];
    // obstacle cells (bit per fluid cell, nwords words; null: none): solid
    // like the wall rows
    const uint32_t *solid;
    int nsolid;
    // 16-bit storage: fluid kernel preference (0 and 1 two cells per thread
    // where the shape allows, 2 the warp-specialised two-cells kernel, 3 one
    // cell per thread)
    int fkern;
};

#ifdef __CUDACC__
__device__ __forceinline__ bool solid_bit(const SimDev &s, int f) {
    return (__ldg(s.solid + (f >> 5)) >> (f & 31)) & 1u;
}
#endif

// Raises a kernel's dynamic shared-memory limit (and, for cluster kernels,
// allows non-portable cluster sizes) once per device and size; safe to call
// from several threads.
struct SmemAttr {
    std::mutex mu;
    size_t done[64] = {};
    cudaError_t ensure(const void *fn, size_t bytes, bool cluster) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lock(mu);
        if (bytes <= done[dev] && done[dev] != 0) return cudaSuccess;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e == cudaSuccess && cluster) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e == cudaSuccess) done[dev] = bytes > 0 ? bytes : 1;
        return e;
    }
};

// ---- programmatic dependent launch -------------------------------------------
// A kernel launched with `pdl` may start while the kernel before it in the
// stream finishes.  It reads, before dep_wait(), only data that no kernel
// still running can be writing (see lbib_step), and after dep_wait() lets
// the next such kernel start (dep_release()).  Without the launch attribute
// both are no-ops.
#if defined(__CUDACC__)
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches k<<<grid, block, 0, st>>>(args...), with programmatic stream
// serialization when pdl.
template <typename... KArgs, typename... Args>
cudaError_t launch_dep(void (*k)(KArgs...), unsigned grid, unsigned block, cudaStream_t st, bool pdl, Args... args) {
    if (!pdl) {
        k<<<grid, block, 0, st>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}
#endif

// ---- launchers (fluid.cu) -------------------------------------------------
// pdl: launch with programmatic stream serialization (only right after the
// node kernel of the same step)
cudaError_t launch_fluid(const SimDev &s, int par, long long t, cudaStream_t st, bool pdl = false);
// the kernel launch_fluid picks (lbib_info out[7]): 0 one cell per thread,
// 1 two cells per thread, 2 warp-specialised two cells per thread
int fluid_kernel_kind(const SimDev &s);
// fluid_tma.cu: the warp-specialised kernel and whether the shape allows it
bool fluid_tma_shape(const SimDev &s);
cudaError_t launch_fluid_tma(const SimDev &s, int par, uint32_t seed, cudaStream_t st);
// the bounded-wait check of fluid_tma.cu (lbib_check_bounded_wait)
cudaError_t run_wait_probe(uint32_t *status, unsigned long long bound_ns, int arrive, cudaStream_t st);
cudaError_t launch_fields(const SimDev &s, int pop_par, int gmode, float *u_full, float *rho_full, int to_ufield,
                          cudaStream_t st);
cudaError_t launch_read_coupling(const SimDev &s, int gpar, float *g_full, cudaStream_t st);
cudaError_t launch_set_coupling(const SimDev &s, int gpar, const float *g_full, cudaStream_t st);
cudaError_t launch_read_pops(const SimDev &s, int pop_par, double *h_full, cudaStream_t st);
cudaError_t launch_set_pops(const SimDev &s, int pop_par, const double *h_full, cudaStream_t st);
cudaError_t launch_mass(const SimDev &s, int pop_par, double *acc, cudaStream_t st);
// allocation-free mass reduction: per-block partials into a static scratch
// array of MASS_SCRATCH_SLOTS doubles (8 KB) per device
constexpr int MASS_SCRATCH_SLOTS = 1024;
constexpr int MASS_SCRATCH_DEVICES = 64;
cudaError_t mass_scratch(double **ptr);
cudaError_t launch_mass_partials(const SimDev &s, int pop_par, double *part, int blocks, cudaStream_t st);

// ---- launchers (ib.cu) -----------------------------------------------------
// membrane part: clusters of `cluster` blocks, one per object or at most
// max_clusters (> 0) looping over the objects (max_nodes sizes shared
// memory); coupling part: one thread per node
// threads: block size (a multiple of 32, at most IB_THREADS)
// group > 1: `group` objects per block of group * threads threads instead
cudaError_t launch_membrane(const SimDev &s, int max_nodes, int cluster, int max_clusters, int threads, int group,
                            cudaStream_t st);
// pdl: launch with programmatic stream serialization (only right after the
// previous step's fluid kernel, a mask rebuild or a membrane kernel)
cudaError_t launch_nodes(const SimDev &s, int par, int threads, cudaStream_t st, bool pdl = false);
// object-object repulsion added to Fel (after the membrane kernel, which
// also writes the object bounding boxes); max_nodes sizes shared memory
cudaError_t launch_repulsion(const SimDev &s, int max_nodes, cudaStream_t st);
// oid >= 0: one object into out[14]; oid < 0: every object into out[nobj][14]
cudaError_t launch_mark_all(const SimDev &s, cudaStream_t st);
cudaError_t launch_analyze(const SimDev &s, int oid, double *out, cudaStream_t st);

}  // namespace lbib
