// Batched step: many independent simulations advanced together.
//
// A step of the batch is the step of lbib_step (see capi.cu) with every
// kernel launched once for all simulations over a flat work list:
//   node kernel      one block per (simulation, run of IB_THREADS nodes)
//   fluid kernel     one block per (simulation, run of FLUID_THREADS cells),
//                    one launch per storage type present
//   membrane kernel  one thread-block cluster per (simulation, object), on a
//                    second stream while the fluid kernel runs (it prepares
//                    the next step)
// so the launch count per step does not grow with the number of
// simulations, and small simulations fill the GPU together.  Every block
// reads its simulation's descriptor and step counter from device arrays;
// the step offset inside a chunk is a kernel argument.  Chunks of
// LBIB_BATCH_GRAPH_STEPS steps are captured once as a CUDA graph (both
// streams) and replayed; a small kernel at the end of the graph advances
// the per-simulation step counters, so one graph serves every chunk of a
// call and later calls on the same set of simulations.
//
// The per-item device code is the code of the single-simulation kernels, so
// a simulation advanced in a batch computes what lbib_step computes for it
// alone, up to the order of the FP32 atomics of the spreading and of the
// membrane-force sums (as between two runs of lbib_step).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fluid_core.cuh"
#include "ib_core.cuh"
#include "sim.h"

namespace lbib {

constexpr int LBIB_BATCH_GRAPH_STEPS = 16;  // steps per captured graph

extern __shared__ float batch_smem[];

// One launch per storage type and boundary-condition variant present in the
// batch (items grouped by both; BC: obstacles or an inlet).
// L2 prefetch of the sources of work item blockIdx.x + pf of the same
// launch (items of one launch run roughly in index order); CELLS cells per
// item.
template <int ESZ, int CELLS>
__device__ __forceinline__ void prefetch_item(const SimDev *__restrict__ sims, const long long *__restrict__ t_base,
                                              int step_off, const int2 *__restrict__ items, int pf) {
    if (threadIdx.x >= NQ || (int)(blockIdx.x + pf) >= (int)gridDim.x) return;
    const int2 it = items[blockIdx.x + pf];
    const SimDev &s = sims[it.x];
    prefetch_cells<ESZ, CELLS>(s, s.pop[(t_base[it.x] + step_off) & 1], (long long)it.y * CELLS);
}

template <typename T, bool BC>
__global__ void __launch_bounds__(FLUID_THREADS, 5)
    k_batch_fluid(const SimDev *__restrict__ sims, const long long *__restrict__ t_base, int step_off,
                  const int2 *__restrict__ items, int pf) {
    prefetch_item<sizeof(T), FLUID_THREADS>(sims, t_base, step_off, items, pf);
    const int2 it = items[blockIdx.x];  // (simulation, block of cells)
    const SimDev &s = sims[it.x];
    const long long t = t_base[it.x] + step_off;
    fluid_block<T, BC, false>(s, (int)(t & 1), it.y * FLUID_THREADS, step_seed(t));
}

// 16-bit storage, even nx, plain boundaries: two cells per thread.
template <typename T>
__global__ void __launch_bounds__(FLUID_THREADS, 3)
    k_batch_fluid_pair(const SimDev *__restrict__ sims, const long long *__restrict__ t_base, int step_off,
                       const int2 *__restrict__ items, int pf) {
    prefetch_item<2, 2 * FLUID_THREADS>(sims, t_base, step_off, items, pf);
    const int2 it = items[blockIdx.x];  // (simulation, block of FLUID_THREADS cell pairs)
    const SimDev &s = sims[it.x];
    const long long t = t_base[it.x] + step_off;
    const int f = 2 * (it.y * FLUID_THREADS + (int)threadIdx.x);
    if (f < s.nf) fluid_pair<T, false>(s, (int)(t & 1), f, step_seed(t));
}

// NT nodes per work item (the plan's node chunk); 64 registers, a full
// SM of threads (the small spill costs less than the fifth wave of the
// 80-register form: 0.317 against 0.318 ms per step for 64 channels)
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT)
    k_batch_nodes(const SimDev *__restrict__ sims, const long long *__restrict__ t_base, int step_off,
                  const int2 *__restrict__ items) {
    const int2 it = items[blockIdx.x];  // (simulation, first node)
    const SimDev &s = sims[it.x];
    const int i = it.y + (int)threadIdx.x;
    if (i < s.nn_total) node_step<false>(s, i, (int)((t_base[it.x] + step_off) & 1));
}

__global__ void __launch_bounds__(IB_THREADS, 4)
    k_batch_membrane(const SimDev *__restrict__ sims, const int2 *__restrict__ items) {
    cg::cluster_group cl = cg::this_cluster();
    const int2 it = items[blockIdx.x / cl.num_blocks()];  // (simulation, object)
    membrane_object(sims[it.x], it.y, batch_smem, ClusterTeam());
}

// Several (simulation, object) items per block: group g of block b takes
// item b G + g with its own shared memory and named barrier g + 1.
__global__ void __launch_bounds__(1024, 1)
    k_batch_membrane_groups(const SimDev *__restrict__ sims, const int2 *__restrict__ items, int n_items, int T,
                            int group_floats) {
    const int g = (int)threadIdx.x / T, G = (int)blockDim.x / T;
    const int k = (int)blockIdx.x * G + g;
    if (k >= n_items) return;  // whole groups only
    const int2 it = items[k];
    const GroupTeam tm{(int)threadIdx.x - g * T, T, g + 1};
    membrane_object(sims[it.x], it.y, batch_smem + (size_t)g * group_floats, tm);
}

__global__ void k_batch_advance(long long *t_base, int n, int steps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) t_base[i] += steps;
}

// A batch plan: device copies of the descriptors and the work lists, and
// the captured graph; rebuilt when the set of simulations, their objects or
// the cluster size change.
struct BatchPlan {
    std::vector<lbib_sim *> sims;
    std::vector<uint64_t> serial;  // identity of each simulation (addresses can be reused)
    std::vector<int> nobj, nn, group;  // group: fluid kernel variant (2 * precision + BC)
    std::vector<SimDev> dev;  // descriptors the device copy holds
    int cluster = 0, device = -1, mthreads = IB_THREADS, nthreads = IB_THREADS_DEFAULT, mgroup = 1;
    SimDev *d_sims = nullptr;
    long long *d_t = nullptr;
    int2 *d_items = nullptr;  // fluid (by storage type x obstacles), then node, then membrane items
    int n_flp[8] = {};  // fluid items per kernel variant (see fluid_group)
    int n_fl = 0, n_nd = 0, n_mb = 0;
    int max_nodes = 0;
    // size classes of the membrane items (largest first): the n_big items
    // within a factor 2 of the largest, and the rest, whose largest has
    // rest_nodes nodes (0: one class)
    int n_big = 0, rest_nodes = 0;
    int pf_cell = 0, pf_pair = 0;  // L2 prefetch distances of the fluid launches (work items)
    cudaStream_t aux = nullptr;   // membrane kernel
    cudaStream_t aux2 = nullptr;  // membrane kernel of the smaller size class
    cudaEvent_t ev_rest = nullptr;
    cudaStream_t gst = nullptr;   // graph launches (the caller's stream may be the legacy one, which cannot be captured)
    cudaEvent_t ev_nodes = nullptr, ev_membrane = nullptr, ev_join = nullptr;
    cudaGraphExec_t graph = nullptr;

    void release_graph() {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
    }
    void release() {
        release_graph();
        cudaFree(d_sims);
        cudaFree(d_t);
        cudaFree(d_items);
        d_sims = nullptr;
        d_t = nullptr;
        d_items = nullptr;
        sims.clear();
        serial.clear();
        nobj.clear();
        nn.clear();
        group.clear();
        dev.clear();
    }
};

// One plan per process; lbib_batch_step calls are serialised on it.
static BatchPlan g_plan;
static std::mutex g_plan_mu;

// Fluid kernel variant of a simulation: 2 * precision + BC (obstacles or an
// inlet) for the one-cell-per-thread kernels; 6 / 7 for the two-cells
// kernels of FP16 / BF16 storage (even nx, plain boundaries).
static int fluid_group(const lbib_sim *s) {
    const bool bc = s->d.solid || s->d.in_on;
    if (s->d.prec != LBIB_POP_F32 && (s->d.nx & 1) == 0 && !bc && s->d.fkern != 3) return 6 + (s->d.prec - 1);
    return 2 * s->d.prec + (bc ? 1 : 0);
}

static bool plan_matches(lbib_sim *const *sims, int n, int cluster) {
    if ((int)g_plan.sims.size() != n || g_plan.cluster != cluster || g_plan.device != sims[0]->device ||
        g_plan.nthreads != sims[0]->node_threads)
        return false;
    for (int i = 0; i < n; ++i)
        if (g_plan.sims[i] != sims[i] || g_plan.serial[i] != sims[i]->serial ||
            g_plan.nobj[i] != (int)sims[i]->objs.size() || g_plan.group[i] != fluid_group(sims[i]) ||
            g_plan.nn[i] != sims[i]->nn_total)
            return false;
    return true;
}

static cudaError_t set_membrane_attrs(size_t smem) {
    static SmemAttr attr;
    return attr.ensure((const void *)k_batch_membrane, smem, true);
}

static cudaError_t build_plan(lbib_sim *const *sims, int n, int cluster, cudaStream_t st) {
    g_plan.release();
    const int nthreads = sims[0]->node_threads;  // node chunk of the batch
    if (!g_plan.aux) {
        int lo = 0, hi = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&g_plan.aux, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&g_plan.aux2, cudaStreamNonBlocking, hi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g_plan.ev_rest, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g_plan.gst, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g_plan.ev_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g_plan.ev_nodes, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g_plan.ev_membrane, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    std::vector<int2> flp[8], fl, nd, mb;
    int max_nodes = 0;
    for (int i = 0; i < n; ++i) {
        const lbib_sim *s = sims[i];
        const int grp = fluid_group(s);
        const int cells_per_block = grp >= 6 ? 2 * FLUID_THREADS : FLUID_THREADS;
        const int blocks = (s->d.nf + cells_per_block - 1) / cells_per_block;
        for (int b = 0; b < blocks; ++b) flp[grp].push_back(make_int2(i, b));
        if (!s->objs.empty()) {
            for (int f = 0; f < s->nn_total; f += nthreads) nd.push_back(make_int2(i, f));
            for (int o = 0; o < (int)s->objs.size(); ++o) mb.push_back(make_int2(i, o));
            max_nodes = std::max(max_nodes, s->max_nodes);
        }
    }
    // largest objects first: their clusters start in the first wave and the
    // small ones fill in behind them (longest-processing-time-first order),
    // so a level-4 cell does not start late and set the launch's tail
    std::stable_sort(mb.begin(), mb.end(), [&](const int2 &a, const int2 &b) {
        return sims[a.x]->objs[a.y].nn > sims[b.x]->objs[b.y].nn;
    });
    for (int k = 0; k < 8; ++k) {
        g_plan.n_flp[k] = (int)flp[k].size();
        fl.insert(fl.end(), flp[k].begin(), flp[k].end());
    }
    std::vector<int2> items(fl);
    items.insert(items.end(), nd.begin(), nd.end());
    items.insert(items.end(), mb.begin(), mb.end());
    cudaError_t e;
    if ((e = cudaMalloc(&g_plan.d_sims, n * sizeof(SimDev))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_t, n * sizeof(long long))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_items, std::max<size_t>(1, items.size()) * sizeof(int2))) != cudaSuccess) return e;
    if (!items.empty() &&
        (e = cudaMemcpyAsync(g_plan.d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    g_plan.sims.assign(sims, sims + n);
    for (int i = 0; i < n; ++i) {
        g_plan.serial.push_back(sims[i]->serial);
        g_plan.group.push_back(fluid_group(sims[i]));
        g_plan.nobj.push_back((int)sims[i]->objs.size());
        g_plan.nn.push_back(sims[i]->nn_total);
    }
    g_plan.n_fl = (int)fl.size();
    g_plan.n_nd = (int)nd.size();
    g_plan.n_mb = (int)mb.size();
    g_plan.cluster = cluster;
    g_plan.nthreads = nthreads;
    g_plan.device = sims[0]->device;
    {
        int sms = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g_plan.device)) != cudaSuccess) return e;
        g_plan.pf_cell = 3 * sms / 2;  // 1.5 blocks per SM ahead (5 resident)
        g_plan.pf_pair = sms;          // 1 block per SM ahead (3 resident)
    }
    g_plan.max_nodes = max_nodes;
    g_plan.n_big = 0;
    while (g_plan.n_big < (int)mb.size() && 2 * sims[mb[g_plan.n_big].x]->objs[mb[g_plan.n_big].y].nn > max_nodes)
        ++g_plan.n_big;
    g_plan.rest_nodes = g_plan.n_big < (int)mb.size() ? sims[mb[g_plan.n_big].x]->objs[mb[g_plan.n_big].y].nn : 0;
    return g_plan.n_mb ? set_membrane_attrs(ib_smem_bytes(max_nodes)) : cudaSuccess;
}

static cudaError_t launch_repulsion_batch(cudaStream_t st) {
    for (lbib_sim *s : g_plan.sims) {
        if (!s->d.rep_on) continue;
        cudaError_t e = launch_repulsion(s->d, s->max_nodes, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Membrane items [first, first + n) with up to G per block, each with a
// shared-memory slice for max_nodes nodes (G drops to what fits).
static cudaError_t launch_membrane_groups(cudaStream_t st, int first, int n, int max_nodes, int G) {
    const size_t per = ib_smem_bytes(max_nodes);
    while (G > 1 && (G * g_plan.mthreads > 1024 || per * G > (size_t)227 * 1024)) --G;
    static SmemAttr gattr;
    cudaError_t e = gattr.ensure((const void *)k_batch_membrane_groups, per * G, false);
    if (e != cudaSuccess) return e;
    const int blocks = (n + G - 1) / G;
    k_batch_membrane_groups<<<blocks, G * g_plan.mthreads, per * G, st>>>(
        (const SimDev *)g_plan.d_sims, (const int2 *)(g_plan.d_items + g_plan.n_fl + g_plan.n_nd + first), n,
        g_plan.mthreads, (int)(per / sizeof(float)));
    return cudaGetLastError();
}

// On `st` (which waits for the node update): the membrane forces, then the
// repulsion.  With several objects per block, the objects within a factor 2
// of the largest run in one launch (their slices sized for the largest) and
// the others beside it on a second stream (slices sized for theirs), so a
// level-2 object does not hold the shared memory of a level-4 one.
static cudaError_t launch_membrane_batch(cudaStream_t st) {
    if (g_plan.n_mb == 0) return cudaSuccess;
    const int G = g_plan.mgroup;
    const size_t per = ib_smem_bytes(g_plan.max_nodes);
    if (G > 1 && g_plan.n_big < g_plan.n_mb) {
        cudaError_t e;
        if ((e = cudaStreamWaitEvent(g_plan.aux2, g_plan.ev_nodes, 0)) != cudaSuccess) return e;
        if ((e = launch_membrane_groups(g_plan.aux2, g_plan.n_big, g_plan.n_mb - g_plan.n_big, g_plan.rest_nodes, G)) !=
            cudaSuccess)
            return e;
        if ((e = cudaEventRecord(g_plan.ev_rest, g_plan.aux2)) != cudaSuccess) return e;
        if ((e = launch_membrane_groups(st, 0, g_plan.n_big, g_plan.max_nodes, G)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, g_plan.ev_rest, 0)) != cudaSuccess) return e;
        return launch_repulsion_batch(st);
    }
    if (G > 1 && G * g_plan.mthreads <= 1024 && per * G <= (size_t)227 * 1024) {
        cudaError_t e = launch_membrane_groups(st, 0, g_plan.n_mb, g_plan.max_nodes, G);
        return e == cudaSuccess ? launch_repulsion_batch(st) : e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(g_plan.n_mb * g_plan.cluster));
    cfg.blockDim = dim3((unsigned)g_plan.mthreads);
    cfg.dynamicSmemBytes = ib_smem_bytes(g_plan.max_nodes);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)g_plan.cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_batch_membrane, (const SimDev *)g_plan.d_sims,
                                       (const int2 *)(g_plan.d_items + g_plan.n_fl + g_plan.n_nd));
    // object-object repulsion of the simulations that set it (per simulation)
    return e == cudaSuccess ? launch_repulsion_batch(st) : e;
}

// Steps step_off .. step_off + k - 1 relative to the device step counters,
// on `st` and the plan's second stream; `st` has caught up with the second
// stream at the end.
static cudaError_t enqueue_steps(cudaStream_t st, int step_off, int k) {
    cudaError_t e = cudaSuccess;
    const int2 *fl = g_plan.d_items, *nd = g_plan.d_items + g_plan.n_fl;
    for (int j = 0; j < k && e == cudaSuccess; ++j) {
        const int off = step_off + j;
        if (g_plan.n_nd) {
            switch (g_plan.nthreads) {
                case 32: k_batch_nodes<32><<<g_plan.n_nd, 32, 0, st>>>(g_plan.d_sims, g_plan.d_t, off, nd); break;
                case 64: k_batch_nodes<64><<<g_plan.n_nd, 64, 0, st>>>(g_plan.d_sims, g_plan.d_t, off, nd); break;
                case 128: k_batch_nodes<128><<<g_plan.n_nd, 128, 0, st>>>(g_plan.d_sims, g_plan.d_t, off, nd); break;
                default: k_batch_nodes<256><<<g_plan.n_nd, 256, 0, st>>>(g_plan.d_sims, g_plan.d_t, off, nd); break;
            }
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaEventRecord(g_plan.ev_nodes, st)) != cudaSuccess) break;
            if ((e = cudaStreamWaitEvent(g_plan.aux, g_plan.ev_nodes, 0)) != cudaSuccess) break;
            if ((e = launch_membrane_batch(g_plan.aux)) != cudaSuccess) break;
            if ((e = cudaEventRecord(g_plan.ev_membrane, g_plan.aux)) != cudaSuccess) break;
        }
        {
            const int2 *g = fl;
            const int *n = g_plan.n_flp;
            const SimDev *ds = g_plan.d_sims;
            const long long *dt = g_plan.d_t;
            // prefetch distances as in the single-simulation launches
            const int p1 = g_plan.pf_cell, p2 = g_plan.pf_pair;
            if (n[0]) k_batch_fluid<float, false><<<n[0], FLUID_THREADS, 0, st>>>(ds, dt, off, g, p1);
            g += n[0];
            if (n[1]) k_batch_fluid<float, true><<<n[1], FLUID_THREADS, 0, st>>>(ds, dt, off, g, p1);
            g += n[1];
            if (n[2]) k_batch_fluid<__half, false><<<n[2], FLUID_THREADS, 0, st>>>(ds, dt, off, g, p1);
            g += n[2];
            if (n[3]) k_batch_fluid<__half, true><<<n[3], FLUID_THREADS, 0, st>>>(ds, dt, off, g, p1);
            g += n[3];
            if (n[4]) k_batch_fluid<__nv_bfloat16, false><<<n[4], FLUID_THREADS, 0, st>>>(ds, dt, off, g, p1);
            g += n[4];
            if (n[5]) k_batch_fluid<__nv_bfloat16, true><<<n[5], FLUID_THREADS, 0, st>>>(ds, dt, off, g, p1);
            g += n[5];
            if (n[6]) k_batch_fluid_pair<__half><<<n[6], FLUID_THREADS, 0, st>>>(ds, dt, off, g, p2);
            g += n[6];
            if (n[7]) k_batch_fluid_pair<__nv_bfloat16><<<n[7], FLUID_THREADS, 0, st>>>(ds, dt, off, g, p2);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if (g_plan.n_nd) e = cudaStreamWaitEvent(st, g_plan.ev_membrane, 0);
    }
    return e;
}

// Captures LBIB_BATCH_GRAPH_STEPS steps and the advance of the counters
// (on the plan's graph stream).
static cudaError_t capture_graph(cudaStream_t st) {
    g_plan.release_graph();
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t e2 = enqueue_steps(st, 0, LBIB_BATCH_GRAPH_STEPS);
    if (e2 == cudaSuccess) {
        const int n = (int)g_plan.sims.size();
        k_batch_advance<<<(n + 127) / 128, 128, 0, st>>>(g_plan.d_t, n, LBIB_BATCH_GRAPH_STEPS);
        e2 = cudaGetLastError();
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (e2 != cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g_plan.graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    return e;
}

}  // namespace lbib

using namespace lbib;

extern "C" lbib_status lbib_batch_step(lbib_sim *const *sims, int n, int n_steps) {
    if (!sims || n <= 0 || n_steps < 0) return LBIB_ERR_ARG;
    std::lock_guard<std::mutex> plan_lock(g_plan_mu);
    for (int i = 0; i < n; ++i) {
        if (!sims[i]) return LBIB_ERR_ARG;
        if (sims[i]->sticky != LBIB_OK) return sims[i]->sticky;
        if (sims[i]->device != sims[0]->device) return LBIB_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (sims[j] == sims[i]) return LBIB_ERR_ARG;
    }
    if (cudaSetDevice(sims[0]->device) != cudaSuccess) return LBIB_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        lbib_status r = sim_prepare_step(sims[i]);
        if (r != LBIB_OK) return r;
    }
    cudaStream_t st = sims[0]->stream;
    // other simulations' pending work (uploads, refreshes, their own second
    // streams) must be done
    for (int i = 0; i < n; ++i) {
        if (sims[i]->stream != st && cudaStreamSynchronize(sims[i]->stream) != cudaSuccess) return LBIB_ERR_CUDA;
        if (cudaStreamSynchronize(sims[i]->aux) != cudaSuccess) return LBIB_ERR_CUDA;
        if (cudaStreamSynchronize(sims[i]->side) != cudaSuccess) return LBIB_ERR_CUDA;
    }
    cudaError_t e = cudaSuccess;
    const int cluster = sims[0]->cluster;
    if (!plan_matches(sims, n, cluster)) e = build_plan(sims, n, cluster, st);
    if (g_plan.mthreads != sims[0]->membrane_threads || g_plan.mgroup != sims[0]->membrane_group) {
        g_plan.mthreads = sims[0]->membrane_threads;  // captured in the graph
        g_plan.mgroup = sims[0]->membrane_group;
        g_plan.release_graph();
    }
    // descriptors (node arrays may have been reallocated, tables uploaded)
    // and the step counters of this call
    std::vector<long long> tb(n);
    for (int i = 0; i < n; ++i) tb[i] = (long long)sims[i]->t;
    bool same_dev = (int)g_plan.dev.size() == n;
    for (int i = 0; i < n && same_dev; ++i) same_dev = std::memcmp(&g_plan.dev[i], &sims[i]->d, sizeof(SimDev)) == 0;
    if (e == cudaSuccess && !same_dev) {
        // the batched kernels read the descriptors from the device copy, but
        // the repulsion launches of a captured graph hold them by value: a
        // changed descriptor (repulsion switched or retuned, node arrays
        // reallocated) needs a new graph
        g_plan.release_graph();
        g_plan.dev.resize(n);
        for (int i = 0; i < n; ++i) g_plan.dev[i] = sims[i]->d;
        e = cudaMemcpyAsync(g_plan.d_sims, g_plan.dev.data(), n * sizeof(SimDev), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_plan.d_t, tb.data(), n * sizeof(long long), cudaMemcpyHostToDevice, st);
    // membrane forces of the current positions where they are not ready
    bool need_membrane = false;
    for (int i = 0; i < n; ++i) need_membrane |= !sims[i]->objs.empty() && !sims[i]->fel_valid;
    if (e == cudaSuccess && need_membrane && n_steps > 0) e = launch_membrane_batch(st);

    int done = 0;
    while (e == cudaSuccess && done < n_steps) {
        for (int i = 0; i < n && e == cudaSuccess; ++i)
            if (sims[i]->since_mark >= ACTIVE_RESET_STEPS) e = sim_remark(sims[i], st);
        if (e != cudaSuccess) break;
        const int left = n_steps - done;
        const int k = left >= LBIB_BATCH_GRAPH_STEPS ? LBIB_BATCH_GRAPH_STEPS : left;
        if (k == LBIB_BATCH_GRAPH_STEPS) {
            // the graph advances the device counters by its own step count;
            // it runs on the graph stream, ordered after and before `st`
            if (!g_plan.graph) e = capture_graph(g_plan.gst);
            if (e == cudaSuccess) e = cudaEventRecord(g_plan.ev_join, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(g_plan.gst, g_plan.ev_join, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(g_plan.graph, g_plan.gst);
            if (e == cudaSuccess) e = cudaEventRecord(g_plan.ev_join, g_plan.gst);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g_plan.ev_join, 0);
        } else {
            e = enqueue_steps(st, 0, k);
        }
        for (int i = 0; i < n; ++i) sims[i]->since_mark += k;
        done += k;
    }
    // host copies of the descriptors and counters must outlive the copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_plan.release();
        for (int i = 0; i < n; ++i) {
            sims[i]->sticky = LBIB_ERR_CUDA;
            sims[i]->err = std::string("batch step: ") + cudaGetErrorString(e);
        }
        return LBIB_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i) {
        lbib_sim *s = sims[i];
        if (n_steps > 0) {
            s->gmode = (int)((s->t + n_steps - 1) & 1);
            s->t += n_steps;
            if (s->nn_total > 0) {
                s->dev_newer = true;
                s->fel_valid = true;  // the last membrane pass used the final positions
                s->side_ok = false;   // the batch ran on its own streams
            }
        }
    }
    return LBIB_OK;
}
