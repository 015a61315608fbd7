// Batched step: many independent simulations advanced by one persistent
// launch per step.
//
// The grid is made of thread-block clusters (as many as fit on the GPU at
// once).  Phase A: each cluster takes objects, of any simulation, from an
// atomic ticket (rank 0 draws it and the cluster reads it through
// distributed shared memory) and updates them as in ib_core.cuh (membrane
// part, then the coupling part of the object's nodes by the same cluster).  Phase B:
// once the objects are handed out, every block takes blocks of
// FLUID_THREADS fluid cells, of any simulation, from a second ticket.  A warp
// whose 32 cells include active cells (cells near objects, see
// lbib_internal.h) first waits until all of its simulation's objects are
// done; the other warps need nothing from this step's object update and run
// while it is still in progress.
// Every object was handed out to a running cluster before any block reached
// phase B, and objects never wait, so every wait ends; it is nevertheless
// bounded, and on expiry the block flags the simulation (ST_TIMEOUT,
// surfaced as LBIB_ERR_TIMEOUT) instead of spinning on.
//
// A simulation advanced inside a batch computes what lbib_step computes for
// it alone: the per-item code is the same device code; only the order of the
// FP32 vector atomics of the spreading may differ, as between two runs of
// the single-simulation path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fluid_core.cuh"
#include "ib_core.cuh"
#include "sim.h"

namespace lbib {

constexpr unsigned BATCH_WAIT_SPINS = 1u << 24;  // x ~64 ns: about one second

extern __shared__ float batch_smem[];

// ib_items: (simulation, object); fl_items: (simulation, block of cells).
// counters[0]: object ticket; counters[1]: fluid ticket; counters[2 + s]:
// finished objects of simulation s; need[s]: objects of s.
__global__ void __launch_bounds__(FLUID_THREADS) k_batch_step(const SimDev *__restrict__ sims,
                                                              const int *__restrict__ par_base,
                                                              const long long *__restrict__ t_base, int step_off,
                                                              const int2 *__restrict__ ib_items, int n_ib,
                                                              const int2 *__restrict__ fl_items, int n_fl,
                                                              const int *__restrict__ need, unsigned *counters) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ int s_item;
    for (;;) {  // phase A: one object per cluster
        if (cl.block_rank() == 0 && threadIdx.x == 0) s_item = (int)atomicAdd(counters, 1u);
        cl.sync();
        const int k = *cl.map_shared_rank(&s_item, 0);
        cl.sync();  // every block has read the ticket before rank 0 draws again
        if (k >= n_ib) break;
        const int2 it = ib_items[k];
        const SimDev &s = sims[it.x];
        const int par = (par_base[it.x] + step_off) & 1;
        membrane_object(s, it.y, batch_smem);
        // the object's nodes: coupling and update (membrane forces visible
        // after the cluster barrier that ends membrane_object)
        {
            const ObjDev ob = s.obj[it.y];
            const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
            for (int p = share_lo(ob.nn, r, C) + threadIdx.x; p < share_lo(ob.nn, r + 1, C); p += blockDim.x)
                node_step(s, ob.first + p, par);
        }
        __syncthreads();
        if (threadIdx.x == 0) __threadfence();  // this block's node updates, device-wide
        cl.sync();
        if (cl.block_rank() == 0 && threadIdx.x == 0) atomicAdd(counters + 2 + it.x, 1u);
    }
    for (;;) {  // phase B: blocks of fluid cells
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counters + 1, 1u);
        __syncthreads();
        const int k = s_item;
        __syncthreads();
        if (k >= n_fl) break;
        const int2 it = fl_items[k];
        const SimDev &s = sims[it.x];
        const int par = (par_base[it.x] + step_off) & 1;
        const int f = it.y * FLUID_THREADS + (int)threadIdx.x;
        const uint32_t act = active_word(s, f);  // warp-uniform
        if (act) {
            // cells near objects need this step's spread force: wait for the
            // simulation's objects (warps without such cells go ahead)
            if ((threadIdx.x & 31) == 0) {
                const volatile unsigned *done = counters + 2 + it.x;
                const unsigned want = (unsigned)need[it.x];
                unsigned spins = 0;
                while (*done < want) {
                    __nanosleep(64);
                    if (++spins > BATCH_WAIT_SPINS) {
                        atomicOr(s.status, ST_TIMEOUT);
                        break;
                    }
                }
                __threadfence();
            }
            __syncwarp();
        }
        if (f < s.nf) {
            const uint32_t seed = step_seed(t_base[it.x] + step_off);
            const bool a = (act >> (threadIdx.x & 31)) & 1u;
            switch (s.prec) {
                case LBIB_POP_F32: fluid_cell<float>(s, par, f, a, seed); break;
                case LBIB_POP_F16S: fluid_cell<__half>(s, par, f, a, seed); break;
                default: fluid_cell<__nv_bfloat16>(s, par, f, a, seed); break;
            }
        }
    }
}

// A batch plan: device copies of the descriptors and the item lists,
// rebuilt whenever the set of simulations or their objects change.
struct BatchPlan {
    std::vector<lbib_sim *> sims;
    std::vector<int> nobj;
    SimDev *d_sims = nullptr;
    int *d_par = nullptr;
    long long *d_t = nullptr;
    int2 *d_items = nullptr;
    int *d_need = nullptr;
    unsigned *d_counters = nullptr;
    int n_ib = 0, n_fl = 0, cluster = 4, grid = 0;
    size_t smem = 0;

    void release() {
        cudaFree(d_sims);
        cudaFree(d_par);
        cudaFree(d_t);
        cudaFree(d_items);
        cudaFree(d_need);
        cudaFree(d_counters);
        d_sims = nullptr;
        d_par = nullptr;
        d_t = nullptr;
        d_items = nullptr;
        d_need = nullptr;
        d_counters = nullptr;
        sims.clear();
        nobj.clear();
    }
};

static BatchPlan g_plan;

static bool plan_matches(lbib_sim *const *sims, int n, int cluster) {
    if ((int)g_plan.sims.size() != n || g_plan.cluster != cluster) return false;
    for (int i = 0; i < n; ++i)
        if (g_plan.sims[i] != sims[i] || g_plan.nobj[i] != (int)sims[i]->objs.size()) return false;
    return true;
}

static cudaError_t build_plan(lbib_sim *const *sims, int n, int cluster, cudaStream_t st) {
    g_plan.release();
    std::vector<SimDev> dev(n);
    std::vector<int2> ib, fl;
    std::vector<int> need(n);
    int max_nodes = 0;
    for (int i = 0; i < n; ++i) {
        dev[i] = sims[i]->d;
        need[i] = (int)sims[i]->objs.size();
        max_nodes = std::max(max_nodes, sims[i]->max_nodes);
        for (int o = 0; o < need[i]; ++o) ib.push_back(make_int2(i, o));
        const int blocks = (dev[i].nf + FLUID_THREADS - 1) / FLUID_THREADS;
        for (int b = 0; b < blocks; ++b) fl.push_back(make_int2(i, b));
    }
    std::vector<int2> items(ib);
    items.insert(items.end(), fl.begin(), fl.end());
    cudaError_t e;
    if ((e = cudaMalloc(&g_plan.d_sims, n * sizeof(SimDev))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_par, n * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_t, n * sizeof(long long))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_items, std::max<size_t>(1, items.size()) * sizeof(int2))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_need, n * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_counters, (n + 2) * sizeof(unsigned))) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(g_plan.d_sims, dev.data(), n * sizeof(SimDev), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
    if (!items.empty() &&
        (e = cudaMemcpyAsync(g_plan.d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(g_plan.d_need, need.data(), n * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    g_plan.sims.assign(sims, sims + n);
    for (int i = 0; i < n; ++i) g_plan.nobj.push_back((int)sims[i]->objs.size());
    g_plan.n_ib = (int)ib.size();
    g_plan.n_fl = (int)fl.size();
    g_plan.cluster = cluster;
    g_plan.smem = ib_smem_bytes(max_nodes);
    if ((e = cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_plan.smem)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
        return e;
    // as many clusters as can be resident at once (a persistent grid)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster);
    cfg.blockDim = dim3(FLUID_THREADS);
    cfg.dynamicSmemBytes = g_plan.smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    if ((e = cudaOccupancyMaxActiveClusters(&clusters, k_batch_step, &cfg)) != cudaSuccess) return e;
    g_plan.grid = std::max(1, clusters) * cluster;
    return cudaSuccess;
}

}  // namespace lbib

using namespace lbib;

extern "C" lbib_status lbib_batch_step(lbib_sim *const *sims, int n, int n_steps) {
    if (!sims || n <= 0 || n_steps < 0) return LBIB_ERR_ARG;
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
    // other simulations' pending work (uploads, refreshes) must be done
    for (int i = 1; i < n; ++i)
        if (sims[i]->stream != st && cudaStreamSynchronize(sims[i]->stream) != cudaSuccess) return LBIB_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    const int cluster = sims[0]->cluster;
    if (!plan_matches(sims, n, cluster)) {
        e = build_plan(sims, n, cluster, st);
        if (e != cudaSuccess) {
            sims[0]->err = std::string("batch plan: ") + cudaGetErrorString(e);
            return LBIB_ERR_CUDA;
        }
    } else {
        // descriptors may have changed (node arrays reallocated, tables re-uploaded)
        std::vector<SimDev> dev(n);
        for (int i = 0; i < n; ++i) dev[i] = sims[i]->d;
        e = cudaMemcpyAsync(g_plan.d_sims, dev.data(), n * sizeof(SimDev), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    std::vector<int> par(n);
    std::vector<long long> tb(n);
    for (int i = 0; i < n; ++i) {
        par[i] = (int)(sims[i]->t & 1);
        tb[i] = (long long)sims[i]->t;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_plan.d_par, par.data(), n * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_plan.d_t, tb.data(), n * sizeof(long long), cudaMemcpyHostToDevice, st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g_plan.grid);
    cfg.blockDim = dim3(FLUID_THREADS);
    cfg.dynamicSmemBytes = g_plan.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const int2 *fl_items = g_plan.d_items + g_plan.n_ib;
    for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
        for (int i = 0; i < n && e == cudaSuccess; ++i) {
            if (sims[i]->since_mark >= ACTIVE_RESET_STEPS) e = sim_remark(sims[i], st);
            sims[i]->since_mark++;
        }
        if (e != cudaSuccess) break;
        e = cudaMemsetAsync(g_plan.d_counters, 0, (n + 2) * sizeof(unsigned), st);
        if (e != cudaSuccess) break;
        e = cudaLaunchKernelEx(&cfg, k_batch_step, (const SimDev *)g_plan.d_sims, (const int *)g_plan.d_par,
                               (const long long *)g_plan.d_t, k, (const int2 *)g_plan.d_items, g_plan.n_ib, fl_items,
                               g_plan.n_fl, (const int *)g_plan.d_need, g_plan.d_counters);
    }
    // host copies of par/dev must outlive the async copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        for (int i = 0; i < n; ++i) {
            sims[i]->sticky = LBIB_ERR_CUDA;
            sims[i]->err = std::string("batch step: ") + cudaGetErrorString(e);
        }
        return LBIB_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i) {
        lbib_sim *s = sims[i];
        for (int k = 0; k < n_steps; ++k) {
            s->gmode = (int)(s->t & 1);
            s->t++;
        }
        if (n_steps > 0 && s->nn_total > 0) {
            s->dev_newer = true;
            s->fel_valid = false;  // membrane forces are those of the last step, not the next
        }
    }
    return LBIB_OK;
}
