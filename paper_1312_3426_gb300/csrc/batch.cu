// Batched step: many independent simulations advanced by one persistent
// launch per step.
//
// The work of one step is a list of items: first one item per object of
// every simulation (the immersed-boundary update of that object), then one
// item per block of FLUID_THREADS fluid cells of every simulation.  A
// persistent grid (a few blocks per SM) takes items in list order from an
// atomic ticket.  A fluid item of simulation s must see all of s's spread
// forces, so it waits until s's object counter reaches its object count.
// Every object item was handed out before any fluid item (ticket order) and
// object items never wait, so the wait always ends; it is nevertheless
// bounded, and on expiry the block flags the simulation (ST_TIMEOUT, surfaced
// as LBIB_ERR_TIMEOUT) instead of spinning on.
//
// A simulation advanced inside a batch computes exactly what lbib_step would
// compute for it alone: the per-item code is the same device code, only the
// scheduling differs (the floating-point order of the vector atomics of the
// spreading is the one freedom, as in the single-simulation path).
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

// counters[0]: ticket; counters[1 + s]: finished object items of simulation s.
__global__ void __launch_bounds__(FLUID_THREADS) k_batch_step(const SimDev *__restrict__ sims,
                                                              const int *__restrict__ par_base, int step_off,
                                                              const int2 *__restrict__ items, int n_ib,
                                                              int n_items, const int *__restrict__ ib_need,
                                                              unsigned *counters) {
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counters, 1u);
        __syncthreads();
        const int k = s_item;
        __syncthreads();
        if (k >= n_items) break;
        const int2 it = items[k];
        const SimDev s = sims[it.x];
        const int par = (par_base[it.x] + step_off) & 1;
        if (k < n_ib) {
            ib_object(s, it.y, par, batch_smem);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(counters + 1 + it.x, 1u);
            }
        } else {
            if (threadIdx.x == 0) {
                const unsigned need = (unsigned)ib_need[it.x];
                const volatile unsigned *done = counters + 1 + it.x;
                unsigned spins = 0;
                while (*done < need) {
                    __nanosleep(64);
                    if (++spins > BATCH_WAIT_SPINS) {
                        atomicOr(s.status, ST_TIMEOUT);
                        break;
                    }
                }
                __threadfence();
            }
            __syncthreads();
            const int f0 = it.y * FLUID_THREADS;
            switch (s.prec) {
                case LBIB_POP_F32: fluid_block<float>(s, par, f0); break;
                case LBIB_POP_F16S: fluid_block<__half>(s, par, f0); break;
                default: fluid_block<__nv_bfloat16>(s, par, f0); break;
            }
        }
    }
}

// A batch plan: device copies of the descriptors and the item list, rebuilt
// whenever the set of simulations or their object counts change.
struct BatchPlan {
    std::vector<lbib_sim *> sims;
    std::vector<int> nobj;
    SimDev *d_sims = nullptr;
    int *d_par = nullptr;
    int2 *d_items = nullptr;
    int *d_need = nullptr;
    unsigned *d_counters = nullptr;
    int n_ib = 0, n_items = 0, max_nodes = 0, grid = 0;
    size_t smem = 0;

    void release() {
        cudaFree(d_sims);
        cudaFree(d_par);
        cudaFree(d_items);
        cudaFree(d_need);
        cudaFree(d_counters);
        d_sims = nullptr;
        d_par = nullptr;
        d_items = nullptr;
        d_need = nullptr;
        d_counters = nullptr;
        sims.clear();
        nobj.clear();
    }
};

static BatchPlan g_plan;

static bool plan_matches(lbib_sim *const *sims, int n) {
    if ((int)g_plan.sims.size() != n) return false;
    for (int i = 0; i < n; ++i)
        if (g_plan.sims[i] != sims[i] || g_plan.nobj[i] != (int)sims[i]->objs.size()) return false;
    return true;
}

static cudaError_t build_plan(lbib_sim *const *sims, int n, cudaStream_t st) {
    g_plan.release();
    std::vector<SimDev> dev(n);
    std::vector<int2> items;
    std::vector<int> need(n);
    int max_nodes = 0;
    for (int i = 0; i < n; ++i) {
        dev[i] = sims[i]->d;
        need[i] = (int)sims[i]->objs.size();
        max_nodes = std::max(max_nodes, sims[i]->max_nodes);
        for (int o = 0; o < need[i]; ++o) items.push_back(make_int2(i, o));
    }
    const int n_ib = (int)items.size();
    for (int i = 0; i < n; ++i) {
        const int blocks = (dev[i].nf + FLUID_THREADS - 1) / FLUID_THREADS;
        for (int b = 0; b < blocks; ++b) items.push_back(make_int2(i, b));
    }
    cudaError_t e;
    if ((e = cudaMalloc(&g_plan.d_sims, n * sizeof(SimDev))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_par, n * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_items, std::max<size_t>(1, items.size()) * sizeof(int2))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_need, n * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&g_plan.d_counters, (n + 1) * sizeof(unsigned))) != cudaSuccess) return e;
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
    g_plan.n_ib = n_ib;
    g_plan.n_items = (int)items.size();
    g_plan.max_nodes = max_nodes;
    g_plan.smem = (size_t)IB_SMEM_PER_NODE * max_nodes;
    const int smem_attr = std::max<int>((int)g_plan.smem, 48 * 1024);
    if ((e = cudaFuncSetAttribute(k_batch_step, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_attr)) != cudaSuccess)
        return e;
    int dev_id = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev_id);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step, FLUID_THREADS, g_plan.smem)) !=
        cudaSuccess)
        return e;
    g_plan.grid = std::max(1, sms * std::max(1, per_sm));
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
    if (!plan_matches(sims, n)) {
        e = build_plan(sims, n, st);
        if (e != cudaSuccess) {
            sims[0]->err = std::string("batch plan: ") + cudaGetErrorString(e);
            return LBIB_ERR_CUDA;
        }
    } else {
        // descriptors may have changed (node arrays reallocated, tables re-uploaded)
        std::vector<SimDev> dev(n);
        for (int i = 0; i < n; ++i) dev[i] = sims[i]->d;
        e = cudaMemcpyAsync(g_plan.d_sims, dev.data(), n * sizeof(SimDev), cudaMemcpyHostToDevice, st);
    }
    std::vector<int> par(n);
    for (int i = 0; i < n; ++i) par[i] = (int)(sims[i]->t & 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g_plan.d_par, par.data(), n * sizeof(int), cudaMemcpyHostToDevice, st);
    for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
        e = cudaMemsetAsync(g_plan.d_counters, 0, (n + 1) * sizeof(unsigned), st);
        if (e != cudaSuccess) break;
        k_batch_step<<<g_plan.grid, FLUID_THREADS, g_plan.smem, st>>>(g_plan.d_sims, g_plan.d_par, k, g_plan.d_items,
                                                                      g_plan.n_ib, g_plan.n_items, g_plan.d_need,
                                                                      g_plan.d_counters);
        e = cudaGetLastError();
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
        if (n_steps > 0 && s->nn_total > 0) s->dev_newer = true;
    }
    return LBIB_OK;
}
