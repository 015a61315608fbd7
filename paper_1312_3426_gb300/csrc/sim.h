// Host-side state of one simulation (the opaque lbib_sim of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "lbib.h"
#include "lbib_internal.h"
#include "topology.h"

struct lbib_sim {
    lbib_fluid_params p{};
    uint64_t serial = 0;         // unique per simulation of the process (an address may be reused)
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    lbib_status sticky = LBIB_OK;

    lbib::SimDev d{};            // device descriptor handed to kernels
    void *fluid_mem = nullptr;   // populations, coupling fields, masks, status
    size_t fluid_bytes = 0;

    std::vector<lbib::Topology> topo;   // host copy of every template
    std::vector<lbib::TplDev> tpl_dev;  // device descriptors of the templates
    std::vector<void *> tpl_mem;        // device records of every template
    size_t tpl_bytes = 0;
    int max_nodes = 0;                  // largest template

    std::vector<lbib::ObjDev> objs;
    int nn_total = 0;
    std::vector<double> hX, hV;  // host mirror of node state, [nn][3]
    bool host_newer = false;     // host mirror changed since the last upload
    bool dev_newer = false;      // device state advanced since the last download
    bool tables_dirty = false;   // object/template tables need an upload
    float *dnodes = nullptr;     // Xh, Xl, Vh, Vl, Fel, each [3][nn_total], then node_obj [nn_total]
    int dev_nn_cap = 0;
    size_t node_bytes = 0;
    lbib::ObjDev *d_obj = nullptr;
    lbib::TplDev *d_tpl = nullptr;
    std::vector<float> fext;     // [nobj][3]
    float *fext_pinned = nullptr;      // page-locked staging of fext for asynchronous uploads
    size_t fext_pinned_cap = 0;
    cudaEvent_t ev_fext = nullptr;     // the last upload out of the staging buffer
    uint32_t *status_pinned = nullptr; // page-locked copy of the device status word
    std::vector<double> masses;
    float *d_fext = nullptr;
    int cluster = 1;             // thread blocks per object in the membrane kernel
    bool fext_dirty = false;
    double *d_analyze = nullptr; // [nobj][14] read-out buffer
    // asynchronous analysis: two page-locked slots of [nobj][14] doubles
    // followed by the status word, each with its event
    double *ana_pinned[2] = {nullptr, nullptr};
    int ana_cap[2] = {0, 0};
    int ana_nobj[2] = {0, 0};
    bool ana_pending[2] = {false, false};
    cudaEvent_t ana_ev[2] = {nullptr, nullptr};
    int d_obj_cap = 0;

    // The membrane part of step t+1 runs on a second stream while the fluid
    // part of step t runs on `stream`; events order the two.
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_nodes = nullptr;     // node update of the current step done
    cudaEvent_t ev_membrane = nullptr;  // membrane forces of the next step ready
    bool fel_valid = false;             // Fel holds the membrane forces of the current node positions
    // The last step recorded ev_nodes after its node update and nothing has
    // changed node state or tables since: the per-step object-force upload
    // and analysis may run on `side` (after ev_nodes) beside the fluid and
    // membrane kernels
    bool side_ok = false;
    cudaStream_t side = nullptr;
    bool overlap = true;                // membrane of step t+1 on `aux` during fluid of step t
    int membrane_clusters = 0;          // clusters of the membrane kernel (0: one per object)
    int membrane_threads = 192;         // block size of the membrane kernel (per object)
    int membrane_group = 1;             // objects per block of the membrane kernel
    bool early_launch = false;          // programmatic dependent launch of the node and fluid kernels
    int node_threads = lbib::IB_THREADS_DEFAULT;  // nodes per block of the node kernel

    double rep_obj[3] = {0, 1, 0};      // soft-sphere repulsion (a, n, cutoff) between objects
    double rep_wall[3] = {0, 1, 0};     // and against the walls
    uint32_t *solid_mem = nullptr;      // obstacle bits (one per fluid cell)
    void *rep_mem = nullptr;            // object boxes, pair list, pair count
    int rep_cap_obj = 0;                // objects the buffers hold
    size_t rep_bytes = 0;

    bool prof_on = false;        // per-phase CUDA-event timing
    int prof_every = 1;          // ... of every prof_every-th step
    bool prof_now = false;       // the step being enqueued is timed
    std::vector<cudaEvent_t> prof_ev;   // 3 per step on `stream`
    std::vector<cudaEvent_t> prof_aux;  // 2 per membrane launch on `aux`
    size_t prof_used = 0, prof_aux_used = 0;

    bool fluid_ready = false;
    int64_t t = 0;               // steps since lbib_fluid_init (buffer parity)
    int gmode = -1;              // force applied by the collision that produced the current populations
    bool ufield_stale = false;   // velocity samples must be recomputed before the next step
    bool mark_stale = true;      // the active-cell mask must be rebuilt before the next step
    int since_mark = 0;          // steps since the active-cell mask was rebuilt
};

namespace lbib {
lbib_status sim_check_status(lbib_sim *s);
lbib_status sim_download_nodes(lbib_sim *s);
lbib_status sim_upload(lbib_sim *s);
lbib_status sim_prepare_step(lbib_sim *s);
cudaError_t sim_remark(lbib_sim *s, cudaStream_t st);
}  // namespace lbib
