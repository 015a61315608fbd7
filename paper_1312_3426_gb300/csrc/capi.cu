// C ABI of the library (declared in include/lbib.h): simulation objects,
// templates, objects, host<->device transfers, step orchestration and the
// sticky error model.  Host code only; the kernels live in fluid.cu, ib.cu
// and batch.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "lbib.h"
#include "lbib_internal.h"
#include "sim.h"
#include "topology.h"

using namespace lbib;

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

size_t pop_elem_bytes(int prec) { return prec == LBIB_POP_F32 ? 4 : 2; }

struct FluidLayout {
    int nyf, nf, nfp, nwords;
    size_t off_pop[2], off_G[2], off_amask, off_ufield, off_status, off_dropped, total;
};

bool fluid_layout(const lbib_fluid_params &p, FluidLayout &L) {
    L.nyf = p.walls_y ? p.ny - 2 : p.ny;
    const int64_t nf = (int64_t)p.nx * L.nyf * p.nz;
    if (nf <= 0 || nf >= (int64_t)1 << 31) return false;
    L.nf = (int)nf;
    L.nfp = (int)align_up((size_t)nf, 64);
    if ((int64_t)NQ * L.nfp >= ((int64_t)1 << 32)) return false;  // 32-bit population indices
    L.nwords = (L.nf + 31) / 32;
    size_t o = 0;
    const size_t popb = (size_t)NQ * L.nfp * pop_elem_bytes(p.precision);
    for (int k = 0; k < 2; ++k) { L.off_pop[k] = o; o = align_up(o + popb, 256); }
    for (int k = 0; k < 2; ++k) { L.off_G[k] = o; o = align_up(o + (size_t)L.nf * 16, 256); }
    L.off_amask = o; o = align_up(o + (size_t)L.nwords * 4, 256);
    L.off_ufield = o; o = align_up(o + (size_t)L.nf * 16, 256);
    L.off_status = o; o = align_up(o + 4, 256);
    L.off_dropped = o; o = align_up(o + 24, 256);
    L.total = o;
    return true;
}

// device records of a template: triangles (int4), and per edge its hinge
// nodes (int4) and constants (float4)
size_t template_bytes(const Topology &T) {
    return align_up((size_t)T.nt * 16, 256) + 2 * align_up((size_t)T.ne * 16, 256);
}

lbib_status fail(lbib_sim *s, lbib_status code, const std::string &msg) {
    if (s) s->err = msg;
    return code;
}

lbib_status cuda_fail(lbib_sim *s, cudaError_t e, const char *where) {
    const lbib_status code = (e == cudaErrorMemoryAllocation) ? LBIB_ERR_NOMEM : LBIB_ERR_CUDA;
    if (s) {
        s->err = std::string(where) + ": " + cudaGetErrorString(e);
        if (code == LBIB_ERR_CUDA) s->sticky = code;
    }
    return code;
}

#define LBIB_CUDA(s, call, where)                   \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail((s), e_, (where)); \
    } while (0)

#define LBIB_GUARD(s)                                                      \
    do {                                                                   \
        if (!(s)) return LBIB_ERR_ARG;                                     \
        if ((s)->sticky != LBIB_OK) return (s)->sticky;                    \
        if (cudaSetDevice((s)->device) != cudaSuccess) return LBIB_ERR_CUDA; \
    } while (0)

void rotation_zyx(const double r[3], double R[3][3]) {
    const double cx = std::cos(r[0]), sx = std::sin(r[0]), cy = std::cos(r[1]), sy = std::sin(r[1]),
                 cz = std::cos(r[2]), sz = std::sin(r[2]);
    // R = Rz * Ry * Rx
    R[0][0] = cz * cy;
    R[0][1] = cz * sy * sx - sz * cx;
    R[0][2] = cz * sy * cx + sz * sx;
    R[1][0] = sz * cy;
    R[1][1] = sz * sy * sx + cz * cx;
    R[1][2] = sz * sy * cx - cz * sx;
    R[2][0] = -sy;
    R[2][1] = cy * sx;
    R[2][2] = cy * cx;
}

}  // namespace

namespace lbib {

// Status word -> sticky error.
static lbib_status apply_status(lbib_sim *s, uint32_t st) {
    if (st & ST_TIMEOUT) {
        s->sticky = LBIB_ERR_TIMEOUT;
        s->err = "a bounded device-side wait gave up";
    } else if (st & ST_PAIRS) {
        s->sticky = LBIB_ERR_NOMEM;
        s->err = "more close object pairs than the repulsion pair list holds";
    } else if (st & (ST_UNSTABLE | ST_NODE_NAN)) {
        s->sticky = LBIB_ERR_UNSTABLE;
        s->err = (st & ST_UNSTABLE) ? "fluid became unstable (NaN or |u| > 0.3)" : "a node position became non-finite";
    }
    return s->sticky;
}

// Waits for the stream and folds the device status word into the sticky error.
lbib_status sim_check_status(lbib_sim *s) {
    cudaError_t e = cudaMemcpyAsync(s->status_pinned, s->d.status, 4, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stream");
    return apply_status(s, *s->status_pinned);
}

lbib_status sim_download_nodes(lbib_sim *s) {
    if (!s->dev_newer) return LBIB_OK;
    const int nn = s->nn_total;
    std::vector<float> st(12 * (size_t)nn);  // Xh, Xl, Vh, Vl, each [3][nn]
    LBIB_CUDA(s, cudaMemcpyAsync(st.data(), s->dnodes, st.size() * 4, cudaMemcpyDeviceToHost, s->stream), "nodes D2H");
    LBIB_CUDA(s, cudaStreamSynchronize(s->stream), "nodes D2H");
    const size_t n3 = 3 * (size_t)nn;
    for (int i = 0; i < nn; ++i)
        for (int k = 0; k < 3; ++k) {
            const size_t j = (size_t)k * nn + i;
            s->hX[3 * (size_t)i + k] = (double)st[j] + (double)st[n3 + j];
            s->hV[3 * (size_t)i + k] = (double)st[2 * n3 + j] + (double)st[3 * n3 + j];
        }
    s->dev_newer = false;
    return LBIB_OK;
}

lbib_status sim_upload(lbib_sim *s) {
    if (s->tables_dirty || s->host_newer) s->side_ok = false;
    if (s->tables_dirty) {
        if (!s->tpl_dev.empty()) {
            if (s->d_tpl) cudaFree(s->d_tpl);
            s->d_tpl = nullptr;
            LBIB_CUDA(s, cudaMalloc(&s->d_tpl, s->tpl_dev.size() * sizeof(TplDev)), "template table");
            LBIB_CUDA(s, cudaMemcpyAsync(s->d_tpl, s->tpl_dev.data(), s->tpl_dev.size() * sizeof(TplDev),
                                         cudaMemcpyHostToDevice, s->stream), "template table");
        }
        const int nobj = (int)s->objs.size();
        if (nobj > s->d_obj_cap) {
            const int cap = std::max(nobj, 2 * s->d_obj_cap);
            cudaFree(s->d_obj);
            cudaFree(s->d_fext);
            cudaFree(s->d_analyze);
            s->d_obj = nullptr;
            s->d_fext = nullptr;
            s->d_analyze = nullptr;
            s->d_obj_cap = 0;
            LBIB_CUDA(s, cudaMalloc(&s->d_obj, cap * sizeof(ObjDev)), "object table");
            LBIB_CUDA(s, cudaMalloc(&s->d_fext, cap * 3 * sizeof(float)), "object forces");
            LBIB_CUDA(s, cudaMalloc(&s->d_analyze, cap * 14 * sizeof(double)), "analysis buffer");
            s->d_obj_cap = cap;
            s->fext_dirty = true;
        }
        if (nobj > 0)
            LBIB_CUDA(s, cudaMemcpyAsync(s->d_obj, s->objs.data(), nobj * sizeof(ObjDev), cudaMemcpyHostToDevice,
                                         s->stream), "object table");
        LBIB_CUDA(s, cudaStreamSynchronize(s->stream), "tables");
        s->d.tpl = s->d_tpl;
        s->d.obj = s->d_obj;
        s->d.fext = s->d_fext;
        s->d.nobj = nobj;
        // repulsion buffers: boxes [nobj][8], a pair list of 32 per object
        const bool rep = s->rep_obj[0] > 0.0 && s->rep_obj[2] > 0.0 && nobj >= 2;
        if (rep && nobj > s->rep_cap_obj) {
            const int cap_obj = std::max(nobj, 2 * s->rep_cap_obj);
            if (s->rep_mem) cudaFree(s->rep_mem);
            s->rep_mem = nullptr;
            s->rep_cap_obj = 0;
            s->rep_bytes = 0;
            const size_t pairs = 32 * (size_t)cap_obj + 1024;
            const size_t bytes = align_up((size_t)cap_obj * 8 * sizeof(float), 256) + pairs * sizeof(int4) + 256;
            LBIB_CUDA(s, cudaMalloc(&s->rep_mem, bytes), "repulsion buffers");
            s->rep_cap_obj = cap_obj;
            s->rep_bytes = bytes;
            char *b = (char *)s->rep_mem;
            s->d.aabb = (float *)b;
            s->d.pairs = (int4 *)(b + align_up((size_t)cap_obj * 8 * sizeof(float), 256));
            s->d.npairs = (unsigned *)(b + align_up((size_t)cap_obj * 8 * sizeof(float), 256) + pairs * sizeof(int4));
            s->d.pair_cap = (int)pairs;
        }
        s->d.rep_on = rep ? 1 : 0;
        s->tables_dirty = false;
        s->fel_valid = false;
    }
    if (s->fext_dirty && !s->objs.empty()) {
        // asynchronous upload through a page-locked staging buffer; the
        // buffer is refilled only once the previous upload out of it is done.
        // After a step the copy runs on `side` (after the node update that
        // read the old forces, beside the fluid kernel) and `stream` waits
        // for it before the next node update.
        const size_t n = s->fext.size();
        const bool side = s->side_ok;
        cudaStream_t ust = side ? s->side : s->stream;
        if (side) LBIB_CUDA(s, cudaStreamWaitEvent(ust, s->ev_nodes, 0), "object forces");
        LBIB_CUDA(s, cudaEventSynchronize(s->ev_fext), "object forces");
        if (n > s->fext_pinned_cap) {
            if (s->fext_pinned) cudaFreeHost(s->fext_pinned);
            s->fext_pinned = nullptr;
            s->fext_pinned_cap = 0;
            LBIB_CUDA(s, cudaMallocHost(&s->fext_pinned, n * sizeof(float)), "object force staging");
            s->fext_pinned_cap = n;
        }
        std::memcpy(s->fext_pinned, s->fext.data(), n * sizeof(float));
        LBIB_CUDA(s, cudaMemcpyAsync(s->d_fext, s->fext_pinned, n * sizeof(float), cudaMemcpyHostToDevice, ust),
                  "object forces");
        LBIB_CUDA(s, cudaEventRecord(s->ev_fext, ust), "object forces");
        if (side) LBIB_CUDA(s, cudaStreamWaitEvent(s->stream, s->ev_fext, 0), "object forces");
        s->fext_dirty = false;
    }
    if (s->host_newer) {
        const int nn = s->nn_total;
        if (nn > s->dev_nn_cap) {
            if (s->dnodes) cudaFree(s->dnodes);
            s->dnodes = nullptr;
            s->node_bytes = 0;
            LBIB_CUDA(s, cudaMalloc(&s->dnodes, 16 * (size_t)nn * 4), "node state");
            s->dev_nn_cap = nn;
            s->node_bytes = 16 * (size_t)nn * 4;
        }
        // FP64 host values split exactly into hi + lo FP32 pairs (48 bits);
        // the membrane forces are recomputed before they are used
        std::vector<float> st(16 * (size_t)nn, 0.f);
        const size_t n3 = 3 * (size_t)nn;
        for (int i = 0; i < nn; ++i)
            for (int k = 0; k < 3; ++k) {
                const size_t j = (size_t)k * nn + i;
                const double x = s->hX[3 * (size_t)i + k], v = s->hV[3 * (size_t)i + k];
                st[j] = (float)x;
                st[n3 + j] = (float)(x - (double)st[j]);
                st[2 * n3 + j] = (float)v;
                st[3 * n3 + j] = (float)(v - (double)st[2 * n3 + j]);
            }
        int32_t *owner = (int32_t *)(st.data() + 5 * n3);
        for (int o = 0; o < (int)s->objs.size(); ++o)
            for (int p = 0; p < s->objs[o].nn; ++p) owner[s->objs[o].first + p] = o;
        LBIB_CUDA(s, cudaMemcpyAsync(s->dnodes, st.data(), st.size() * 4, cudaMemcpyHostToDevice, s->stream), "nodes H2D");
        LBIB_CUDA(s, cudaStreamSynchronize(s->stream), "nodes H2D");
        s->d.Xh = s->dnodes;
        s->d.Xl = s->dnodes + n3;
        s->d.Vh = s->dnodes + 2 * n3;
        s->d.Vl = s->dnodes + 3 * n3;
        s->d.Fel = s->dnodes + 4 * n3;
        s->d.node_obj = (const int *)(s->dnodes + 5 * n3);
        s->d.nn_total = nn;
        s->host_newer = false;
        s->fel_valid = false;
        // the velocity samples must be valid at the (new) node corners, and
        // the active cells must follow the nodes
        if (!(s->t == 0 && s->gmode == -1)) s->ufield_stale = true;
        s->mark_stale = true;
    }
    return LBIB_OK;
}

lbib_status sim_prepare_step(lbib_sim *s) {
    if (!s->fluid_ready) return fail(s, LBIB_ERR_STATE, "lbib_fluid_init must precede lbib_step");
    lbib_status r = sim_upload(s);
    if (r != LBIB_OK) return r;
    if (s->ufield_stale) {
        LBIB_CUDA(s, launch_fields(s->d, (int)(s->t & 1), s->gmode, nullptr, nullptr, 1, s->stream), "velocity samples");
        s->ufield_stale = false;
    }
    if (s->mark_stale) {
        // nodes may have moved arbitrarily: the buffer the next step clears
        // holds forces at cells that may no longer be active
        FluidLayout L;
        fluid_layout(s->p, L);
        LBIB_CUDA(s, cudaMemsetAsync((char *)s->fluid_mem + L.off_G[(s->t + 1) & 1], 0, (size_t)L.nf * 16, s->stream),
                  "coupling force");
        LBIB_CUDA(s, sim_remark(s, s->stream), "active cells");
        s->mark_stale = false;
    }
    return LBIB_OK;
}

// Clears the active-cell mask and marks the cells around every node.
cudaError_t sim_remark(lbib_sim *s, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(s->d.amask, 0, (size_t)s->d.nwords * 4, st);
    if (e == cudaSuccess) e = launch_mark_all(s->d, st);
    s->since_mark = 0;
    return e;
}

}  // namespace lbib

extern "C" {

int lbib_abi_version(void) { return 1; }

int lbib_lattice(int32_t *e, double *w) {
    for (int q = 0; q < NQ; ++q) {
        if (e) {
            e[3 * q] = d3q19_ex(q);
            e[3 * q + 1] = d3q19_ey(q);
            e[3 * q + 2] = d3q19_ez(q);
        }
        if (w) w[q] = d3q19_w(q);
    }
    return NQ;
}

int64_t lbib_footprint_bytes(const lbib_fluid_params *p, int64_t n_nodes, int64_t n_tri_total) {
    if (!p) return -1;
    FluidLayout L;
    if (!fluid_layout(*p, L)) return -1;
    // nodes: X, V (hi + lo FP32), membrane force, owner; templates: triangle,
    // edge and bending records
    return (int64_t)L.total + n_nodes * 64 + n_tri_total * (16 + 3 * 16 + 4 * 20);
}

lbib_status lbib_create(const lbib_fluid_params *p, void *stream, lbib_sim **out) {
    if (!p || !out) return LBIB_ERR_ARG;
    *out = nullptr;
    if (p->nx < 1 || p->nz < 1 || p->ny < (p->walls_y ? 3 : 1)) return LBIB_ERR_ARG;
    if (!(p->tau > 0.5) || !(p->rho0 > 0.0) || !(p->friction >= 0.0)) return LBIB_ERR_ARG;
    if (p->precision < 0 || p->precision > 2 || p->pop_scale_log2 < 0 || p->pop_scale_log2 > 30) return LBIB_ERR_ARG;
    FluidLayout L;
    if (!fluid_layout(*p, L)) return LBIB_ERR_ARG;
    static std::atomic<uint64_t> next_serial{1};
    lbib_sim *s = new lbib_sim();
    s->serial = next_serial++;
    s->p = *p;
    s->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return LBIB_ERR_CUDA;
    }
    cudaError_t e = cudaMalloc(&s->fluid_mem, L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return e == cudaErrorMemoryAllocation ? LBIB_ERR_NOMEM : LBIB_ERR_CUDA;
    }
    s->fluid_bytes = L.total;
    char *b = (char *)s->fluid_mem;
    SimDev &d = s->d;
    d.nx = p->nx;
    d.ny = p->ny;
    d.nz = p->nz;
    d.walls = p->walls_y ? 1 : 0;
    d.nyf = L.nyf;
    d.div_nx.init((uint32_t)p->nx);
    d.div_nyf.init((uint32_t)L.nyf);
    d.nf = L.nf;
    d.nfp = L.nfp;
    d.nwords = L.nwords;
    d.prec = p->precision;
    d.omega = (float)(1.0 / p->tau);
    d.fpre = (float)(1.0 - 0.5 / p->tau);
    d.rho0 = (float)p->rho0;
    d.gx = (float)p->body_force[0];
    d.gy = (float)p->body_force[1];
    d.gz = (float)p->body_force[2];
    const int sh = p->precision == LBIB_POP_F32 ? 0 : p->pop_scale_log2;
    d.scale = std::ldexp(1.0f, sh);
    d.inv_scale = std::ldexp(1.0f, -sh);
    d.xi = (float)p->friction;
    for (int k = 0; k < 2; ++k) {
        d.pop[k] = b + L.off_pop[k];
        d.G[k] = (float4 *)(b + L.off_G[k]);
    }
    d.amask = (uint32_t *)(b + L.off_amask);
    d.ufield = (float4 *)(b + L.off_ufield);
    d.status = (uint32_t *)(b + L.off_status);
    d.dropped = (double *)(b + L.off_dropped);
    e = cudaMemsetAsync(s->fluid_mem, 0, L.total, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    // the membrane kernel is short and on the critical path only if it
    // finishes after the fluid kernel: its blocks go first
    int prio_least = 0, prio_greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->aux, cudaStreamNonBlocking, prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, prio_greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_nodes, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_membrane, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fext, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(&s->status_pinned, 64);
    if (e != cudaSuccess) {
        if (s->ev_nodes) cudaEventDestroy(s->ev_nodes);
        if (s->ev_membrane) cudaEventDestroy(s->ev_membrane);
        if (s->ev_fext) cudaEventDestroy(s->ev_fext);
        if (s->aux) cudaStreamDestroy(s->aux);
        if (s->side) cudaStreamDestroy(s->side);
        cudaFree(s->fluid_mem);
        delete s;
        return LBIB_ERR_CUDA;
    }
    *out = s;
    return LBIB_OK;
}

void lbib_destroy(lbib_sim *s) {
    if (!s) return;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    if (s->aux) {
        cudaStreamSynchronize(s->aux);
        cudaStreamDestroy(s->aux);
    }
    if (s->side) {
        cudaStreamSynchronize(s->side);
        cudaStreamDestroy(s->side);
    }
    if (s->ev_nodes) cudaEventDestroy(s->ev_nodes);
    if (s->ev_membrane) cudaEventDestroy(s->ev_membrane);
    if (s->ev_fext) cudaEventDestroy(s->ev_fext);
    if (s->fext_pinned) cudaFreeHost(s->fext_pinned);
    if (s->status_pinned) cudaFreeHost(s->status_pinned);
    for (int k = 0; k < 2; ++k) {
        if (s->ana_pinned[k]) cudaFreeHost(s->ana_pinned[k]);
        if (s->ana_ev[k]) cudaEventDestroy(s->ana_ev[k]);
    }
    for (auto &t : s->tpl_mem) cudaFree(t);
    if (s->d_tpl) cudaFree(s->d_tpl);
    if (s->d_obj) cudaFree(s->d_obj);
    if (s->d_fext) cudaFree(s->d_fext);
    if (s->d_analyze) cudaFree(s->d_analyze);

    for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : s->prof_aux) cudaEventDestroy(e);
    if (s->dnodes) cudaFree(s->dnodes);
    if (s->rep_mem) cudaFree(s->rep_mem);
    if (s->solid_mem) cudaFree(s->solid_mem);
    if (s->fluid_mem) cudaFree(s->fluid_mem);
    delete s;
}

const char *lbib_last_error(const lbib_sim *s) { return s ? s->err.c_str() : "null simulation"; }

lbib_status lbib_template_create(lbib_sim *s, int tid, const double *xyz, int nn, const int32_t *tris, int nt,
                                 const double stretch[3], double ks, double kb, double kal, double kag, double kv,
                                 int nonlinear) {
    LBIB_GUARD(s);
    if (tid != (int)s->topo.size()) return fail(s, LBIB_ERR_ID, "template ids must be consecutive from 0");
    if (!xyz || !tris) return fail(s, LBIB_ERR_ARG, "null mesh array");
    if (nn < 4 || nn > MAX_TEMPLATE_NODES) return fail(s, LBIB_ERR_ARG, "template node count must be in [4, 5120]");
    Topology T;
    std::string err;
    if (!build_template(xyz, nn, tris, nt, stretch, T, err)) return fail(s, LBIB_ERR_MESH, err);
    // device records, one allocation
    const size_t bytes = template_bytes(T);
    void *mem = nullptr;
    LBIB_CUDA(s, cudaMalloc(&mem, bytes), "template records");
    std::vector<char> host(bytes, 0);
    size_t o = 0;
    TplDev dv{};
    auto put = [&](const void *src, size_t n) -> size_t {
        const size_t at = o;
        if (n) std::memcpy(host.data() + o, src, n);
        o = align_up(o + n, 256);
        return at;
    };
    auto fbits = [](double v) {
        const float f = (float)v;
        int32_t i;
        std::memcpy(&i, &f, 4);
        return i;
    };
    std::vector<int32_t> tri4(4 * (size_t)nt), quad4(4 * (size_t)T.ne);
    std::vector<float> hinge4(4 * (size_t)T.ne);
    // device records in the conflict-free evaluation order of each kind
    for (int j = 0; j < nt; ++j) {
        const int t = T.tri_order[j];
        for (int k = 0; k < 3; ++k) tri4[4 * j + k] = T.tri[3 * t + k];
        tri4[4 * j + 3] = fbits(T.S0[t]);
    }
    // edge e is (b, c) of bending quad e = (a, b, c, d): one record per edge
    // carries both (the stretching and the bending of that edge)
    for (int j = 0; j < T.ne; ++j) {
        const int e = T.quad_order[j];
        for (int k = 0; k < 4; ++k) quad4[4 * j + k] = T.quads[4 * e + k];
        hinge4[4 * j] = (float)T.L0[e];
        hinge4[4 * j + 1] = (float)(1.0 / T.L0[e]);
        hinge4[4 * j + 2] = (float)(1.0 / T.theta0[e]);
        hinge4[4 * j + 3] = 0.f;
    }
    const size_t o_tri = put(tri4.data(), tri4.size() * 4);
    const size_t o_quad = put(quad4.data(), quad4.size() * 4);
    const size_t o_hinge = put(hinge4.data(), hinge4.size() * 4);
    cudaError_t e = cudaMemcpyAsync(mem, host.data(), bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return cuda_fail(s, e, "template H2D");
    }
    char *b = (char *)mem;
    dv.nn = T.nn;
    dv.nt = T.nt;
    dv.ks = (float)ks;
    dv.kb = (float)kb;
    dv.kal = (float)kal;
    dv.kag = (float)kag;
    dv.kv = (float)kv;
    dv.nonlinear = nonlinear ? 1 : 0;
    dv.kal_altitude = 0;
    dv.Sg0 = T.Sg0;
    dv.V0 = T.V0;
    dv.ne = T.ne;
    dv.tri = (const int4 *)(b + o_tri);
    dv.quad = (const int4 *)(b + o_quad);
    dv.hinge = (const float4 *)(b + o_hinge);
    s->topo.push_back(std::move(T));
    s->tpl_dev.push_back(dv);
    s->tpl_mem.push_back(mem);
    s->tpl_bytes += bytes;
    s->max_nodes = std::max(s->max_nodes, nn);
    s->tables_dirty = true;
    return LBIB_OK;
}

lbib_status lbib_template_topology(const lbib_sim *s, int tid, int32_t *edges, int32_t *quads, double *L0,
                                   double *theta0, double *S0, double *globals, int *n_edges) {
    if (!s) return LBIB_ERR_ARG;
    if (tid < 0 || tid >= (int)s->topo.size()) return LBIB_ERR_ID;
    const Topology &T = s->topo[tid];
    if (edges) std::memcpy(edges, T.edges.data(), T.edges.size() * 4);
    if (quads) std::memcpy(quads, T.quads.data(), T.quads.size() * 4);
    if (L0) std::memcpy(L0, T.L0.data(), T.L0.size() * 8);
    if (theta0) std::memcpy(theta0, T.theta0.data(), T.theta0.size() * 8);
    if (S0) std::memcpy(S0, T.S0.data(), T.S0.size() * 8);
    if (globals) {
        globals[0] = T.Sg0;
        globals[1] = T.V0;
    }
    if (n_edges) *n_edges = T.ne;
    return LBIB_OK;
}

lbib_status lbib_mesh_check(const double *xyz, int nn, const int32_t *tris, int nt, const double stretch[3],
                            int32_t *edges, int32_t *quads, double *L0, double *theta0, double *S0, double *globals,
                            int *n_edges, char *msg, int msg_cap) {
    auto report = [&](lbib_status code, const std::string &m) {
        if (msg && msg_cap > 0) {
            std::snprintf(msg, (size_t)msg_cap, "%s", m.c_str());
        }
        return code;
    };
    if (!xyz || !tris) return report(LBIB_ERR_ARG, "null mesh array");
    if (nn < 4 || nn > MAX_TEMPLATE_NODES) return report(LBIB_ERR_ARG, "node count must be in [4, 5120]");
    Topology T;
    std::string err;
    if (!build_template(xyz, nn, tris, nt, stretch, T, err)) return report(LBIB_ERR_MESH, err);
    if (edges) std::memcpy(edges, T.edges.data(), T.edges.size() * 4);
    if (quads) std::memcpy(quads, T.quads.data(), T.quads.size() * 4);
    if (L0) std::memcpy(L0, T.L0.data(), T.L0.size() * 8);
    if (theta0) std::memcpy(theta0, T.theta0.data(), T.theta0.size() * 8);
    if (S0) std::memcpy(S0, T.S0.data(), T.S0.size() * 8);
    if (globals) {
        globals[0] = T.Sg0;
        globals[1] = T.V0;
    }
    if (n_edges) *n_edges = T.ne;
    return report(LBIB_OK, "");
}

lbib_status lbib_mesh_orient(const double *xyz, int nn, const int32_t *tris, int nt, int mode, int32_t *out,
                             int *changed) {
    if (!xyz || !tris || nn < 4 || nt < 4 || mode < 0 || mode > 2) return LBIB_ERR_ARG;
    int c = 0;
    std::string err;
    if (!orient_mesh(xyz, nn, tris, nt, mode, out, c, err)) return LBIB_ERR_MESH;
    if (changed) *changed = c;
    return LBIB_OK;
}

lbib_status lbib_object_add(lbib_sim *s, int oid, int tid, const double origin[3], const double rotate[3],
                            double mass) {
    LBIB_GUARD(s);
    if (oid != (int)s->objs.size()) return fail(s, LBIB_ERR_ID, "object ids must be consecutive from 0");
    if (tid < 0 || tid >= (int)s->topo.size()) return fail(s, LBIB_ERR_ID, "unknown template id");
    if (!origin || !(mass > 0.0)) return fail(s, LBIB_ERR_ARG, "origin required and mass must be > 0");
    lbib_status r = sim_download_nodes(s);
    if (r != LBIB_OK) return r;
    const Topology &T = s->topo[tid];
    if ((int64_t)s->nn_total + T.nn >= ((int64_t)1 << 31)) return fail(s, LBIB_ERR_ARG, "too many nodes");
    double R[3][3];
    const double zero[3] = {0, 0, 0};
    rotation_zyx(rotate ? rotate : zero, R);
    for (int i = 0; i < T.nn; ++i) {
        const double *x = &T.x[3 * (size_t)i];
        for (int k = 0; k < 3; ++k) {
            s->hX.push_back(R[k][0] * x[0] + R[k][1] * x[1] + R[k][2] * x[2] + origin[k]);
            s->hV.push_back(0.0);
        }
    }
    ObjDev ob{};
    ob.tid = tid;
    ob.first = s->nn_total;
    ob.nn = T.nn;
    ob.inv_mass = (float)(1.0 / mass);
    s->objs.push_back(ob);
    s->masses.push_back(mass);
    s->fext.insert(s->fext.end(), {0.f, 0.f, 0.f});

    s->nn_total += T.nn;
    s->host_newer = true;
    s->tables_dirty = true;
    return LBIB_OK;
}

lbib_status lbib_template_set_kal_direction(lbib_sim *s, int tid, int altitude) {
    LBIB_GUARD(s);
    if (tid < 0 || tid >= (int)s->tpl_dev.size()) return fail(s, LBIB_ERR_ID, "unknown template id");
    s->tpl_dev[tid].kal_altitude = altitude ? 1 : 0;
    s->tables_dirty = true;
    s->fel_valid = false;
    return LBIB_OK;
}

lbib_status lbib_set_solid(lbib_sim *s, const uint8_t *mask, int64_t n) {
    LBIB_GUARD(s);
    if (s->fluid_ready) return fail(s, LBIB_ERR_STATE, "obstacles must be set before lbib_fluid_init");
    SimDev &d = s->d;
    if (!mask) {
        if (s->solid_mem) cudaFree(s->solid_mem);
        s->solid_mem = nullptr;
        d.solid = nullptr;
        d.nsolid = 0;
        return LBIB_OK;
    }
    const int64_t ncell = (int64_t)s->p.nx * s->p.ny * s->p.nz;
    if (n != ncell) return fail(s, LBIB_ERR_ARG, "mask must cover the whole lattice [nz][ny][nx]");
    std::vector<uint32_t> bits((size_t)d.nwords, 0u);
    int count = 0;
    for (int z = 0; z < d.nz; ++z)
        for (int yf = 0; yf < d.nyf; ++yf)
            for (int x = 0; x < d.nx; ++x) {
                const int y = yf + d.walls;
                if (!mask[((int64_t)z * d.ny + y) * d.nx + x]) continue;
                const int f = x + d.nx * (yf + d.nyf * z);
                bits[f >> 5] |= 1u << (f & 31);
                ++count;
            }
    if (!s->solid_mem) LBIB_CUDA(s, cudaMalloc(&s->solid_mem, (size_t)d.nwords * 4), "obstacle mask");
    LBIB_CUDA(s, cudaMemcpyAsync(s->solid_mem, bits.data(), bits.size() * 4, cudaMemcpyHostToDevice, s->stream),
              "obstacle mask");
    LBIB_CUDA(s, cudaStreamSynchronize(s->stream), "obstacle mask");
    d.solid = s->solid_mem;
    d.nsolid = count;
    return LBIB_OK;
}

lbib_status lbib_set_inlet(lbib_sim *s, const int32_t box[6], const double u[3]) {
    LBIB_GUARD(s);
    if (!box || !u) return fail(s, LBIB_ERR_ARG, "null parameters");
    const int n[3] = {s->p.nx, s->p.ny, s->p.nz};
    int b[6];
    for (int k = 0; k < 3; ++k) {
        b[2 * k] = std::max(0, std::min(box[2 * k], n[k]));
        b[2 * k + 1] = std::max(b[2 * k], std::min(box[2 * k + 1], n[k]));
    }
    const double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    if (!(usq < 0.09)) return fail(s, LBIB_ERR_ARG, "inlet speed must be below 0.3");
    SimDev &d = s->d;
    for (int k = 0; k < 6; ++k) d.in_box[k] = b[k];
    for (int k = 0; k < 3; ++k) d.in_u[k] = (float)u[k];
    d.in_on = (b[0] < b[1] && b[2] < b[3] && b[4] < b[5]) ? 1 : 0;
    return LBIB_OK;
}

lbib_status lbib_set_repulsion(lbib_sim *s, const double object[3], const double wall[3]) {
    LBIB_GUARD(s);
    if (!object || !wall) return fail(s, LBIB_ERR_ARG, "null parameters");
    for (const double *p : {object, wall}) {
        if (!(p[0] >= 0.0) || !(p[2] >= 0.0) || (p[0] > 0.0 && !(p[1] > 0.0)))
            return fail(s, LBIB_ERR_ARG, "repulsion needs a >= 0, n > 0, cutoff >= 0");
    }
    // the nearest periodic image must be the only one within the cutoff
    const double half = 0.5 * std::min(s->p.nx, s->p.nz);
    if (object[2] >= half || (!s->p.walls_y && object[2] >= 0.5 * s->p.ny))
        return fail(s, LBIB_ERR_ARG, "repulsion cutoff must be below half the periodic box");
    for (int k = 0; k < 3; ++k) {
        s->rep_obj[k] = object[k];
        s->rep_wall[k] = wall[k];
    }
    SimDev &d = s->d;
    d.rep_a = (float)object[0];
    d.rep_n = (float)object[1];
    d.rep_rc = (float)object[2];
    d.rep_wa = (float)wall[0];
    d.rep_wn = (float)wall[1];
    d.rep_wrc = (float)wall[2];
    d.rep_wall_on = (s->p.walls_y && wall[0] > 0.0 && wall[2] > 0.0) ? 1 : 0;
    s->tables_dirty = true;  // (re)sizes the pair buffers and sets rep_on
    s->fel_valid = false;
    return LBIB_OK;
}

lbib_status lbib_object_set_force(lbib_sim *s, int oid, const double f[3]) {
    LBIB_GUARD(s);
    if (oid < 0 || oid >= (int)s->objs.size()) return fail(s, LBIB_ERR_ID, "unknown object id");
    if (!f) return fail(s, LBIB_ERR_ARG, "null force");
    for (int k = 0; k < 3; ++k) s->fext[3 * (size_t)oid + k] = (float)f[k];
    s->fext_dirty = true;
    return LBIB_OK;
}

static lbib_status set_node_array(lbib_sim *s, int oid, const double *src, int n, bool positions) {
    LBIB_GUARD(s);
    if (oid < 0 || oid >= (int)s->objs.size()) return fail(s, LBIB_ERR_ID, "unknown object id");
    if (!src || n != s->objs[oid].nn) return fail(s, LBIB_ERR_ARG, "node count must equal the template's");
    lbib_status r = sim_download_nodes(s);
    if (r != LBIB_OK) return r;
    std::vector<double> &dst = positions ? s->hX : s->hV;
    std::memcpy(&dst[3 * (size_t)s->objs[oid].first], src, 3 * (size_t)n * 8);
    s->host_newer = true;
    return LBIB_OK;
}

lbib_status lbib_object_set_nodes(lbib_sim *s, int oid, const double *xyz, int n) {
    return set_node_array(s, oid, xyz, n, true);
}

lbib_status lbib_object_set_velocities(lbib_sim *s, int oid, const double *v, int n) {
    return set_node_array(s, oid, v, n, false);
}

lbib_status lbib_fluid_init(lbib_sim *s) {
    LBIB_GUARD(s);
    // everything but the sticky status word is zeroed: h = 0, G = 0, u = 0
    FluidLayout L;
    fluid_layout(s->p, L);
    LBIB_CUDA(s, cudaMemsetAsync(s->fluid_mem, 0, L.off_status, s->stream), "fluid init");
    LBIB_CUDA(s, cudaMemsetAsync((char *)s->fluid_mem + L.off_dropped, 0, 24, s->stream), "fluid init");
    s->t = 0;
    s->gmode = -1;
    s->ufield_stale = false;
    s->mark_stale = true;
    s->fluid_ready = true;
    return LBIB_OK;
}

// Profiling events: `k` more from pool `pool`, created on demand.
static lbib_status prof_events(lbib_sim *s, std::vector<cudaEvent_t> &pool, size_t &used, int k, cudaEvent_t **ev) {
    while (pool.size() < used + k) {
        cudaEvent_t e;
        LBIB_CUDA(s, cudaEventCreate(&e), "profile event");
        pool.push_back(e);
    }
    *ev = &pool[used];
    used += k;
    return LBIB_OK;
}

// Membrane forces of the current node positions, on stream `st`.
static lbib_status launch_membrane_timed(lbib_sim *s, cudaStream_t st) {
    cudaEvent_t *ev = nullptr;
    if (s->prof_now) {
        lbib_status r = prof_events(s, s->prof_aux, s->prof_aux_used, 2, &ev);
        if (r != LBIB_OK) return r;
        LBIB_CUDA(s, cudaEventRecord(ev[0], st), "profile event");
    }
    LBIB_CUDA(s, launch_membrane(s->d, s->max_nodes, s->cluster, s->membrane_clusters, s->membrane_threads,
                                 s->membrane_group, st), "membrane forces");
    LBIB_CUDA(s, launch_repulsion(s->d, s->max_nodes, st), "repulsion");
    if (ev) LBIB_CUDA(s, cudaEventRecord(ev[1], st), "profile event");
    return LBIB_OK;
}

// One step is: coupling part of the object update (node kernel), then the
// fluid step; the membrane part of the NEXT step depends only on the node
// positions the node kernel wrote, so (overlap on) it runs on the second
// stream while the fluid step runs:
//   stream: [membrane(t) if not ready] nodes(t) -> ev_nodes, fluid(t), wait ev_membrane
//   aux:    wait ev_nodes, membrane(t+1) -> ev_membrane
// and `stream` has caught up with `aux` when the call returns.  With overlap
// off every step is membrane(t), nodes(t), fluid(t) on `stream`.
lbib_status lbib_step(lbib_sim *s, int n) {
    LBIB_GUARD(s);
    if (n < 0) return fail(s, LBIB_ERR_ARG, "negative step count");
    lbib_status r = sim_prepare_step(s);
    if (r != LBIB_OK) return r;
    const bool objects = s->nn_total > 0 && !s->objs.empty();
    s->prof_now = false;
    if (n > 0 && objects && !s->fel_valid && s->overlap) {
        r = launch_membrane_timed(s, s->stream);
        if (r != LBIB_OK) return r;
        s->fel_valid = true;
    }
    for (int i = 0; i < n; ++i) {
        const int par = (int)(s->t & 1);
        if (s->since_mark >= ACTIVE_RESET_STEPS) LBIB_CUDA(s, sim_remark(s, s->stream), "active cells");
        s->since_mark++;
        // timing events on sampled steps only: each event between two
        // kernels costs a few microseconds of the step
        s->prof_now = s->prof_on && (s->t % s->prof_every) == 0;
        if (objects && !s->overlap) {
            r = launch_membrane_timed(s, s->stream);
            if (r != LBIB_OK) return r;
        }
        cudaEvent_t *ev = nullptr;
        if (s->prof_now) {
            r = prof_events(s, s->prof_ev, s->prof_used, 3, &ev);
            if (r != LBIB_OK) return r;
            LBIB_CUDA(s, cudaEventRecord(ev[0], s->stream), "profile event");
        }
        // Early launch (programmatic dependent launch), after the first step
        // of the call and off the sampled steps: the node kernel may start
        // while the previous fluid kernel (or the mask rebuild or membrane
        // kernel after it) finishes, reading only node positions,
        // velocities and object tables before it waits (the previous node
        // kernel, their only writer, completed before that fluid kernel got
        // past its own wait); the fluid kernel may start while the node
        // kernel finishes, pulling populations the previous fluid kernel
        // wrote (complete once the node kernel got past its wait, and the
        // node kernel releases only after it) before it waits for the mask
        // and the coupling buffer.
        const bool early = s->early_launch && i > 0 && !s->prof_now;
        if (objects) LBIB_CUDA(s, launch_nodes(s->d, par, s->node_threads, s->stream, early), "node update");
        if (objects && s->overlap) {
            LBIB_CUDA(s, cudaEventRecord(s->ev_nodes, s->stream), "event");
            LBIB_CUDA(s, cudaStreamWaitEvent(s->aux, s->ev_nodes, 0), "event");
            r = launch_membrane_timed(s, s->aux);
            if (r != LBIB_OK) return r;
            LBIB_CUDA(s, cudaEventRecord(s->ev_membrane, s->aux), "event");
        }
        if (ev) LBIB_CUDA(s, cudaEventRecord(ev[1], s->stream), "profile event");
        LBIB_CUDA(s, launch_fluid(s->d, par, (long long)s->t, s->stream, early && objects), "fluid step");
        if (ev) LBIB_CUDA(s, cudaEventRecord(ev[2], s->stream), "profile event");
        if (objects && s->overlap) LBIB_CUDA(s, cudaStreamWaitEvent(s->stream, s->ev_membrane, 0), "event");
        s->t++;
        s->gmode = par;
    }
    s->prof_now = false;
    // with overlap, ev_nodes marks the last node update
    s->side_ok = n > 0 && objects && s->overlap;
    if (!s->overlap) s->fel_valid = false;
    if (n > 0 && s->nn_total > 0) s->dev_newer = true;
    return LBIB_OK;
}

lbib_status lbib_sync(lbib_sim *s) {
    LBIB_GUARD(s);
    return sim_check_status(s);
}

lbib_status lbib_read_nodes(lbib_sim *s, int oid, double *xyz, double *v, int64_t cap) {
    LBIB_GUARD(s);
    if (oid < -1 || oid >= (int)s->objs.size()) return fail(s, LBIB_ERR_ID, "unknown object id");
    const int64_t first = oid < 0 ? 0 : s->objs[oid].first;
    const int64_t n = oid < 0 ? s->nn_total : s->objs[oid].nn;
    if (cap < n) return fail(s, LBIB_ERR_ARG, "capacity too small");
    lbib_status r = sim_check_status(s);
    if (r != LBIB_OK) return r;
    r = sim_download_nodes(s);
    if (r != LBIB_OK) return r;
    if (xyz) std::memcpy(xyz, &s->hX[3 * first], 3 * n * 8);
    if (v) std::memcpy(v, &s->hV[3 * first], 3 * n * 8);
    return LBIB_OK;
}

static lbib_status read_fields(lbib_sim *s, float *u, float *rho, int64_t cap) {
    LBIB_GUARD(s);
    if (!s->fluid_ready) return fail(s, LBIB_ERR_STATE, "fluid not initialised");
    const int64_t ncell = (int64_t)s->p.nx * s->p.ny * s->p.nz;
    if (cap < (u ? 3 : 1) * ncell) return fail(s, LBIB_ERR_ARG, "capacity too small");
    lbib_status r = sim_check_status(s);
    if (r != LBIB_OK) return r;
    const size_t bytes = (size_t)(u ? 3 : 1) * ncell * 4;
    float *tmp = nullptr;
    LBIB_CUDA(s, cudaMallocAsync((void **)&tmp, bytes, s->stream), "read-out buffer");
    cudaError_t e = cudaMemsetAsync(tmp, 0, bytes, s->stream);
    if (e == cudaSuccess)
        e = launch_fields(s->d, (int)(s->t & 1), s->gmode, u ? tmp : nullptr, u ? nullptr : tmp, 0, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u ? u : rho, tmp, bytes, cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(tmp, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "read-out");
    if (rho && s->p.walls_y) {
        for (int z = 0; z < s->p.nz; ++z)
            for (int y : {0, s->p.ny - 1})
                for (int x = 0; x < s->p.nx; ++x)
                    rho[((int64_t)z * s->p.ny + y) * s->p.nx + x] = (float)s->p.rho0;
    }
    return LBIB_OK;
}

lbib_status lbib_read_velocity(lbib_sim *s, float *u, int64_t cap) {
    if (!u) return LBIB_ERR_ARG;
    return read_fields(s, u, nullptr, cap);
}

lbib_status lbib_read_density(lbib_sim *s, float *rho, int64_t cap) {
    if (!rho) return LBIB_ERR_ARG;
    return read_fields(s, nullptr, rho, cap);
}

lbib_status lbib_read_coupling_force(lbib_sim *s, float *g, int64_t cap) {
    LBIB_GUARD(s);
    if (!g) return fail(s, LBIB_ERR_ARG, "null output");
    const int64_t ncell = (int64_t)s->p.nx * s->p.ny * s->p.nz;
    if (cap < 3 * ncell) return fail(s, LBIB_ERR_ARG, "capacity too small");
    lbib_status r = sim_check_status(s);
    if (r != LBIB_OK) return r;
    const size_t bytes = (size_t)3 * ncell * 4;
    float *tmp = nullptr;
    LBIB_CUDA(s, cudaMallocAsync((void **)&tmp, bytes, s->stream), "read-out buffer");
    cudaError_t e = cudaMemsetAsync(tmp, 0, bytes, s->stream);
    if (e == cudaSuccess && s->gmode >= 0) e = launch_read_coupling(s->d, s->gmode, tmp, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g, tmp, bytes, cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(tmp, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "read coupling force");
    return LBIB_OK;
}

lbib_status lbib_set_coupling_force(lbib_sim *s, const float *g, int64_t n) {
    LBIB_GUARD(s);
    if (!g) return fail(s, LBIB_ERR_ARG, "null input");
    if (!s->fluid_ready) return fail(s, LBIB_ERR_STATE, "fluid not initialised");
    const int64_t ncell = (int64_t)s->p.nx * s->p.ny * s->p.nz;
    if (n != 3 * ncell) return fail(s, LBIB_ERR_ARG, "expected 3 * nx * ny * nz values");
    const int gpar = (int)((s->t + 1) & 1);  // the buffer of step t - 1
    FluidLayout L;
    fluid_layout(s->p, L);
    const size_t bytes = (size_t)3 * ncell * 4;
    float *tmp = nullptr;
    LBIB_CUDA(s, cudaMallocAsync((void **)&tmp, bytes, s->stream), "upload buffer");
    cudaError_t e = cudaMemcpyAsync(tmp, g, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = launch_set_coupling(s->d, gpar, tmp, s->stream);
    cudaFreeAsync(tmp, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "set coupling force");
    s->gmode = gpar;
    s->ufield_stale = true;
    return LBIB_OK;
}

lbib_status lbib_read_populations(lbib_sim *s, double *h, int64_t cap) {
    LBIB_GUARD(s);
    if (!h) return fail(s, LBIB_ERR_ARG, "null output");
    if (!s->fluid_ready) return fail(s, LBIB_ERR_STATE, "fluid not initialised");
    const int64_t ncell = (int64_t)s->p.nx * s->p.ny * s->p.nz;
    if (cap < NQ * ncell) return fail(s, LBIB_ERR_ARG, "capacity too small");
    lbib_status r = sim_check_status(s);
    if (r != LBIB_OK) return r;
    const size_t bytes = (size_t)NQ * ncell * 8;
    double *tmp = nullptr;
    LBIB_CUDA(s, cudaMallocAsync((void **)&tmp, bytes, s->stream), "read-out buffer");
    cudaError_t e = cudaMemsetAsync(tmp, 0, bytes, s->stream);
    if (e == cudaSuccess) e = launch_read_pops(s->d, (int)(s->t & 1), tmp, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, tmp, bytes, cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(tmp, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "read populations");
    return LBIB_OK;
}

lbib_status lbib_set_populations(lbib_sim *s, const double *h, int64_t n) {
    LBIB_GUARD(s);
    if (!h) return fail(s, LBIB_ERR_ARG, "null input");
    if (!s->fluid_ready) return fail(s, LBIB_ERR_STATE, "fluid not initialised");
    const int64_t ncell = (int64_t)s->p.nx * s->p.ny * s->p.nz;
    if (n != NQ * ncell) return fail(s, LBIB_ERR_ARG, "expected 19 * nx * ny * nz values");
    const size_t bytes = (size_t)NQ * ncell * 8;
    double *tmp = nullptr;
    LBIB_CUDA(s, cudaMallocAsync((void **)&tmp, bytes, s->stream), "upload buffer");
    cudaError_t e = cudaMemcpyAsync(tmp, h, bytes, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = launch_set_pops(s->d, (int)(s->t & 1), tmp, s->stream);
    cudaFreeAsync(tmp, s->stream);
    // the coupling-force history is not part of the populations
    FluidLayout L;
    fluid_layout(s->p, L);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = cudaMemsetAsync((char *)s->fluid_mem + L.off_G[k], 0, (size_t)L.nf * 16, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "set populations");
    s->gmode = -2;
    s->ufield_stale = true;
    s->mark_stale = true;
    return LBIB_OK;
}

lbib_status lbib_object_analyze(lbib_sim *s, int oid, double out[14]) {
    LBIB_GUARD(s);
    if (oid < 0 || oid >= (int)s->objs.size()) return fail(s, LBIB_ERR_ID, "unknown object id");
    if (!out) return fail(s, LBIB_ERR_ARG, "null output");
    lbib_status r = sim_upload(s);
    if (r != LBIB_OK) return r;
    double *tmp = nullptr;
    LBIB_CUDA(s, cudaMallocAsync((void **)&tmp, 14 * 8, s->stream), "analyze buffer");
    cudaError_t e = launch_analyze(s->d, oid, tmp, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, 14 * 8, cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(tmp, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "analyze");
    return LBIB_OK;
}

lbib_status lbib_fluid_mass(lbib_sim *s, double *mass) {
    LBIB_GUARD(s);
    if (!mass) return fail(s, LBIB_ERR_ARG, "null output");
    if (!s->fluid_ready) return fail(s, LBIB_ERR_STATE, "fluid not initialised");
    double *acc = nullptr;
    LBIB_CUDA(s, cudaMallocAsync((void **)&acc, 8, s->stream), "mass buffer");
    cudaError_t e = cudaMemsetAsync(acc, 0, 8, s->stream);
    double dev = 0.0;
    if (e == cudaSuccess) e = launch_mass(s->d, (int)(s->t & 1), acc, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dev, acc, 8, cudaMemcpyDeviceToHost, s->stream);
    cudaFreeAsync(acc, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "mass");
    *mass = (double)(s->d.nf - s->d.nsolid) * s->p.rho0 + dev;
    return LBIB_OK;
}

// Allocation-free form of lbib_fluid_mass (see include/lbib.h): no
// cudaMalloc / cudaMallocAsync / cudaFree and no pinned host buffer; the
// partials live in the library's static device scratch and come back into
// a stack array.
lbib_status lbib_check_bounded_wait(double seconds, int arrive, int *timed_out) {
    if (!timed_out || !(seconds > 0.0) || seconds > 10.0) return LBIB_ERR_ARG;
    uint32_t *d = nullptr, h = 0;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(d, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = run_wait_probe(d, (unsigned long long)(seconds * 1e9), arrive ? 1 : 0, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d) cudaFree(d);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) return LBIB_ERR_CUDA;
    *timed_out = (h & ST_TIMEOUT) ? 1 : 0;
    return LBIB_OK;
}

lbib_status lbib_fluid_mass_noalloc(lbib_sim *s, double *mass) {
    LBIB_GUARD(s);  // makes the simulation's device current
    if (!mass) return fail(s, LBIB_ERR_ARG, "null output");
    if (!s->fluid_ready) return fail(s, LBIB_ERR_STATE, "fluid not initialised");
    int sms = 0;
    LBIB_CUDA(s, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device), "device attribute");
    int blocks = 4 * sms;
    const int need = (s->d.nf + 255) / 256;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    if (blocks > MASS_SCRATCH_SLOTS)
        return fail(s, LBIB_ERR_ARG, "the reduction grid would need more partial slots than the static scratch holds");
    double *part = nullptr;
    LBIB_CUDA(s, mass_scratch(&part), "static scratch address");
    double host[MASS_SCRATCH_SLOTS];
    cudaError_t e = launch_mass_partials(s->d, (int)(s->t & 1), part, blocks, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, part, (size_t)blocks * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "mass");
    double dev = 0.0;
    for (int b = 0; b < blocks; ++b) dev += host[b];
    *mass = (double)(s->d.nf - s->d.nsolid) * s->p.rho0 + dev;
    return LBIB_OK;
}

lbib_status lbib_info(const lbib_sim *s, int64_t out[8]) {
    if (!s || !out) return LBIB_ERR_ARG;
    out[0] = (int64_t)s->topo.size();
    out[1] = (int64_t)s->objs.size();
    out[2] = s->nn_total;
    out[3] = s->d.nf;
    out[4] = s->t;
    out[5] = (int64_t)(s->fluid_bytes + s->tpl_bytes + s->node_bytes + s->rep_bytes +
                       (s->solid_mem ? (size_t)s->d.nwords * 4 : 0));
    out[6] = s->p.precision;
    out[7] = fluid_kernel_kind(s->d);
    return LBIB_OK;
}

lbib_status lbib_dropped_momentum(lbib_sim *s, double out[3]) {
    LBIB_GUARD(s);
    if (!out) return fail(s, LBIB_ERR_ARG, "null output");
    LBIB_CUDA(s, cudaMemcpyAsync(out, s->d.dropped, 24, cudaMemcpyDeviceToHost, s->stream), "dropped");
    LBIB_CUDA(s, cudaStreamSynchronize(s->stream), "dropped");
    return LBIB_OK;
}

lbib_status lbib_objects_set_force(lbib_sim *s, const double *f, int n_obj) {
    LBIB_GUARD(s);
    if (!f || n_obj != (int)s->objs.size()) return fail(s, LBIB_ERR_ARG, "need one force per object");
    for (size_t k = 0; k < 3 * (size_t)n_obj; ++k) s->fext[k] = (float)f[k];
    s->fext_dirty = true;
    return sim_upload(s);
}

lbib_status lbib_objects_analyze(lbib_sim *s, double *out, int64_t cap) {
    LBIB_GUARD(s);
    const int nobj = (int)s->objs.size();
    if (!out || cap < nobj) return fail(s, LBIB_ERR_ARG, "capacity too small");
    if (nobj == 0) return LBIB_OK;
    lbib_status r = sim_upload(s);
    if (r != LBIB_OK) return r;
    LBIB_CUDA(s, launch_analyze(s->d, -1, s->d_analyze, s->stream), "analyze");
    LBIB_CUDA(s, cudaMemcpyAsync(out, s->d_analyze, (size_t)nobj * 14 * sizeof(double), cudaMemcpyDeviceToHost,
                                 s->stream), "analyze");
    // the status word comes back with the analysis: one wait for both
    LBIB_CUDA(s, cudaMemcpyAsync(s->status_pinned, s->d.status, 4, cudaMemcpyDeviceToHost, s->stream), "analyze");
    LBIB_CUDA(s, cudaStreamSynchronize(s->stream), "analyze");
    return apply_status(s, *s->status_pinned);
}

lbib_status lbib_objects_analyze_async(lbib_sim *s, int slot) {
    LBIB_GUARD(s);
    if (slot != 0 && slot != 1) return fail(s, LBIB_ERR_ARG, "slot must be 0 or 1");
    if (s->ana_pending[slot]) return fail(s, LBIB_ERR_STATE, "slot not waited for");
    const int nobj = (int)s->objs.size();
    lbib_status r = sim_upload(s);
    if (r != LBIB_OK) return r;
    if (s->ana_cap[slot] < nobj || !s->ana_pinned[slot]) {
        if (s->ana_pinned[slot]) cudaFreeHost(s->ana_pinned[slot]);
        s->ana_pinned[slot] = nullptr;
        s->ana_cap[slot] = 0;
        const int cap = nobj > 0 ? nobj : 1;
        LBIB_CUDA(s, cudaMallocHost((void **)&s->ana_pinned[slot], ((size_t)cap * 14 + 1) * sizeof(double)),
                  "analysis buffer");
        s->ana_cap[slot] = cap;
    }
    if (!s->ana_ev[slot]) LBIB_CUDA(s, cudaEventCreateWithFlags(&s->ana_ev[slot], cudaEventDisableTiming), "event");
    double *h = s->ana_pinned[slot];
    // After a step the analysis (it reads node state only) runs on `side`
    // after the node update, beside the fluid and membrane kernels, and
    // `stream` waits for it before the next node update moves the nodes; the
    // status word it carries may then miss a flag the running fluid kernel
    // is about to set (the next read sees it).
    const bool side = s->side_ok;
    cudaStream_t ast = side ? s->side : s->stream;
    if (side) LBIB_CUDA(s, cudaStreamWaitEvent(ast, s->ev_nodes, 0), "analyze");
    if (nobj > 0) {
        LBIB_CUDA(s, launch_analyze(s->d, -1, s->d_analyze, ast), "analyze");
        LBIB_CUDA(s, cudaMemcpyAsync(h, s->d_analyze, (size_t)nobj * 14 * sizeof(double), cudaMemcpyDeviceToHost,
                                     ast), "analyze");
    }
    // the status word after the objects' records (the slot holds cap records)
    LBIB_CUDA(s, cudaMemcpyAsync(h + (size_t)s->ana_cap[slot] * 14, s->d.status, 4, cudaMemcpyDeviceToHost, ast),
              "analyze");
    LBIB_CUDA(s, cudaEventRecord(s->ana_ev[slot], ast), "analyze");
    if (side) LBIB_CUDA(s, cudaStreamWaitEvent(s->stream, s->ana_ev[slot], 0), "analyze");
    s->ana_nobj[slot] = nobj;
    s->ana_pending[slot] = true;
    return LBIB_OK;
}

lbib_status lbib_objects_analyze_wait(lbib_sim *s, int slot, double *out, int64_t cap) {
    LBIB_GUARD(s);
    if (slot != 0 && slot != 1) return fail(s, LBIB_ERR_ARG, "slot must be 0 or 1");
    if (!s->ana_pending[slot]) return fail(s, LBIB_ERR_STATE, "nothing enqueued in this slot");
    const int nobj = s->ana_nobj[slot];
    if (nobj > 0 && (!out || cap < nobj)) return fail(s, LBIB_ERR_ARG, "capacity too small");
    s->ana_pending[slot] = false;
    LBIB_CUDA(s, cudaEventSynchronize(s->ana_ev[slot]), "analyze");
    const double *h = s->ana_pinned[slot];
    if (nobj > 0) std::memcpy(out, h, (size_t)nobj * 14 * sizeof(double));
    uint32_t st;
    std::memcpy(&st, h + (size_t)s->ana_cap[slot] * 14, 4);
    return apply_status(s, st);
}

lbib_status lbib_set_tuning(lbib_sim *s, int key, int value) {
    LBIB_GUARD(s);
    if (key == LBIB_TUNE_IB_CLUSTER) {
        if (value < 1 || value > 8) return fail(s, LBIB_ERR_ARG, "cluster size must be in [1, 8]");
        s->cluster = value;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_OVERLAP) {
        if (value != 0 && value != 1) return fail(s, LBIB_ERR_ARG, "overlap must be 0 or 1");
        s->overlap = value != 0;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_MEMBRANE_THREADS) {
        if (value < 32 || value > IB_THREADS || value % 32) return fail(s, LBIB_ERR_ARG, "membrane threads must be a multiple of 32 in [32, 256]");
        s->membrane_threads = value;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_MEMBRANE_CLUSTERS) {
        if (value < 0 || value > (1 << 20)) return fail(s, LBIB_ERR_ARG, "membrane clusters must be in [0, 2^20]");
        s->membrane_clusters = value;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_FLUID_KERNEL) {
        if (value < 0 || value > 3) return fail(s, LBIB_ERR_ARG, "fluid kernel must be 0, 1, 2 or 3");
        s->d.fkern = value;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_MEMBRANE_GROUP) {
        if (value < 1 || value > 15) return fail(s, LBIB_ERR_ARG, "membrane group must be in [1, 15]");
        s->membrane_group = value;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_NODE_THREADS) {
        if (value != 32 && value != 64 && value != 128 && value != 256)
            return fail(s, LBIB_ERR_ARG, "node threads must be 32, 64, 128 or 256");
        s->node_threads = value;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_EARLY_LAUNCH) {
        if (value != 0 && value != 1) return fail(s, LBIB_ERR_ARG, "early launch must be 0 or 1");
        s->early_launch = value != 0;
        return LBIB_OK;
    }
    return fail(s, LBIB_ERR_ARG, "unknown tuning key");
}

lbib_status lbib_get_tuning(const lbib_sim *s, int key, int *value) {
    if (!s || !value) return LBIB_ERR_ARG;
    if (key == LBIB_TUNE_IB_CLUSTER) {
        *value = s->cluster;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_OVERLAP) {
        *value = s->overlap ? 1 : 0;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_MEMBRANE_THREADS) {
        *value = s->membrane_threads;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_MEMBRANE_CLUSTERS) {
        *value = s->membrane_clusters;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_FLUID_KERNEL) {
        *value = s->d.fkern;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_NODE_THREADS) {
        *value = s->node_threads;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_MEMBRANE_GROUP) {
        *value = s->membrane_group;
        return LBIB_OK;
    }
    if (key == LBIB_TUNE_EARLY_LAUNCH) {
        *value = s->early_launch ? 1 : 0;
        return LBIB_OK;
    }
    return LBIB_ERR_ARG;
}

lbib_status lbib_profile_enable(lbib_sim *s, int on) {
    LBIB_GUARD(s);
    s->prof_on = on != 0;
    s->prof_every = on > 1 ? on : 1;
    s->prof_used = 0;
    s->prof_aux_used = 0;
    return LBIB_OK;
}

lbib_status lbib_profile_read(lbib_sim *s, double out[6]) {
    LBIB_GUARD(s);
    if (!out) return fail(s, LBIB_ERR_ARG, "null output");
    LBIB_CUDA(s, cudaStreamSynchronize(s->stream), "profile");
    LBIB_CUDA(s, cudaStreamSynchronize(s->aux), "profile");
    double fl = 0.0, nodes = 0.0, mem = 0.0;
    for (size_t k = 0; k + 3 <= s->prof_used; k += 3) {
        float a = 0.f, b = 0.f;
        LBIB_CUDA(s, cudaEventElapsedTime(&a, s->prof_ev[k], s->prof_ev[k + 1]), "profile");
        LBIB_CUDA(s, cudaEventElapsedTime(&b, s->prof_ev[k + 1], s->prof_ev[k + 2]), "profile");
        nodes += a;
        fl += b;
    }
    for (size_t k = 0; k + 2 <= s->prof_aux_used; k += 2) {
        float a = 0.f;
        LBIB_CUDA(s, cudaEventElapsedTime(&a, s->prof_aux[k], s->prof_aux[k + 1]), "profile");
        mem += a;
    }
    const double steps = (double)(s->prof_used / 3);
    out[0] = fl;
    out[1] = steps;
    out[2] = nodes;
    out[3] = s->objs.empty() ? 0.0 : steps;
    out[4] = mem;
    out[5] = (double)(s->prof_aux_used / 2);
    return LBIB_OK;
}

}  // extern "C"
