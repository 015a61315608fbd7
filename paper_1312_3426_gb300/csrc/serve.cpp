// Continuous-batching scheduler (lbib_server_*): many simulations resident
// on one device, all advanced together by lbib_batch_step.  New
// simulations join the resident set between advances as soon as a slot and
// enough of the byte budget are free, and leave it the moment their step
// count is reached, so a long request does not hold back short ones that
// arrive later (unlike a first-come-first-served loop that runs one request
// to completion at a time).  Host-only: every device operation goes through
// the public C ABI.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "lbib.h"

struct lbib_server {
    int64_t budget = 0;
    int max_resident = 0;
    int chunk = 1;
    struct Entry {
        lbib_sim *sim;
        int64_t left;   // steps still to run
        int64_t tag;
        int64_t bytes;  // device bytes held
        int64_t cells;  // fluid cells
    };
    std::vector<Entry> res;
    int64_t bytes = 0;
    int64_t advances = 0;
    int64_t updates = 0;
};

extern "C" {

lbib_status lbib_server_create(int64_t budget_bytes, int max_resident, int chunk_steps, lbib_server **out) {
    if (!out) return LBIB_ERR_ARG;
    *out = nullptr;
    if (budget_bytes <= 0 || max_resident < 1 || chunk_steps < 1) return LBIB_ERR_ARG;
    lbib_server *s = new lbib_server();
    s->budget = budget_bytes;
    s->max_resident = max_resident;
    s->chunk = chunk_steps;
    *out = s;
    return LBIB_OK;
}

void lbib_server_destroy(lbib_server *srv) { delete srv; }

lbib_status lbib_server_admit(lbib_server *srv, lbib_sim *sim, int64_t n_steps, int64_t tag) {
    if (!srv || !sim || n_steps < 1) return LBIB_ERR_ARG;
    for (const auto &e : srv->res)
        if (e.sim == sim) return LBIB_ERR_ARG;
    int64_t info[8];
    lbib_status r = lbib_info(sim, info);
    if (r != LBIB_OK) return r;
    const int64_t bytes = info[5];
    if ((int)srv->res.size() >= srv->max_resident || srv->bytes + bytes > srv->budget) return LBIB_ERR_NOMEM;
    srv->res.push_back({sim, n_steps, tag, bytes, info[3]});
    srv->bytes += bytes;
    return LBIB_OK;
}

lbib_status lbib_server_advance(lbib_server *srv, int64_t *done, int cap, int *n_done) {
    if (!srv || !n_done || cap < 0 || (cap > 0 && !done)) return LBIB_ERR_ARG;
    *n_done = 0;
    if (srv->res.empty()) return LBIB_OK;
    int64_t k = srv->chunk;
    for (const auto &e : srv->res) k = std::min(k, e.left);
    if (k > 0) {
        std::vector<lbib_sim *> sims;
        sims.reserve(srv->res.size());
        for (const auto &e : srv->res) sims.push_back(e.sim);
        const lbib_status r = lbib_batch_step(sims.data(), (int)sims.size(), (int)k);
        if (r == LBIB_ERR_ARG) return r;
        srv->advances++;
        for (auto &e : srv->res) {
            if (r != LBIB_OK) {
                // lbib_batch_step failed: a device error makes every
                // simulation of the batch sticky, and one that entered the
                // call sticky or failed to prepare stays so; those are
                // retired now as failed.  A simulation that lbib_sync still
                // finds healthy did not advance and runs again next time.
                if (lbib_sync(e.sim) != LBIB_OK) e.left = 0;
                continue;
            }
            e.left -= k;
            srv->updates += e.cells * k;
        }
    }
    // retire in admission order
    std::vector<lbib_server::Entry> keep;
    keep.reserve(srv->res.size());
    for (const auto &e : srv->res) {
        if (e.left == 0 && *n_done < cap) {
            done[(*n_done)++] = e.tag;
            srv->bytes -= e.bytes;
        } else {
            keep.push_back(e);
        }
    }
    srv->res.swap(keep);
    return LBIB_OK;
}

lbib_status lbib_server_stats(const lbib_server *srv, int64_t out[4]) {
    if (!srv || !out) return LBIB_ERR_ARG;
    out[0] = (int64_t)srv->res.size();
    out[1] = srv->bytes;
    out[2] = srv->advances;
    out[3] = srv->updates;
    return LBIB_OK;
}

}  // extern "C"
