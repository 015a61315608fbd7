// Host driver for the bounds test of the lattice-index arithmetic
// (paper_1312_3426_gb300/csrc/lattice_index.h), compiled by the CPU test
// suite with the host C++ compiler.  It applies to every node what the node
// kernel applies: interpolation corners at the position, then the 4x4x4
// marking halo around the lower corner, both skipped for a non-finite
// leading part, and counts indices outside the fluid cells.
//
// usage: lattice_index_bounds nx ny nz walls < records
// records: 6 float32 per node (x hi, x lo, y hi, y lo, z hi, z lo)
// prints:  nodes skipped corner_refs halo_refs bad max_index max_word nf nwords
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "lattice_index.h"

struct Box {
    int nx, ny, nz, walls, nyf;
};

int main(int argc, char **argv) {
    if (argc != 5) {
        std::fprintf(stderr, "usage: %s nx ny nz walls < records\n", argv[0]);
        return 2;
    }
    Box g{std::atoi(argv[1]), std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]) ? 1 : 0, 0};
    g.nyf = g.walls ? g.ny - 2 : g.ny;
    const long long nf = (long long)g.nx * g.nyf * g.nz;
    const long long nwords = (nf + 31) / 32;
    long long nodes = 0, skipped = 0, corner_refs = 0, halo_refs = 0, bad = 0, max_f = -1, max_w = -1;
    float r[6];
    while (std::fread(r, sizeof(float), 6, stdin) == 6) {
        ++nodes;
        if (!std::isfinite(r[0]) || !std::isfinite(r[2]) || !std::isfinite(r[4])) {
            ++skipped;
            continue;
        }
        int f[8];
        float w[8];
        lbib::corner_cells(g, r[0], r[1], r[2], r[3], r[4], r[5], f, w);
        for (int k = 0; k < 8; ++k) {
            if (f[k] < 0) {
                if (f[k] != -1) ++bad;
                continue;
            }
            ++corner_refs;
            if (f[k] >= nf) ++bad;
            if (f[k] > max_f) max_f = f[k];
            if ((f[k] >> 5) > max_w) max_w = f[k] >> 5;
        }
        int ix, iy, iz;
        float t;
        lbib::lattice_coord(r[0], r[1], ix, t);
        lbib::lattice_coord(r[2], r[3], iy, t);
        lbib::lattice_coord(r[4], r[5], iz, t);
        int seq[64], ns = 0;
        lbib::for_each_halo(g, ix, iy, iz, [&](int c) {
            ++halo_refs;
            if (c < 0 || c >= nf || (c >> 5) >= nwords) ++bad;
            if (c > max_f) max_f = c;
            if ((c >> 5) > max_w) max_w = c >> 5;
            if (ns < 64) seq[ns] = c;
            ++ns;
        });
        // halo_cell over j = 0..63 gives the same cells in the same order
        int nj = 0;
        for (int j = 0; j < 64; ++j) {
            const int c = lbib::halo_cell(g, ix, iy, iz, j);
            if (c < -1 || c >= nf) ++bad;
            if (c >= 0) {
                if (nj >= ns || seq[nj] != c) ++bad;
                ++nj;
            }
        }
        if (nj != ns || ns > 64) ++bad;
    }
    std::printf("%lld %lld %lld %lld %lld %lld %lld %lld %lld\n", nodes, skipped, corner_refs, halo_refs, bad, max_f,
                max_w, nf, nwords);
    return 0;
}
