// Lattice-index arithmetic of the immersed-boundary coupling (Sec. 2: the
// velocity is interpolated from, and the drag spread to, the 8 lattice nodes
// around a membrane node).  Host and device compile the same functions, so
// the index bounds can be checked on the host with any coordinates,
// including non-finite and saturated ones.
//
// D is any descriptor with int members nx, ny, nz, walls and nyf (fluid
// rows: ny - 2 with walls, ny without).  Fluid cell index
// f = x + nx (y' + nyf z) with y' = y - 1 with walls, y' = y without.
//
// Bounds, for every float input:
//   lattice_coord   i0 in [-2^30 - 1, 2^30 + 1], so i0 + d for the small
//                   offsets d used below never overflows
//   corner_cells    every f[k] is -1 or in [0, nx nyf nz)
//   for_each_halo   calls fn(f) only with f in [0, nx nyf nz)
//   halo_cell       -1 or in [0, nx nyf nz)
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define LBIB_HD __host__ __device__ __forceinline__
#else
#define LBIB_HD inline
#endif

namespace lbib {

// i mod n in [0, n) for n >= 1 and any i.
LBIB_HD int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Fluid index of lattice node (cx, cy, cz) with cx in [0, nx), cz in
// [0, nz) already wrapped, or -1 when cy is a solid row or outside the
// walled box (y is wrapped without walls).
template <class D>
LBIB_HD int fluid_index(const D &g, int cx, int cy, int cz) {
    if (g.walls) {
        if (cy < 1 || cy > g.ny - 2) return -1;
        cy -= 1;
    } else {
        cy = wrapi(cy, g.ny);
    }
    return cx + g.nx * (cy + g.nyf * cz);
}

// Lower lattice index and fraction of one coordinate given as hi + lo:
// i0 = floor(x - 1/2), w = x - 1/2 - i0 in [0, 1) (lattice node i sits at
// i + 1/2).  hi - 1/2 and the subtraction of the integer are exact for
// |x| < 2^22.  Coordinates beyond +-2^30 (a simulation that has already
// failed) are clamped, so the integer conversion is defined on every
// platform and later offsets cannot overflow.
LBIB_HD void lattice_coord(float hi, float lo, int &i0, float &w) {
    const float p = hi - 0.5f;
    float fl = floorf(p);
    float fr = (p - fl) + lo;
    if (fr < 0.f) {
        fl -= 1.f;
        fr += 1.f;
    } else if (fr >= 1.f) {
        fl += 1.f;
        fr -= 1.f;
    }
    const float lim = 1073741824.0f;  // 2^30
    fl = fminf(fmaxf(fl, -lim), lim);  // a NaN fl becomes -2^30 (fmaxf drops NaN)
    i0 = (int)fl;
    w = fr;
}

// The 8 interpolation corners of a point: corner k = (dx, dy, dz) =
// (k & 1, k >> 1 & 1, k >> 2 & 1) is lattice node (i0 + dx, j0 + dy,
// k0 + dz) with trilinear weight w[k] (the volume of the box between the
// point and the diagonally opposite corner); f[k] = -1 on a solid row.
template <class D>
LBIB_HD void corner_cells(const D &g, float xh, float xl, float yh, float yl, float zh, float zl, int (&f)[8],
                          float (&w)[8]) {
    int ix, iy, iz;
    float wx, wy, wz;
    lattice_coord(xh, xl, ix, wx);
    lattice_coord(yh, yl, iy, wy);
    lattice_coord(zh, zl, iz, wz);
    // one modulo per axis (positions are not wrapped), then the +1 neighbour
    const int cx0 = wrapi(ix, g.nx), cx1 = cx0 + 1 == g.nx ? 0 : cx0 + 1;
    const int cz0 = wrapi(iz, g.nz), cz1 = cz0 + 1 == g.nz ? 0 : cz0 + 1;
    int cy0, cy1;
    bool in0 = true, in1 = true;
    if (g.walls) {  // fluid row = lattice row - 1; rows 0 and ny - 1 are solid
        cy0 = iy - 1;
        cy1 = iy;
        in0 = iy >= 1 && iy <= g.ny - 2;
        in1 = iy >= 0 && iy <= g.ny - 3;
    } else {
        cy0 = wrapi(iy, g.ny);
        cy1 = cy0 + 1 == g.ny ? 0 : cy0 + 1;
    }
#if defined(__CUDACC__)
#pragma unroll
#endif
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        f[k] = (dy ? in1 : in0) ? (dx ? cx1 : cx0) + g.nx * ((dy ? cy1 : cy0) + g.nyf * (dz ? cz1 : cz0)) : -1;
        w[k] = (dx ? wx : 1.f - wx) * (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
    }
}

// Fluid index of halo node j in [0, 64) of lower corner (ix, iy, iz):
// offsets dx = j % 4 - 1, dy = (j / 4) % 4 - 1, dz = j / 16 - 1, so that the
// 64 values of j give the nodes for_each_halo visits; -1 on a solid row.
template <class D>
LBIB_HD int halo_cell(const D &g, int ix, int iy, int iz, int j) {
    return fluid_index(g, wrapi(ix + (j & 3) - 1, g.nx), iy + ((j >> 2) & 3) - 1, wrapi(iz + (j >> 4) - 1, g.nz));
}

// Calls fn(f) for every fluid cell of the 4x4x4 lattice nodes
// (ix-1 .. ix+2, iy-1 .. iy+2, iz-1 .. iz+2) around lower corner
// (ix, iy, iz) as lattice_coord returns it (solid rows skipped).
template <class D, class F>
LBIB_HD void for_each_halo(const D &g, int ix, int iy, int iz, F &&fn) {
    for (int dz = -1; dz <= 2; ++dz) {
        const int cz = wrapi(iz + dz, g.nz);
        for (int dy = -1; dy <= 2; ++dy)
            for (int dx = -1; dx <= 2; ++dx) {
                const int f = fluid_index(g, wrapi(ix + dx, g.nx), iy + dy, cz);
                if (f >= 0) fn(f);
            }
    }
}

}  // namespace lbib
