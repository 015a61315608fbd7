// Device-side body of the per-object immersed-boundary update, shared by the
// single-simulation kernel (ib.cu) and the batched persistent kernel
// (batch.cu).  See ib.cu for the description of the update.
#pragma once

#include "lbib_internal.h"

namespace lbib {

struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

struct Stage {
    const float *hx, *hy, *hz, *lx, *ly, *lz;
    // position of node q relative to node p
    __device__ __forceinline__ f3 rel(int q, int p) const {
        return {(hx[q] - hx[p]) + (lx[q] - lx[p]), (hy[q] - hy[p]) + (ly[q] - ly[p]),
                (hz[q] - hz[p]) + (lz[q] - lz[p])};
    }
    __device__ __forceinline__ f3 pos(int q) const { return {hx[q] + lx[q], hy[q] + ly[q], hz[q] + lz[q]}; }
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Fluid index of lattice node (cx, cy, cz) (cx, cz already wrapped), or -1
// when the node is in a solid row (or outside the walled box).
__device__ __forceinline__ int fluid_index(const SimDev &s, int cx, int cy, int cz) {
    if (s.walls) {
        if (cy < 1 || cy > s.ny - 2) return -1;
        cy -= 1;
    } else {
        cy = wrapi(cy, s.ny);
    }
    return cx + s.nx * (cy + s.nyf * cz);
}

struct Corners {
    int f[8];
    float w[8];
};

// Trilinear weights: corner (i0+dx, j0+dy, k0+dz) gets the volume of the
// box between the point and the diagonally opposite corner.
__device__ __forceinline__ void corners(const SimDev &s, double x, double y, double z, Corners &c) {
    const double px = x - 0.5, py = y - 0.5, pz = z - 0.5;
    const double fx = floor(px), fy = floor(py), fz = floor(pz);
    const float wx = (float)(px - fx), wy = (float)(py - fy), wz = (float)(pz - fz);
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    const int cx0 = wrapi(ix, s.nx), cx1 = wrapi(ix + 1, s.nx);
    const int cz0 = wrapi(iz, s.nz), cz1 = wrapi(iz + 1, s.nz);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        c.f[k] = fluid_index(s, dx ? cx1 : cx0, iy + dy, dz ? cz1 : cz0);
        c.w[k] = (dx ? wx : 1.f - wx) * (dy ? wy : 1.f - wy) * (dz ? wz : 1.f - wz);
    }
}

__device__ __forceinline__ void mark(uint32_t *mask, int f) { atomicOr(mask + (f >> 5), 1u << (f & 31)); }

// Shared memory: 6 floats per node of the largest template.
constexpr int IB_SMEM_PER_NODE = 6 * sizeof(float);

__device__ __forceinline__ void ib_object(const SimDev &s, int o, int par, float *sh) {
    __syncthreads();  // a persistent block may still read the previous object's staging
    const ObjDev ob = s.obj[o];
    const TplDev T = s.tpl[ob.tid];
    const int nn = ob.nn;
    const int NN = s.nn_total;
    double *Xx = s.X, *Xy = s.X + NN, *Xz = s.X + 2 * NN;
    double *Vx = s.V, *Vy = s.V + NN, *Vz = s.V + 2 * NN;

    Stage P{sh, sh + nn, sh + 2 * nn, sh + 3 * nn, sh + 4 * nn, sh + 5 * nn};
    const double Rx = Xx[ob.first], Ry = Xy[ob.first], Rz = Xz[ob.first];
    for (int p = threadIdx.x; p < nn; p += IB_THREADS) {
        const double dx = Xx[ob.first + p] - Rx, dy = Xy[ob.first + p] - Ry, dz = Xz[ob.first + p] - Rz;
        const float hx = (float)dx, hy = (float)dy, hz = (float)dz;
        sh[p] = hx;
        sh[nn + p] = hy;
        sh[2 * nn + p] = hz;
        sh[3 * nn + p] = (float)(dx - (double)hx);
        sh[4 * nn + p] = (float)(dy - (double)hy);
        sh[5 * nn + p] = (float)(dz - (double)hz);
    }
    __syncthreads();

    // ---- total area and volume (FP64 accumulation)
    double sg = 0.0, vol = 0.0;
    for (int t = threadIdx.x; t < T.nt; t += IB_THREADS) {
        const int4 tr = T.tri[t];
        const f3 eb = P.rel(tr.y, tr.x), ec = P.rel(tr.z, tr.x);
        const f3 N = cross(eb, ec);
        sg += 0.5 * (double)sqrtf(dot(N, N));
        vol += (double)dot(P.pos(tr.x), N);
    }
    __shared__ double red[2][IB_THREADS / 32];
    sg = warp_sum_d(sg);
    vol = warp_sum_d(vol);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sg;
        red[1][threadIdx.x >> 5] = vol;
    }
    __syncthreads();
    sg = 0.0;
    vol = 0.0;
#pragma unroll
    for (int k = 0; k < IB_THREADS / 32; ++k) {
        sg += red[0][k];
        vol += red[1][k];
    }
    const double V = -vol / 6.0;
    const float dSg = (float)((sg - T.Sg0) / sg);
    const float dV = (float)((V - T.V0) / T.V0);

    const float PI_F = 3.14159265358979f;
    for (int p = threadIdx.x; p < nn; p += IB_THREADS) {
        f3 F = mk(0.f, 0.f, 0.f);
        // stretching
        if (T.ks != 0.f) {
            for (int k = T.eoff[p]; k < T.eoff[p + 1]; ++k) {
                const int2 r = T.erec[k];
                const float L0 = __int_as_float(r.y);
                const f3 d = P.rel(r.x, p);
                const float L = sqrtf(dot(d, d));
                const float lam = L / L0;
                float kap = 1.f;
                if (T.nonlinear) {
                    const float sl = sqrtf(lam);
                    kap = (sl + 1.f / (lam * lam * sl)) / (lam + 1.f / (lam * lam * lam));
                }
                F = F + (T.ks * kap * (L - L0) / (L0 * L)) * d;
            }
        }
        // bending
        if (T.kb != 0.f) {
            for (int k = T.qoff[p]; k < T.qoff[p + 1]; ++k) {
                const int4 id = T.qrec[k];
                const float th0 = T.qth0[k];
                const f3 A = P.rel(id.x, p), B = P.rel(id.y, p), C = P.rel(id.z, p), D = P.rel(id.w, p);
                f3 n1 = cross(B - A, C - A);
                f3 n2 = cross(C - D, B - D);
                n1 = rsqrtf(dot(n1, n1)) * n1;
                n2 = rsqrtf(dot(n2, n2)) * n2;
                const f3 cr = cross(n1, n2);
                const float alpha = atan2f(sqrtf(dot(cr, cr)), dot(n1, n2));
                const float theta = dot(D - B, n1) > 0.f ? PI_F - alpha : PI_F + alpha;
                const float sb = T.kb * (theta - th0) / th0;
                if (id.x == p)
                    F = F + sb * n1;
                else
                    F = F - (0.5f * sb) * (n1 + n2);
            }
        }
        // local area, global area, volume
        if (T.kal != 0.f || T.kag != 0.f || T.kv != 0.f) {
            for (int k = T.toff[p]; k < T.toff[p + 1]; ++k) {
                const int4 tr = T.trec[k];
                const float S0 = __int_as_float(tr.w);
                const f3 B = P.rel(tr.y, p), C = P.rel(tr.z, p);
                const f3 N = cross(B, C);
                const float nlen = sqrtf(dot(N, N));
                const float S = 0.5f * nlen;
                const f3 cen = (1.f / 3.f) * (B + C);  // centroid relative to the node
                const f3 w = (-rsqrtf(dot(cen, cen))) * cen;
                const float cw = -T.kal * (S - S0) / S - T.kag * dSg;
                const float cv = T.kv * dV * S / (3.f * nlen);
                F = F + cw * w + cv * N;
            }
        }

        // ---- coupling: interpolation, drag, spreading
        const int i = ob.first + p;
        double x = Xx[i], y = Xy[i], z = Xz[i];
        double vx = Vx[i], vy = Vy[i], vz = Vz[i];
        Corners c;
        corners(s, x, y, z, c);
        float ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (c.f[k] >= 0) {
                const float4 u = s.ufield[c.f[k]];
                ux += c.w[k] * u.x;
                uy += c.w[k] * u.y;
                uz += c.w[k] * u.z;
            }
        }
        const double fdx = s.xi * ((double)ux - vx);
        const double fdy = s.xi * ((double)uy - vy);
        const double fdz = s.xi * ((double)uz - vz);
        const float gx = (float)-fdx, gy = (float)-fdy, gz = (float)-fdz;
        float dropx = 0.f, dropy = 0.f, dropz = 0.f;
        float4 *G = s.G[par];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (c.f[k] >= 0) {
                atomicAdd(G + c.f[k], make_float4(c.w[k] * gx, c.w[k] * gy, c.w[k] * gz, 0.f));
                mark(s.gmask[par], c.f[k]);
            } else {
                dropx += c.w[k] * gx;
                dropy += c.w[k] * gy;
                dropz += c.w[k] * gz;
            }
        }
        if (dropx != 0.f || dropy != 0.f || dropz != 0.f) {
            atomicAdd(s.dropped, (double)dropx);
            atomicAdd(s.dropped + 1, (double)dropy);
            atomicAdd(s.dropped + 2, (double)dropz);
        }

        // ---- Newton update
        const double im = 1.0 / ob.mass;
        const double *fe = s.fext + 3 * o;
        vx += ((double)F.x + fdx + fe[0]) * im;
        vy += ((double)F.y + fdy + fe[1]) * im;
        vz += ((double)F.z + fdz + fe[2]) * im;
        x += vx;
        y += vy;
        z += vz;
        Vx[i] = vx;
        Vy[i] = vy;
        Vz[i] = vz;
        Xx[i] = x;
        Xy[i] = y;
        Xz[i] = z;
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
            atomicOr(s.status, ST_NODE_NAN);
        } else {
            corners(s, x, y, z, c);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (c.f[k] >= 0) mark(s.umask, c.f[k]);
        }
    }
}


}  // namespace lbib
