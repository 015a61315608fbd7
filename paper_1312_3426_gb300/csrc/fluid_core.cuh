// Device-side body of the fused fluid update (Eq. lbequation), shared by the
// single-simulation kernel (fluid.cu) and the batched persistent kernel
// (batch.cu).  See fluid.cu for the description of the update.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbib_internal.h"

namespace lbib {

// Storage of one population.  FP32 is stored as is.  FP16/BF16 store the
// deviation times 2^s with stochastic rounding: a random integer below the
// weight of the first dropped bit is added to the FP32 bit pattern, which is
// then truncated, so the stored value is unbiased.  Rounding to nearest
// would turn the per-step forcing increment, which is far below one unit in
// the last place of a 16-bit number once the flow has built up, into a
// systematic error.  The random bits come from a counter-based hash of
// (cell, step, direction), so results are reproducible.
template <typename T>
struct PopIO;

template <>
struct PopIO<float> {
    static __device__ __forceinline__ float ld(const float *p, float) { return __ldg(p); }
    static __device__ __forceinline__ void st(float *p, float v, float, uint32_t) { __stcs(p, v); }
};
template <>
struct PopIO<__half> {
    static __device__ __forceinline__ float ld(const __half *p, float inv) { return __half2float(__ldg(p)) * inv; }
    static __device__ __forceinline__ void st(__half *p, float v, float sc, uint32_t rnd) {
        const uint32_t b = __float_as_uint(v * sc) + (rnd & 0x1fffu);  // 13 bits dropped by FP16
        *p = __float2half_rz(__uint_as_float(b));
    }
};
template <>
struct PopIO<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, float inv) {
        return __bfloat162float(__ldg(p)) * inv;
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v, float sc, uint32_t rnd) {
        const uint32_t b = __float_as_uint(v * sc) + (rnd & 0xffffu);  // 16 bits dropped by BF16
        *p = __float2bfloat16_rz(__uint_as_float(b));
    }
};

// 32-bit integer hash (xor-shift / multiply finaliser) for the rounding bits.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Neighbour offsets of one cell in the fluid index space.
struct Nbr {
    int dxm, dxp, dym, dyp, dzm, dzp;  // index delta to the cell at x-1, x+1, ...
    bool ylo_solid, yhi_solid;         // the row below / above is a wall
};

__device__ __forceinline__ Nbr neighbours(const SimDev &s, int x, int y, int z) {
    Nbr n;
    const int plane = s.nx * s.nyf;
    n.dxm = (x == 0) ? s.nx - 1 : -1;
    n.dxp = (x == s.nx - 1) ? -(s.nx - 1) : 1;
    n.dzm = (z == 0) ? (s.nz - 1) * plane : -plane;
    n.dzp = (z == s.nz - 1) ? -(s.nz - 1) * plane : plane;
    if (s.walls) {
        n.ylo_solid = (y == 0);
        n.yhi_solid = (y == s.nyf - 1);
        n.dym = -s.nx;
        n.dyp = s.nx;
    } else {
        n.ylo_solid = n.yhi_solid = false;
        n.dym = (y == 0) ? (s.nyf - 1) * s.nx : -s.nx;
        n.dyp = (y == s.nyf - 1) ? -(s.nyf - 1) * s.nx : s.nx;
    }
    return n;
}

// Pull the population of direction Q arriving at cell f.
template <typename T, int Q>
__device__ __forceinline__ float pull(const T *__restrict__ src, int nfp, int f, const Nbr &n, float inv) {
    constexpr int ex = d3q19_ex(Q), ey = d3q19_ey(Q), ez = d3q19_ez(Q);
    if ((ey == 1 && n.ylo_solid) || (ey == -1 && n.yhi_solid))
        return PopIO<T>::ld(src + (size_t)d3q19_opp(Q) * nfp + f, inv);
    int g = f;
    if (ex == 1) g += n.dxm;
    if (ex == -1) g += n.dxp;
    if (ey == 1) g += n.dym;
    if (ey == -1) g += n.dyp;
    if (ez == 1) g += n.dzm;
    if (ez == -1) g += n.dzp;
    return PopIO<T>::ld(src + (size_t)Q * nfp + g, inv);
}

template <typename T, int Q>
__device__ __forceinline__ void collide_store(T *__restrict__ dst, int nfp, int f, float h, float drho, float rho,
                                              float ux, float uy, float uz, float usq, float Gx, float Gy,
                                              float Gz, float omega, float fpre, float sc, uint32_t &rng) {
    constexpr float ex = (float)d3q19_ex(Q), ey = (float)d3q19_ey(Q), ez = (float)d3q19_ez(Q);
    constexpr float w = (float)d3q19_w(Q);
    const float eu = ex * ux + ey * uy + ez * uz;
    const float heq = w * (drho + rho * (3.0f * eu + 4.5f * eu * eu - 1.5f * usq));
    const float eG = ex * Gx + ey * Gy + ez * Gz;
    const float uG = ux * Gx + uy * Gy + uz * Gz;
    const float Fq = w * (3.0f * (eG - uG) + 9.0f * eu * eG);
    const float out = h - omega * (h - heq) + fpre * Fq;
    uint32_t rnd = 0;
    if (sizeof(T) == 2) {  // one linear-congruential step per population
        rng = rng * 747796405u + 2891336453u;
        rnd = rng ^ (rng >> 15);
    }
    PopIO<T>::st(dst + (size_t)Q * nfp + f, out, sc, rnd);
}

template <typename T>
__device__ __forceinline__ void fluid_cell(const SimDev &s, int par, int f, bool active, uint32_t step_seed) {
    const T *__restrict__ src = (const T *)s.pop[par];
    T *__restrict__ dst = (T *)s.pop[par ^ 1];
    const int nfp = s.nfp;
    const float inv = s.inv_scale;
    const int x = f % s.nx;
    const int r = f / s.nx;
    const int y = r % s.nyf;
    const int z = r / s.nyf;
    const Nbr n = neighbours(s, x, y, z);

    float h[NQ];
#define LBIB_PULL(q) h[q] = pull<T, q>(src, nfp, f, n, inv);
    LBIB_PULL(0) LBIB_PULL(1) LBIB_PULL(2) LBIB_PULL(3) LBIB_PULL(4) LBIB_PULL(5) LBIB_PULL(6)
    LBIB_PULL(7) LBIB_PULL(8) LBIB_PULL(9) LBIB_PULL(10) LBIB_PULL(11) LBIB_PULL(12) LBIB_PULL(13)
    LBIB_PULL(14) LBIB_PULL(15) LBIB_PULL(16) LBIB_PULL(17) LBIB_PULL(18)
#undef LBIB_PULL

    float Gx = s.gx, Gy = s.gy, Gz = s.gz;
    if (active) {  // spread force of this step; clear the buffer of the next
        const float4 g = __ldcg(s.G[par] + f);
        Gx += g.x;
        Gy += g.y;
        Gz += g.z;
        s.G[par ^ 1][f] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        drho += h[q];
        jx += (float)d3q19_ex(q) * h[q];
        jy += (float)d3q19_ey(q) * h[q];
        jz += (float)d3q19_ez(q) * h[q];
    }
    const float rho = s.rho0 + drho;
    const float irho = 1.0f / rho;
    const float ux = (jx + 0.5f * Gx) * irho;
    const float uy = (jy + 0.5f * Gy) * irho;
    const float uz = (jz + 0.5f * Gz) * irho;
    const float usq = ux * ux + uy * uy + uz * uz;
    const float om = s.omega, fp = s.fpre, sc = s.scale;
    uint32_t rng = (sizeof(T) == 2) ? mix32((uint32_t)f ^ step_seed) : 0u;
#define LBIB_COLL(q) collide_store<T, q>(dst, nfp, f, h[q], drho, rho, ux, uy, uz, usq, Gx, Gy, Gz, om, fp, sc, rng);
    LBIB_COLL(0) LBIB_COLL(1) LBIB_COLL(2) LBIB_COLL(3) LBIB_COLL(4) LBIB_COLL(5) LBIB_COLL(6)
    LBIB_COLL(7) LBIB_COLL(8) LBIB_COLL(9) LBIB_COLL(10) LBIB_COLL(11) LBIB_COLL(12) LBIB_COLL(13)
    LBIB_COLL(14) LBIB_COLL(15) LBIB_COLL(16) LBIB_COLL(17) LBIB_COLL(18)
#undef LBIB_COLL

    if (active) s.ufield[f] = make_float4(ux, uy, uz, rho);
    if (!(usq < 0.09f)) atomicOr(s.status, ST_UNSTABLE);
}

// Seed of the rounding bits of step t.
__host__ __device__ __forceinline__ uint32_t step_seed(long long t) {
    uint32_t x = (uint32_t)t * 0x9e3779b9u + 0x632be5abu;
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    return x;
}

// The active-cell word of the warp that owns fluid cell f (blocks start at
// multiples of 32, so a warp owns exactly one word).  Read through L2: the
// object update of the same launch may set bits.
__device__ __forceinline__ uint32_t active_word(const SimDev &s, int f) {
    const int w = f >> 5;
    return (w < s.nwords) ? __ldcg(s.amask + w) : 0u;
}

// One block of FLUID_THREADS consecutive fluid cells starting at f0.
template <typename T>
__device__ __forceinline__ void fluid_block(const SimDev &s, int par, int f0, uint32_t step_seed) {
    const int f = f0 + (int)threadIdx.x;
    const uint32_t act = active_word(s, f);
    if (f < s.nf) fluid_cell<T>(s, par, f, (act >> (threadIdx.x & 31)) & 1u, step_seed);
}

}  // namespace lbib
