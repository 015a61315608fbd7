// Device-side body of the fused fluid update (Eq. lbequation), shared by the
// single-simulation kernel (fluid.cu) and the batched persistent kernel
// (batch.cu).  See fluid.cu for the description of the update.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbib_internal.h"

namespace lbib {

// Storage of one population.  FP32 is stored as is.  FP16/BF16 store the
// deviation times 2^s with stochastic rounding: the conversion moves to the
// neighbouring representable value of larger magnitude with probability
// equal to the dropped fraction of a unit in the last place, so the stored
// value is unbiased.  Rounding to nearest would turn
// the per-step forcing increment, which is far below one unit in the last
// place of a 16-bit number once the flow has built up, into a systematic
// error.  The rounding is the hardware's (cvt.rs, which converts two FP32
// numbers into a packed pair with 32 random bits); the random bits come
// from a counter-based hash of (cell, step) stepped by a linear
// congruential generator across the directions, so results are
// reproducible.
//
// PopIO::ld reads a deviation (read-outs and reductions); Raw below is the
// step kernel's access to the stored numbers themselves.
template <typename T>
struct PopIO;

template <>
struct PopIO<float> {
    static __device__ __forceinline__ float ld(const float *p, float) { return __ldg(p); }
};
template <>
struct PopIO<__half> {
    static __device__ __forceinline__ float ld(const __half *p, float inv) { return __half2float(__ldg(p)) * inv; }
};
template <>
struct PopIO<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p, float inv) {
        return __bfloat162float(__ldg(p)) * inv;
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

// Two FP32 numbers to a packed pair of 16-bit numbers (lo in the low half)
// with stochastic rounding; r supplies the random bits of both.  Beyond the
// largest finite number the result saturates.
template <typename T>
struct Pack2;
template <>
struct Pack2<__half> {
    static __device__ __forceinline__ uint32_t rs(float lo, float hi, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
};
template <>
struct Pack2<__nv_bfloat16> {
    static __device__ __forceinline__ uint32_t rs(float lo, float hi, uint32_t r) {
        uint32_t d;
        asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
        return d;
    }
};

// Raw storage access for the step kernel: the stored number as float (the
// deviation times 2^s for FP16/BF16), and the store of two such numbers at
// two addresses, rounded together with the random bits r.
template <typename T>
struct Raw;
template <>
struct Raw<float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void st2(float *p, float *q, float a, float b, uint32_t) {
        __stcs(p, a);
        __stcs(q, b);
    }
};
template <>
struct Raw<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st2(__half *p, __half *q, float a, float b, uint32_t r) {
        const uint32_t d = Pack2<__half>::rs(a, b, r);
        __stcs((unsigned short *)p, (unsigned short)d);
        __stcs((unsigned short *)q, (unsigned short)(d >> 16));
    }
};
template <>
struct Raw<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) {
        return __uint_as_float((uint32_t)__ldg((const unsigned short *)p) << 16);
    }
    static __device__ __forceinline__ void st2(__nv_bfloat16 *p, __nv_bfloat16 *q, float a, float b, uint32_t r) {
        const uint32_t d = Pack2<__nv_bfloat16>::rs(a, b, r);
        __stcs((unsigned short *)p, (unsigned short)d);
        __stcs((unsigned short *)q, (unsigned short)(d >> 16));
    }
};

// Pull the (raw) population of direction Q arriving at cell f.  In the
// boundary-condition variant (BC) a population coming from an obstacle cell
// is the cell's own opposite one, as at the walls.
template <typename T, int Q, bool BC>
__device__ __forceinline__ float pull(const SimDev &s, const T *__restrict__ src, uint32_t nfp, uint32_t f,
                                      const Nbr &n) {
    constexpr int ex = d3q19_ex(Q), ey = d3q19_ey(Q), ez = d3q19_ez(Q);
    if ((ey == 1 && n.ylo_solid) || (ey == -1 && n.yhi_solid))
        return Raw<T>::ld(src + (uint32_t)d3q19_opp(Q) * nfp + f);
    int g = (int)f;
    if (ex == 1) g += n.dxm;
    if (ex == -1) g += n.dxp;
    if (ey == 1) g += n.dym;
    if (ey == -1) g += n.dyp;
    if (ez == 1) g += n.dzm;
    if (ez == -1) g += n.dzp;
    if (BC && Q != 0 && s.solid && solid_bit(s, g)) return Raw<T>::ld(src + (uint32_t)d3q19_opp(Q) * nfp + f);
    return Raw<T>::ld(src + (uint32_t)Q * nfp + (uint32_t)g);
}

// BGK + Guo update of the opposite pair (Q, Q+1) (e_{Q+1} = -e_Q, same
// weight w), from the split into the parts even and odd in e:
//   out_{Q/Q+1} = (1 - omega) h + w 2^s [A +- B],
//   A = omega (K + 4.5 rho (e.u)^2) + fpre (9 (e.u)(e.G) - 3 u.G),
//   B = 3 omega rho (e.u) + 3 fpre (e.G),   K = drho - 1.5 rho u.u,
// which is h - omega (h - h_eq) + fpre w [3 (e - u) + 9 (e.u) e].G written
// out for both directions (2^s: raw storage units).  Per cell the
// constants Kb = omega K - 3 fpre u.G and Rb = 3 omega rho are formed once;
// per weight class (wsc = w 2^s) Kc = wsc Kb, Rc = wsc Rb, R15 = 1.5 Rc
// and Gc = 3 fpre wsc G.  As 4.5 omega rho = 1.5 Rb, a pair then costs
//   w 2^s B = Rc (e.u) + e.Gc,   w 2^s A = Kc + (e.u) (R15 (e.u) + 3 e.Gc).
// A does not reuse the rounded B (A = Kc + 1.5 (e.u) (B + e.Gc) is the same
// number in exact arithmetic): that product of e.u with a rounded multiple
// of e.u has a rounding error of one sign, which drifted the total mass of
// a 512x256x256 channel with 16-bit storage by 7.6e-6 in 20,000 steps.
struct Coll {
    float ux, uy, uz, Gx, Gy, Gz, Kb, Rb;
};
struct Cls {
    float K, R, R15, gx, gy, gz;
};
struct CollK {
    float om, c1, fp3, om3;
};

// e component E (-1, 0, 1) times v without a multiply; the zero is -0.0f,
// which the compiler drops from a sum (x + -0 = x for every x), so the
// dot products and moment sums below carry only their non-zero terms.
template <int E>
__device__ __forceinline__ float eterm(float v) {
    if constexpr (E == 1) return v;
    else if constexpr (E == -1) return -v;
    else return -0.0f;
}
template <int Q>
__device__ __forceinline__ float edot(float x, float y, float z) {
    return eterm<d3q19_ex(Q)>(x) + eterm<d3q19_ey(Q)>(y) + eterm<d3q19_ez(Q)>(z);
}

// Moments sum h and sum h e from the opposite pairs: h_Q + h_{Q+1} and
// h_Q - h_{Q+1} for Q = 1, 3, ..., 17.
struct Moments {
    float r, x, y, z;
};
template <int Q>
__device__ __forceinline__ void add_pair(Moments &m, float hq, float ho) {
    const float d = hq - ho;
    m.r += hq + ho;
    m.x += eterm<d3q19_ex(Q)>(d);
    m.y += eterm<d3q19_ey(Q)>(d);
    m.z += eterm<d3q19_ez(Q)>(d);
}
__device__ __forceinline__ Moments moments19(const float (&h)[NQ]) {
    Moments m{h[0], -0.0f, -0.0f, -0.0f};
    add_pair<1>(m, h[1], h[2]);
    add_pair<3>(m, h[3], h[4]);
    add_pair<5>(m, h[5], h[6]);
    add_pair<7>(m, h[7], h[8]);
    add_pair<9>(m, h[9], h[10]);
    add_pair<11>(m, h[11], h[12]);
    add_pair<13>(m, h[13], h[14]);
    add_pair<15>(m, h[15], h[16]);
    add_pair<17>(m, h[17], h[18]);
    return m;
}

// The constants of one weight class (wsc = w 2^s).
__device__ __forceinline__ Cls make_cls(const Coll &c, const CollK &k, float wsc) {
    const float g = k.fp3 * wsc, R = wsc * c.Rb;
    return Cls{wsc * c.Kb, R, 1.5f * R, g * c.Gx, g * c.Gy, g * c.Gz};
}

// w 2^s (A + B, A - B) for the opposite pair (Q, Q+1) of one cell.
template <int Q>
__device__ __forceinline__ float2 pair_terms(const Coll &c, const Cls &w) {
    const float eu = edot<Q>(c.ux, c.uy, c.uz);
    const float eg = edot<Q>(w.gx, w.gy, w.gz);
    const float B = fmaf(w.R, eu, eg);
    const float A = fmaf(eu, fmaf(w.R15, eu, 3.0f * eg), w.K);
    return make_float2(A + B, A - B);
}

template <typename T, int Q>
__device__ __forceinline__ void collide_pair(T *__restrict__ dst, uint32_t nfp, uint32_t f, float hq, float ho,
                                             const Coll &c, const CollK &k, const Cls &w, uint32_t rnd) {
    const float2 ab = pair_terms<Q>(c, w);
    Raw<T>::st2(dst + (uint32_t)Q * nfp + f, dst + (uint32_t)(Q + 1) * nfp + f, fmaf(k.c1, hq, ab.x),
                fmaf(k.c1, ho, ab.y), rnd);
}

// Collision constants of one cell from the raw moments.
__device__ __forceinline__ Coll make_coll(const SimDev &s, const CollK &k, float sr, float sx, float sy, float sz,
                                          float Gx, float Gy, float Gz, float &rho, float &usq) {
    const float inv = s.inv_scale;
    const float drho = sr * inv;
    rho = s.rho0 + drho;
    const float irho = __fdividef(1.0f, rho);  // rho is near 1: the fast reciprocal is within 2 ulp
    Coll c;
    c.ux = fmaf(0.5f, Gx, sx * inv) * irho;
    c.uy = fmaf(0.5f, Gy, sy * inv) * irho;
    c.uz = fmaf(0.5f, Gz, sz * inv) * irho;
    c.Gx = Gx;
    c.Gy = Gy;
    c.Gz = Gz;
    usq = c.ux * c.ux + c.uy * c.uy + c.uz * c.uz;
    const float uG = c.ux * Gx + c.uy * Gy + c.uz * Gz;
    const float K = fmaf(-1.5f * rho, usq, drho);
    c.Kb = fmaf(k.om, K, -k.fp3 * uG);
    c.Rb = k.om3 * rho;
    return c;
}

__device__ __forceinline__ CollK make_collk(const SimDev &s) {
    CollK k;
    k.om = s.omega;
    k.c1 = 1.0f - s.omega;
    k.fp3 = 3.0f * s.fpre;
    k.om3 = 3.0f * s.omega;
    return k;
}

// Velocity inlet (the inflow plane of the Sec. 6 example, whose velocity is
// set before every step): the populations pulled into an inlet cell are
// replaced by the equilibrium at the cell's own density and the prescribed
// velocity, w (drho + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u.u)) in deviation
// form, before the collision.  h holds raw numbers (times 2^s).
template <int Q>
__device__ __forceinline__ float inlet_eq(float drho, float rho, float usq, const float *u, float sc) {
    const float eu = edot<Q>(u[0], u[1], u[2]);
    return (float)d3q19_w(Q) * sc * (drho + rho * (3.0f * eu + 4.5f * eu * eu - 1.5f * usq));
}

__device__ __forceinline__ void inlet_cell(const SimDev &s, int x, int yl, int z, float (&h)[NQ]) {
    const int *b = s.in_box;
    if (x < b[0] || x >= b[1] || yl < b[2] || yl >= b[3] || z < b[4] || z >= b[5]) return;
    float sr = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) sr += h[q];
    const float drho = sr * s.inv_scale, rho = s.rho0 + drho, sc = s.scale;
    const float *u = s.in_u;
    const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    h[0] = inlet_eq<0>(drho, rho, usq, u, sc);
    h[1] = inlet_eq<1>(drho, rho, usq, u, sc);
    h[2] = inlet_eq<2>(drho, rho, usq, u, sc);
    h[3] = inlet_eq<3>(drho, rho, usq, u, sc);
    h[4] = inlet_eq<4>(drho, rho, usq, u, sc);
    h[5] = inlet_eq<5>(drho, rho, usq, u, sc);
    h[6] = inlet_eq<6>(drho, rho, usq, u, sc);
    h[7] = inlet_eq<7>(drho, rho, usq, u, sc);
    h[8] = inlet_eq<8>(drho, rho, usq, u, sc);
    h[9] = inlet_eq<9>(drho, rho, usq, u, sc);
    h[10] = inlet_eq<10>(drho, rho, usq, u, sc);
    h[11] = inlet_eq<11>(drho, rho, usq, u, sc);
    h[12] = inlet_eq<12>(drho, rho, usq, u, sc);
    h[13] = inlet_eq<13>(drho, rho, usq, u, sc);
    h[14] = inlet_eq<14>(drho, rho, usq, u, sc);
    h[15] = inlet_eq<15>(drho, rho, usq, u, sc);
    h[16] = inlet_eq<16>(drho, rho, usq, u, sc);
    h[17] = inlet_eq<17>(drho, rho, usq, u, sc);
    h[18] = inlet_eq<18>(drho, rho, usq, u, sc);
}

// FP32 storage: the same BGK + Guo update written as an increment,
// out = h + Delta, where every part of Delta is formed from quantities that
// are small when the cell is near equilibrium, and the only rounding at the
// scale of h is the final addition.  Per opposite pair (Q, Q+1), with
// a = (h_Q - h_Q+1)/2, m = (h_Q + h_Q+1)/2 and j = sum h e (the momentum
// of the stored deviations, without the force):
//   odd   D_o = omega (3w e.j - a) + 3w e.G        (omega/2 + fpre = 1)
//   even  D_e = omega (w (K + 4.5 rho (e.u)^2) - m) + fpre w (9 (e.u)(e.G) - 3 u.G)
//   out_Q = h_Q + (D_e + D_o),  out_Q+1 = h_Q+1 + (D_e - D_o),
// and for the rest population out_0 = h_0 + omega (w0 K - h_0) - 3 fpre w0 u.G,
// with u = (j + G/2)/rho and K = drho - 1.5 rho u.u.  The product 3w e.j
// and the subtraction of a are one FMA (a single rounding at the scale of
// the non-equilibrium part), and 3w (1/6, 1/12) is applied as an unevaluated
// FP32 pair hi + lo: FP32 rounding of 1/6 alone changes every cell's
// momentum in the same direction by 3e-8 of itself per step, which the
// driven channel integrates into a relative velocity bias ~200 times
// larger.  Likewise the force is not added into j before it is rounded:
// adding the same small G/2 to every cell's j rounds the same way in every
// cell of a binade.
struct Inc {
    float sx, sy, sz;      // j
    float ux, uy, uz;      // u
    float Gx, Gy, Gz;      // force density of this step
    float K, r45, m3uG;    // K, 4.5 rho, -3 u.G
    float om, fpre;
};

constexpr double INC_C1 = 1.0 / 6.0;   // 3 w for |e|^2 = 1
constexpr float INC_C1_HI = (float)INC_C1;
constexpr float INC_C1_LO = (float)(INC_C1 - (double)INC_C1_HI);

template <int Q>
__device__ __forceinline__ void inc_pair(float *__restrict__ dst, uint32_t nfp, uint32_t f, float hq, float ho,
                                         const Inc &c) {
    constexpr bool axis = Q < 7;  // |e|^2 = 1; else 2 (weight and 3w halved, exactly)
    constexpr float wq = axis ? (float)(1.0 / 18.0) : (float)(1.0 / 36.0);
    constexpr float chi = axis ? INC_C1_HI : 0.5f * INC_C1_HI, clo = axis ? INC_C1_LO : 0.5f * INC_C1_LO;
    const float a = 0.5f * __fsub_rn(hq, ho), m = 0.5f * __fadd_rn(hq, ho);
    const float ej = edot<Q>(c.sx, c.sy, c.sz);
    const float eu = edot<Q>(c.ux, c.uy, c.uz);
    const float eG = edot<Q>(c.Gx, c.Gy, c.Gz);
    float t = __fmaf_rn(chi, ej, -a);
    t = __fmaf_rn(clo, ej, t);
    const float Do = __fmaf_rn(c.om, t, __fmaf_rn(chi, eG, __fmul_rn(clo, eG)));
    const float Aeq = __fmaf_rn(__fmul_rn(c.r45, wq), __fmul_rn(eu, eu), __fmul_rn(wq, c.K));
    const float Fe = __fmul_rn(__fmul_rn(c.fpre, wq), __fmaf_rn(__fmul_rn(9.0f, eu), eG, c.m3uG));
    const float De = __fmaf_rn(c.om, __fsub_rn(Aeq, m), Fe);
    __stcs(dst + (uint32_t)Q * nfp + f, __fadd_rn(hq, __fadd_rn(De, Do)));
    __stcs(dst + (uint32_t)(Q + 1) * nfp + f, __fadd_rn(ho, __fsub_rn(De, Do)));
}

// The increment-form collision and store of one FP32 cell from its pulled
// populations h; returns u.u (the stability check) and sets u, rho.
__device__ __forceinline__ float collide_increment(const SimDev &s, float *__restrict__ dst, uint32_t nfp, uint32_t f,
                                                   const float (&h)[NQ], float Gx, float Gy, float Gz, float &ux,
                                                   float &uy, float &uz, float &rho) {
    const Moments mo = moments19(h);
    Inc c;
    c.om = s.omega;
    c.fpre = s.fpre;
    c.sx = mo.x;
    c.sy = mo.y;
    c.sz = mo.z;
    c.Gx = Gx;
    c.Gy = Gy;
    c.Gz = Gz;
    const float drho = mo.r;
    rho = s.rho0 + drho;
    const float irho = __fdividef(1.0f, rho);  // rho is near 1: the fast reciprocal is within 2 ulp
    ux = fmaf(0.5f, Gx, mo.x) * irho;
    uy = fmaf(0.5f, Gy, mo.y) * irho;
    uz = fmaf(0.5f, Gz, mo.z) * irho;
    c.ux = ux;
    c.uy = uy;
    c.uz = uz;
    const float usq = ux * ux + uy * uy + uz * uz;
    c.m3uG = -3.0f * (ux * Gx + uy * Gy + uz * Gz);
    c.K = fmaf(-1.5f * rho, usq, drho);
    c.r45 = 4.5f * rho;
    constexpr float w0 = (float)(1.0 / 3.0);
    const float h0 = h[0];
    __stcs(dst + f, __fadd_rn(h0, __fmaf_rn(c.om, __fmaf_rn(w0, c.K, -h0), __fmul_rn(c.fpre * w0, c.m3uG))));
    inc_pair<1>(dst, nfp, f, h[1], h[2], c);
    inc_pair<3>(dst, nfp, f, h[3], h[4], c);
    inc_pair<5>(dst, nfp, f, h[5], h[6], c);
    inc_pair<7>(dst, nfp, f, h[7], h[8], c);
    inc_pair<9>(dst, nfp, f, h[9], h[10], c);
    inc_pair<11>(dst, nfp, f, h[11], h[12], c);
    inc_pair<13>(dst, nfp, f, h[13], h[14], c);
    inc_pair<15>(dst, nfp, f, h[15], h[16], c);
    inc_pair<17>(dst, nfp, f, h[17], h[18], c);
    return usq;
}

// BC: the variant for simulations with obstacles or a velocity inlet (the
// plain variant carries no test for either).
// The active-cell word of the warp that owns fluid cell f (blocks start at
// multiples of 32, so a warp owns exactly one word).  Read through L2: the
// object update of the same launch may set bits.
__device__ __forceinline__ uint32_t active_word(const SimDev &s, int f) {
    const int w = f >> 5;
    return (w < s.nwords) ? __ldcg(s.amask + w) : 0u;
}

// EARLY: the kernel may be launched early (programmatic dependent launch):
// the mask word is read after dep_wait(); otherwise it is `act`, read by the
// caller before the pulls.
template <typename T, bool BC, bool EARLY>
__device__ __forceinline__ void fluid_cell(const SimDev &s, int par, int fi, uint32_t act, uint32_t step_seed) {
    static_assert(d3q19_opp(1) == 2 && d3q19_opp(17) == 18, "directions 2k-1, 2k must be opposite");
    const T *__restrict__ src = (const T *)s.pop[par];
    T *__restrict__ dst = (T *)s.pop[par ^ 1];
    const uint32_t nfp = (uint32_t)s.nfp, f = (uint32_t)fi;
    if (BC && s.solid && solid_bit(s, fi)) return;  // an obstacle cell holds no fluid
    const uint32_t r = s.div_nx.div(f);
    const uint32_t x = f - r * (uint32_t)s.nx;
    const uint32_t z = s.div_nyf.div(r);
    const uint32_t y = r - z * (uint32_t)s.nyf;
    const Nbr n = neighbours(s, (int)x, (int)y, (int)z);

    float h[NQ];
#define LBIB_PULL(q) h[q] = pull<T, q, BC>(s, src, nfp, f, n);
    LBIB_PULL(0) LBIB_PULL(1) LBIB_PULL(2) LBIB_PULL(3) LBIB_PULL(4) LBIB_PULL(5) LBIB_PULL(6)
    LBIB_PULL(7) LBIB_PULL(8) LBIB_PULL(9) LBIB_PULL(10) LBIB_PULL(11) LBIB_PULL(12) LBIB_PULL(13)
    LBIB_PULL(14) LBIB_PULL(15) LBIB_PULL(16) LBIB_PULL(17) LBIB_PULL(18)
#undef LBIB_PULL

    if (BC && s.in_on) inlet_cell(s, (int)x, (int)y + s.walls, (int)z, h);
    // the populations pulled above were written by the previous fluid step;
    // the mask and the coupling buffer below by the node update of this one
    if constexpr (EARLY) {
        dep_wait();
        dep_release();
        act = active_word(s, fi);
    }
    const bool active = (act >> (fi & 31)) & 1u;

    float Gx = s.gx, Gy = s.gy, Gz = s.gz;
    if (active) {  // spread force of this step; clear the buffer of the next
        const float4 g = __ldcg(s.G[par] + f);
        Gx += g.x;
        Gy += g.y;
        Gz += g.z;
        s.G[par ^ 1][f] = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    if constexpr (sizeof(T) == 4) {
        float ux, uy, uz, rho;
        const float usq = collide_increment(s, (float *)dst, nfp, f, h, Gx, Gy, Gz, ux, uy, uz, rho);
        if (active) s.ufield[f] = make_float4(ux, uy, uz, rho);
        if (!(usq < 0.09f)) atomicOr(s.status, ST_UNSTABLE);
        return;
    }

    // moments of the raw numbers, then back to deviations (exact: 2^-s)
    const Moments m = moments19(h);
    const CollK k = make_collk(s);
    float rho, usq;
    const Coll c = make_coll(s, k, m.r, m.x, m.y, m.z, Gx, Gy, Gz, rho, usq);
    const float sc = s.scale;
    const float wsc0 = (float)d3q19_w(0) * sc;
    const Cls w1 = make_cls(c, k, (float)d3q19_w(1) * sc);
    const Cls w2 = make_cls(c, k, (float)d3q19_w(7) * sc);

    // 32 random bits per rounded pair of populations for FP16/BF16 (one
    // step of a linear congruential generator each)
    uint32_t rng = (sizeof(T) == 2) ? mix32(f ^ step_seed) : 0u;
    auto next = [&]() -> uint32_t {
        if (sizeof(T) != 2) return 0u;
        rng = rng * 747796405u + 2891336453u;
        return rng ^ (rng >> 15);
    };
    const float out0 = fmaf(k.c1, h[0], wsc0 * c.Kb);
    if constexpr (sizeof(T) == 2) {  // the rest population alone: the high half is discarded
        const uint32_t d = Pack2<T>::rs(out0, 0.0f, next());
        __stcs((unsigned short *)(dst + f), (unsigned short)d);
    } else {
        __stcs((float *)(dst + f), out0);
    }
    collide_pair<T, 1>(dst, nfp, f, h[1], h[2], c, k, w1, next());
    collide_pair<T, 3>(dst, nfp, f, h[3], h[4], c, k, w1, next());
    collide_pair<T, 5>(dst, nfp, f, h[5], h[6], c, k, w1, next());
    collide_pair<T, 7>(dst, nfp, f, h[7], h[8], c, k, w2, next());
    collide_pair<T, 9>(dst, nfp, f, h[9], h[10], c, k, w2, next());
    collide_pair<T, 11>(dst, nfp, f, h[11], h[12], c, k, w2, next());
    collide_pair<T, 13>(dst, nfp, f, h[13], h[14], c, k, w2, next());
    collide_pair<T, 15>(dst, nfp, f, h[15], h[16], c, k, w2, next());
    collide_pair<T, 17>(dst, nfp, f, h[17], h[18], c, k, w2, next());

    if (active) s.ufield[f] = make_float4(c.ux, c.uy, c.uz, rho);
    if (!(usq < 0.09f)) atomicOr(s.status, ST_UNSTABLE);
}

// ------------------------------------------------------------------
// Two cells per thread for 16-bit storage (nx even, no obstacles, no inlet).
// A thread owns cells f and f+1 (f even, same row).  Populations of the
// two cells sit next to each other in every plane, so the pair is read as
// one 32-bit word where the source is even (directions without an x
// component, bounce-back) and as two 16-bit words at adjacent addresses
// otherwise, and always written as one 32-bit word; the index, neighbour
// and address arithmetic and the random bits are shared by the two cells.

template <typename T>
struct Half2Bits;
template <>
struct Half2Bits<__half> {
    static __device__ __forceinline__ float lo(uint32_t u) { return __half2float(__ushort_as_half((unsigned short)u)); }
    static __device__ __forceinline__ float hi(uint32_t u) {
        return __half2float(__ushort_as_half((unsigned short)(u >> 16)));
    }
};
template <>
struct Half2Bits<__nv_bfloat16> {
    static __device__ __forceinline__ float lo(uint32_t u) { return __uint_as_float(u << 16); }
    static __device__ __forceinline__ float hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
};

// The pair of direction Q arriving at cells f, f+1 (low half: cell f).
// dxm0: x-1 offset of cell f (wraps at x = 0); dxp1: x+1 offset of cell f+1
// (wraps at x+1 = nx-1).  Marking these loads evict-first in L2 kept the
// velocity and force fields for the node update that follows (20.7 -> 18.2
// us at 256x128x128) but slowed the kernel 6% at 512x256x256, where the
// x-shifted lines shared by neighbouring warps were evicted in between; the
// loads keep the default policy.
template <int Q>
__device__ __forceinline__ uint32_t pull2(const uint16_t *__restrict__ src, uint32_t nfp, uint32_t f, const Nbr &n,
                                          int dxm0, int dxp1) {
    constexpr int ex = d3q19_ex(Q), ey = d3q19_ey(Q), ez = d3q19_ez(Q);
    if ((ey == 1 && n.ylo_solid) || (ey == -1 && n.yhi_solid))
        return __ldg((const unsigned int *)(src + (uint32_t)d3q19_opp(Q) * nfp + f));
    int g = (int)f;
    if (ey == 1) g += n.dym;
    if (ey == -1) g += n.dyp;
    if (ez == 1) g += n.dzm;
    if (ez == -1) g += n.dzp;
    const uint16_t *p = src + (uint32_t)Q * nfp;
    if (ex == 0) return __ldg((const unsigned int *)(p + (uint32_t)g));  // g even
    if (ex == 1)  // cell f from x-1, cell f+1 from x
        return (uint32_t)__ldg((const unsigned short *)(p + (uint32_t)(g + dxm0))) |
               ((uint32_t)__ldg((const unsigned short *)(p + (uint32_t)g)) << 16);
    // ex == -1: cell f from x+1, cell f+1 from x+2 (or the row start)
    return (uint32_t)__ldg((const unsigned short *)(p + (uint32_t)(g + 1))) |
           ((uint32_t)__ldg((const unsigned short *)(p + (uint32_t)(g + 1 + dxp1))) << 16);
}

// The arithmetic of the two cells runs in packed FP32 instructions (sm_100
// family: one instruction updates both cells, each component rounded as the
// scalar instruction would round it); x holds cell f, y cell f+1.
__device__ __forceinline__ float2 v2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, v2(-1.0f), a); }  // b * -1 is exact
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// s + E v, E = +-1
template <int E>
__device__ __forceinline__ float2 acc2(float2 s, float2 v) {
    static_assert(E == 1 || E == -1, "unit component");
    if constexpr (E == 1) return add2(s, v);
    else return sub2(s, v);
}

// e_Q . v for a pair representative Q (odd Q: its first non-zero component
// is +1), with only the non-zero terms.
template <int Q>
__device__ __forceinline__ float2 edot2(float2 x, float2 y, float2 z) {
    constexpr int ex = d3q19_ex(Q), ey = d3q19_ey(Q), ez = d3q19_ez(Q);
    static_assert(Q % 2 == 1, "pair representative");
    if constexpr (ex != 0) {
        static_assert(ex == 1, "leading +1");
        float2 s = x;
        if constexpr (ey != 0) s = acc2<ey>(s, y);
        if constexpr (ez != 0) s = acc2<ez>(s, z);
        return s;
    } else if constexpr (ey != 0) {
        static_assert(ey == 1, "leading +1");
        if constexpr (ez != 0) return acc2<ez>(y, z);
        else return y;
    } else {
        static_assert(ez == 1, "leading +1");
        return z;
    }
}

template <typename T>
__device__ __forceinline__ float2 unpack2(uint32_t u) {
    return make_float2(Half2Bits<T>::lo(u), Half2Bits<T>::hi(u));
}

struct Moments2 {
    float2 r, x, y, z;
};
// the difference h_Q - h_{Q+1} of pair Q into the momentum sums
template <int Q>
__device__ __forceinline__ void add_diff2(Moments2 &m, float2 d) {
    if constexpr (d3q19_ex(Q) != 0) m.x = acc2<d3q19_ex(Q)>(m.x, d);
    if constexpr (d3q19_ey(Q) != 0) m.y = acc2<d3q19_ey(Q)>(m.y, d);
    if constexpr (d3q19_ez(Q) != 0) m.z = acc2<d3q19_ez(Q)>(m.z, d);
}
// The moments of both cells: sum h from the pair sums, sum h e from the
// pair differences; the axis pairs (1, 3, 5) open the x, y, z sums.
template <typename T>
__device__ __forceinline__ Moments2 moments2(const uint32_t (&P)[NQ]) {
    static_assert(d3q19_ex(1) == 1 && d3q19_ey(3) == 1 && d3q19_ez(5) == 1, "axis pairs 1, 3, 5");
    Moments2 m;
    float2 a = unpack2<T>(P[1]), b = unpack2<T>(P[2]);
    m.r = add2(unpack2<T>(P[0]), add2(a, b));
    m.x = sub2(a, b);
    a = unpack2<T>(P[3]), b = unpack2<T>(P[4]);
    m.r = add2(m.r, add2(a, b));
    m.y = sub2(a, b);
    a = unpack2<T>(P[5]), b = unpack2<T>(P[6]);
    m.r = add2(m.r, add2(a, b));
    m.z = sub2(a, b);
#define LBIB_M2(q)                          \
    a = unpack2<T>(P[q]), b = unpack2<T>(P[q + 1]); \
    m.r = add2(m.r, add2(a, b));            \
    add_diff2<q>(m, sub2(a, b));
    LBIB_M2(7) LBIB_M2(9) LBIB_M2(11) LBIB_M2(13) LBIB_M2(15) LBIB_M2(17)
#undef LBIB_M2
    return m;
}

// Coll, Cls of both cells
struct Coll2 {
    float2 ux, uy, uz, Gx, Gy, Gz, Kb, Rb;
};
struct Cls2 {
    float2 K, R, R15, gx, gy, gz;
};

__device__ __forceinline__ Coll2 make_coll2(const SimDev &s, const CollK &k, const Moments2 &m, float2 Gx, float2 Gy,
                                            float2 Gz, float2 &rho, float2 &usq) {
    const float2 inv = v2(s.inv_scale), half = v2(0.5f);
    const float2 drho = mul2(m.r, inv);
    rho = add2(drho, v2(s.rho0));
    // rho is near 1: the fast reciprocal is within 2 ulp
    const float2 irho = make_float2(__fdividef(1.0f, rho.x), __fdividef(1.0f, rho.y));
    Coll2 c;
    c.ux = mul2(fma2(half, Gx, mul2(m.x, inv)), irho);
    c.uy = mul2(fma2(half, Gy, mul2(m.y, inv)), irho);
    c.uz = mul2(fma2(half, Gz, mul2(m.z, inv)), irho);
    c.Gx = Gx;
    c.Gy = Gy;
    c.Gz = Gz;
    usq = fma2(c.uz, c.uz, fma2(c.uy, c.uy, mul2(c.ux, c.ux)));
    const float2 uG = fma2(c.uz, Gz, fma2(c.uy, Gy, mul2(c.ux, Gx)));
    const float2 K = fma2(mul2(v2(-1.5f), rho), usq, drho);
    c.Kb = fma2(v2(k.om), K, mul2(v2(-k.fp3), uG));
    c.Rb = mul2(v2(k.om3), rho);
    return c;
}

__device__ __forceinline__ Cls2 make_cls2(const Coll2 &c, const CollK &k, float wsc) {
    const float2 g = v2(k.fp3 * wsc), w = v2(wsc);
    const float2 R = mul2(w, c.Rb);
    return Cls2{mul2(w, c.Kb), R, mul2(v2(1.5f), R), mul2(g, c.Gx), mul2(g, c.Gy), mul2(g, c.Gz)};
}

// pair_terms for both cells
template <int Q>
__device__ __forceinline__ void pair_terms2(const Coll2 &c, const Cls2 &w, float2 &ApB, float2 &AmB) {
    const float2 eu = edot2<Q>(c.ux, c.uy, c.uz);
    const float2 eg = edot2<Q>(w.gx, w.gy, w.gz);
    const float2 B = fma2(w.R, eu, eg);
    const float2 A = fma2(eu, fma2(w.R15, eu, mul2(v2(3.0f), eg)), w.K);
    ApB = add2(A, B);
    AmB = sub2(A, B);
}

template <typename T, int Q>
__device__ __forceinline__ void collide2(uint32_t *__restrict__ dst, uint32_t nfp2, uint32_t f2, uint32_t Pq,
                                         uint32_t Po, const Coll2 &c, const CollK &k, const Cls2 &w,
                                         uint32_t &rng) {
    float2 ApB, AmB;
    pair_terms2<Q>(c, w, ApB, AmB);
    const float2 oq = fma2(v2(k.c1), unpack2<T>(Pq), ApB), oo = fma2(v2(k.c1), unpack2<T>(Po), AmB);
    rng = rng * 747796405u + 2891336453u;
    const uint32_t r1 = rng ^ (rng >> 15);
    // The second store takes the same 32 bits with their halves exchanged:
    // each rounding still sees uniform bits (so stays unbiased); only
    // population q of one cell and q-bar of the other share bits, which
    // changes the variance of sums over two cells, not their mean (the
    // 16-bit Poiseuille errors were unchanged: 2.66e-4 FP16, 1.52e-3 BF16).
    const uint32_t r2 = __byte_perm(r1, 0u, 0x1032);
    __stcs((unsigned int *)(dst + (uint32_t)Q * nfp2 + f2), Pack2<T>::rs(oq.x, oq.y, r1));
    __stcs((unsigned int *)(dst + (uint32_t)(Q + 1) * nfp2 + f2), Pack2<T>::rs(oo.x, oo.y, r2));
}

// Collision and store of the cell pair (f, f+1) from its pulled populations
// P (packed pairs, low half: cell f).
// act: the active-cell bits of f (bit 0) and f + 1 (bit 1).
template <typename T>
__device__ __forceinline__ void pair_update_act(const SimDev &s, int par, uint32_t f, const uint32_t (&P)[NQ],
                                                uint32_t step_seed, uint32_t act) {
    uint32_t *__restrict__ dst = (uint32_t *)s.pop[par ^ 1];
    const uint32_t nfp = (uint32_t)s.nfp;
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga;
    if (act & 1u) {  // spread force of this step; clear the buffer of the next
        ga = __ldcg(s.G[par] + f);
        s.G[par ^ 1][f] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (act & 2u) {
        gb = __ldcg(s.G[par] + f + 1);
        s.G[par ^ 1][f + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const CollK k = make_collk(s);
    float2 rho, usq;
    const Moments2 m = moments2<T>(P);
    const Coll2 c = make_coll2(s, k, m, make_float2(s.gx + ga.x, s.gx + gb.x), make_float2(s.gy + ga.y, s.gy + gb.y),
                               make_float2(s.gz + ga.z, s.gz + gb.z), rho, usq);
    const float sc = s.scale;
    const float wsc0 = (float)d3q19_w(0) * sc, wsc1 = (float)d3q19_w(1) * sc, wsc2 = (float)d3q19_w(7) * sc;
    const uint32_t nfp2 = nfp / 2, f2 = f / 2;
    uint32_t rng = mix32(f ^ step_seed);
    rng = rng * 747796405u + 2891336453u;
    const float2 o0 = fma2(v2(k.c1), unpack2<T>(P[0]), mul2(v2(wsc0), c.Kb));
    __stcs((unsigned int *)(dst + f2), Pack2<T>::rs(o0.x, o0.y, rng ^ (rng >> 15)));
    {
        const Cls2 w = make_cls2(c, k, wsc1);
        collide2<T, 1>(dst, nfp2, f2, P[1], P[2], c, k, w, rng);
        collide2<T, 3>(dst, nfp2, f2, P[3], P[4], c, k, w, rng);
        collide2<T, 5>(dst, nfp2, f2, P[5], P[6], c, k, w, rng);
    }
    const Cls2 w = make_cls2(c, k, wsc2);
    collide2<T, 7>(dst, nfp2, f2, P[7], P[8], c, k, w, rng);
    collide2<T, 9>(dst, nfp2, f2, P[9], P[10], c, k, w, rng);
    collide2<T, 11>(dst, nfp2, f2, P[11], P[12], c, k, w, rng);
    collide2<T, 13>(dst, nfp2, f2, P[13], P[14], c, k, w, rng);
    collide2<T, 15>(dst, nfp2, f2, P[15], P[16], c, k, w, rng);
    collide2<T, 17>(dst, nfp2, f2, P[17], P[18], c, k, w, rng);
    if (act & 1u) s.ufield[f] = make_float4(c.ux.x, c.uy.x, c.uz.x, rho.x);
    if (act & 2u) s.ufield[f + 1] = make_float4(c.ux.y, c.uy.y, c.uz.y, rho.y);
    if (!(usq.x < 0.09f) || !(usq.y < 0.09f)) atomicOr(s.status, ST_UNSTABLE);
}

template <typename T>
__device__ __forceinline__ void pair_update(const SimDev &s, int par, uint32_t f, const uint32_t (&P)[NQ],
                                            uint32_t step_seed) {
    pair_update_act<T>(s, par, f, P, step_seed, (__ldcg(s.amask + (f >> 5)) >> (f & 31)) & 3u);
}

template <typename T, bool EARLY>
__device__ __forceinline__ void fluid_pair(const SimDev &s, int par, int fi, uint32_t step_seed) {
    const uint16_t *__restrict__ src = (const uint16_t *)s.pop[par];
    const uint32_t nfp = (uint32_t)s.nfp, f = (uint32_t)fi;
    const uint32_t r = s.div_nx.div(f);
    const uint32_t x = f - r * (uint32_t)s.nx;
    const uint32_t z = s.div_nyf.div(r);
    const uint32_t y = r - z * (uint32_t)s.nyf;
    const Nbr n = neighbours(s, (int)x, (int)y, (int)z);
    const int dxm0 = n.dxm, dxp1 = ((int)x + 2 == s.nx) ? -(s.nx - 1) : 1;

    uint32_t P[NQ];
#define LBIB_PULL2(q) P[q] = pull2<q>(src, nfp, f, n, dxm0, dxp1);
    LBIB_PULL2(0) LBIB_PULL2(1) LBIB_PULL2(2) LBIB_PULL2(3) LBIB_PULL2(4) LBIB_PULL2(5) LBIB_PULL2(6)
    LBIB_PULL2(7) LBIB_PULL2(8) LBIB_PULL2(9) LBIB_PULL2(10) LBIB_PULL2(11) LBIB_PULL2(12) LBIB_PULL2(13)
    LBIB_PULL2(14) LBIB_PULL2(15) LBIB_PULL2(16) LBIB_PULL2(17) LBIB_PULL2(18)
#undef LBIB_PULL2
    if constexpr (EARLY) {  // as in fluid_cell
        dep_wait();
        dep_release();
    }
    pair_update<T>(s, par, f, P, step_seed);
}

// Pull offset of direction q in the fluid index space away from the
// periodic edges and walls: cell f pulls population q from f - e_q.
__host__ __device__ constexpr unsigned long long pack_e(int axis) {
    unsigned long long p = 0;
    for (int q = 0; q < NQ; ++q) {
        const int e = axis == 0 ? d3q19_ex(q) : (axis == 1 ? d3q19_ey(q) : d3q19_ez(q));
        p |= (unsigned long long)(e + 1) << (2 * q);
    }
    return p;
}
__device__ __forceinline__ int unpack_e(unsigned long long p, int q) { return (int)((p >> (2 * q)) & 3ull) - 1; }

// The bulk L2 prefetch of the stretches of every plane that the CELLS cells
// from fb on pull (thread q < 19 takes plane q).
template <int ESZ, int CELLS>
__device__ __forceinline__ void prefetch_cells(const SimDev &s, const void *src, long long fb) {
    if (fb >= s.nf) return;
    const int q = (int)threadIdx.x;
    constexpr unsigned long long PX = pack_e(0), PY = pack_e(1), PZ = pack_e(2);
    const long long off = -((long long)unpack_e(PX, q) + (long long)s.nx * unpack_e(PY, q) +
                            (long long)s.nx * s.nyf * unpack_e(PZ, q));
    long long a = fb + off - 16, b = fb + CELLS + off + 16;
    if (a < 0) a = 0;
    if (b > s.nfp) b = s.nfp;
    if (b <= a) return;
    // 16-byte aligned start and size inside the plane (nfp is a multiple of 64)
    const long long ab = (a * ESZ) & ~15ll;
    long long bb = (b * ESZ + 15) & ~15ll;
    if (bb > (long long)s.nfp * ESZ) bb = (long long)s.nfp * ESZ;
    const char *p = (const char *)src + (long long)q * s.nfp * ESZ + ab;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((unsigned)(bb - ab)) : "memory");
}

// L2 prefetch for a later block: thread q < 19 of block b asks the L2 to
// fetch, with one bulk prefetch, the stretch of plane q that block b + pf
// (of CELLS cells each) will pull, widened by 16 cells on each side and
// clipped to the plane.  The blocks of a launch run roughly in index order,
// so the DRAM requests run ahead of the warps that wait for them.  A
// prefetch is a hint: it changes no result, and cells near the periodic
// edges and walls (whose sources lie elsewhere) are fetched normally.
template <int ESZ, int CELLS>
__device__ __forceinline__ void prefetch_sources(const SimDev &s, const void *src, int pf) {
    if (pf <= 0 || threadIdx.x >= NQ) return;
    prefetch_cells<ESZ, CELLS>(s, src, (long long)(blockIdx.x + pf) * CELLS);
}

// Seed of the rounding bits of step t.
__host__ __device__ __forceinline__ uint32_t step_seed(long long t) {
    uint32_t x = (uint32_t)t * 0x9e3779b9u + 0x632be5abu;
    x ^= x >> 16;
    x *= 0x85ebca6bu;
    x ^= x >> 13;
    return x;
}


// One block of FLUID_THREADS consecutive fluid cells starting at f0.
template <typename T, bool BC, bool EARLY>
__device__ __forceinline__ void fluid_block(const SimDev &s, int par, int f0, uint32_t step_seed) {
    const int f = f0 + (int)threadIdx.x;
    const uint32_t act = EARLY ? 0u : active_word(s, f);
    if (f < s.nf) fluid_cell<T, BC, EARLY>(s, par, f, act, step_seed);
}

}  // namespace lbib
