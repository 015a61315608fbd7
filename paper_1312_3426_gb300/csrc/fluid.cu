// Fluid kernels: fused pull-stream + collide (Eq. lbequation), read-outs,
// checkpoint conversion and the FP64 mass reduction.
//
// One thread updates one fluid cell.  For each of the 19 directions it pulls
// the post-collision value of the previous step from the neighbour the
// population comes from (periodic in x and z, and in y without walls); a
// population that would come from a solid row is the cell's own opposite
// population reflected at the halfway wall (bounce-back of a resting wall).
// It then forms rho = rho0 + sum h, u = (sum h e + G/2)/rho with G = body
// force + the coupling force spread onto this cell, relaxes towards the
// equilibrium with rate 1/tau (BGK) and adds Guo's force term
// (1 - 1/(2 tau)) w [3(e - u) + 9 (e.u) e].G.  Everything is carried as the
// deviation h = f - w rho0 so that FP32 (or FP16/BF16 storage) keeps the
// small velocity signal; the arithmetic is FP32.
//
// Memory traffic per fluid cell: 19 loads + 19 stores of the storage type
// (152 B in FP32, 76 B in FP16/BF16), plus one 4-byte mask word per 32
// cells for each of the three masks, plus 16 B reads/writes only at cells
// touched by the immersed objects.
#include <mutex>
#include <type_traits>

#include "fluid_core.cuh"

namespace lbib {

// EARLY: the instantiation for an early (programmatic dependent) launch
template <typename T, bool BC, bool EARLY>
__global__ void __launch_bounds__(FLUID_THREADS, 5) k_fluid(SimDev s, int par, uint32_t seed, int pf) {
    prefetch_sources<sizeof(T), FLUID_THREADS>(s, s.pop[par], pf);
    fluid_block<T, BC, EARLY>(s, par, blockIdx.x * FLUID_THREADS, seed);
}

// 16-bit storage, even nx, no obstacles, no inlet: two cells per thread.
// Blocks of 128 threads (6 per SM at 80 registers): when a membrane block
// shares the SM, one of six fluid blocks gives way instead of one of three.
constexpr int PAIR_THREADS = 128;
template <typename T, bool EARLY>
__global__ void __launch_bounds__(PAIR_THREADS, 6) k_fluid_pair(SimDev s, int par, uint32_t seed, int pf) {
    prefetch_sources<2, 2 * PAIR_THREADS>(s, s.pop[par], pf);
    const int f = 2 * (int)(blockIdx.x * PAIR_THREADS + threadIdx.x);
    if (f < s.nf) fluid_pair<T, EARLY>(s, par, f, seed);
}

static bool pair_shape(const SimDev &s) { return (s.nx & 1) == 0 && !s.solid && !s.in_on; }

// The warp-specialised kernel is opt-in (LBIB_TUNE_FLUID_KERNEL = 2): on
// a GB300 it ran slower than the two-cells kernel with L2 prefetch (0.0947
// vs 0.0882 ms in the step at 256x128x128, 0.764 vs 0.709 ms at
// 512x256x256) and slowed the membrane kernel beside it.
int fluid_kernel_kind(const SimDev &s) {
    if (s.prec == LBIB_POP_F32 || !pair_shape(s) || s.fkern == 3) return 0;
    if (s.fkern == 2 && fluid_tma_shape(s)) return 2;
    return 1;
}

// SM count of the current device (cached per device).
static int device_sms() {
    static std::mutex mu;
    static int sms[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (!sms[dev]) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
    return sms[dev];
}

// Prefetch distances (in blocks), measured at 256x128x128 and 512x256x256
// on a GB300: 1.5 blocks per SM ahead for the one-cell kernel (5 resident
// per SM), 3 per SM for the two-cells kernel (6 resident per SM).
// pdl: the warp-specialised kernel is always launched plainly.
template <typename T>
static cudaError_t launch_fluid_t(const SimDev &s, int par, uint32_t seed, int blocks, cudaStream_t st, bool pdl) {
    const int sms = device_sms();
    if constexpr (sizeof(T) == 2) {
        if (fluid_kernel_kind(s) == 2) {
            launch_fluid_tma(s, par, seed, st);
            return cudaGetLastError();
        }
        if (fluid_kernel_kind(s) == 1) {
            const unsigned pblocks = (unsigned)((s.nf / 2 + PAIR_THREADS - 1) / PAIR_THREADS);
            if (pdl) return launch_dep(k_fluid_pair<T, true>, pblocks, PAIR_THREADS, st, true, s, par, seed, 3 * sms);
            return launch_dep(k_fluid_pair<T, false>, pblocks, PAIR_THREADS, st, false, s, par, seed, 3 * sms);
        }
    }
    const unsigned b = (unsigned)blocks;
    const int pf = 3 * sms / 2;
    if (s.solid || s.in_on) {
        if (pdl) return launch_dep(k_fluid<T, true, true>, b, FLUID_THREADS, st, true, s, par, seed, pf);
        return launch_dep(k_fluid<T, true, false>, b, FLUID_THREADS, st, false, s, par, seed, pf);
    }
    if (pdl) return launch_dep(k_fluid<T, false, true>, b, FLUID_THREADS, st, true, s, par, seed, pf);
    return launch_dep(k_fluid<T, false, false>, b, FLUID_THREADS, st, false, s, par, seed, pf);
}

cudaError_t launch_fluid(const SimDev &s, int par, long long t, cudaStream_t st, bool pdl) {
    const uint32_t seed = step_seed(t);
    const int blocks = (s.nf + FLUID_THREADS - 1) / FLUID_THREADS;
    switch (s.prec) {
        case LBIB_POP_F32: return launch_fluid_t<float>(s, par, seed, blocks, st, pdl);
        case LBIB_POP_F16S: return launch_fluid_t<__half>(s, par, seed, blocks, st, pdl);
        case LBIB_POP_BF16S: return launch_fluid_t<__nv_bfloat16>(s, par, seed, blocks, st, pdl);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------- read-outs

__device__ __forceinline__ int64_t full_index(const SimDev &s, int f) {
    const int x = f % s.nx;
    const int r = f / s.nx;
    const int y = r % s.nyf + (s.walls ? 1 : 0);
    const int z = r / s.nyf;
    return ((int64_t)z * s.ny + y) * s.nx + x;
}

template <typename T>
__device__ __forceinline__ float ld_pop(const SimDev &s, int par, int q, int f) {
    return PopIO<T>::ld((const T *)s.pop[par] + (size_t)q * s.nfp + f, s.inv_scale);
}

// Velocity and density of the last collision from the post-collision
// populations it stored: sum f* e = sum n e + G, so u = (sum f* e - G/2)/rho.
// gmode says which force that collision applied: -1 none (fluid as
// initialised), -2 the body force only (populations set from the host),
// 0 or 1 the body force plus the coupling buffer G[gmode].  The result goes
// to full-box arrays (u [3][nz][ny][nx], rho [nz][ny][nx]) or, with
// to_ufield, to the velocity samples of every fluid cell.
template <typename T>
__global__ void k_fields(SimDev s, int pop_par, int gmode, float *u, float *rho_out, int to_ufield) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= s.nf) return;
    if (s.solid && solid_bit(s, f)) {  // obstacle: no fluid
        if (to_ufield) {
            s.ufield[f] = make_float4(0.f, 0.f, 0.f, 0.f);
            return;
        }
        const int64_t c = full_index(s, f);
        const int64_t ncell = (int64_t)s.nx * s.ny * s.nz;
        if (u) u[c] = u[ncell + c] = u[2 * ncell + c] = 0.f;
        if (rho_out) rho_out[c] = 0.f;
        return;
    }
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float h = ld_pop<T>(s, pop_par, q, f);
        drho += h;
        jx += (float)d3q19_ex(q) * h;
        jy += (float)d3q19_ey(q) * h;
        jz += (float)d3q19_ez(q) * h;
    }
    float Gx = 0.f, Gy = 0.f, Gz = 0.f;
    if (gmode != -1) {
        Gx = s.gx;
        Gy = s.gy;
        Gz = s.gz;
    }
    if (gmode >= 0 && ((s.amask[f >> 5] >> (f & 31)) & 1u)) {
        const float4 g = s.G[gmode][f];
        Gx += g.x;
        Gy += g.y;
        Gz += g.z;
    }
    const float rho = s.rho0 + drho;
    const float ux = (jx - 0.5f * Gx) / rho, uy = (jy - 0.5f * Gy) / rho, uz = (jz - 0.5f * Gz) / rho;
    if (to_ufield) {
        s.ufield[f] = make_float4(ux, uy, uz, rho);
        return;
    }
    const int64_t c = full_index(s, f);
    const int64_t ncell = (int64_t)s.nx * s.ny * s.nz;
    if (u) {
        u[c] = ux;
        u[ncell + c] = uy;
        u[2 * ncell + c] = uz;
    }
    if (rho_out) rho_out[c] = rho;
}

cudaError_t launch_fields(const SimDev &s, int pop_par, int gmode, float *u_full, float *rho_full, int to_ufield,
                          cudaStream_t st) {
    const int blocks = (s.nf + 255) / 256;
    switch (s.prec) {
        case LBIB_POP_F32:
            k_fields<float><<<blocks, 256, 0, st>>>(s, pop_par, gmode, u_full, rho_full, to_ufield);
            break;
        case LBIB_POP_F16S:
            k_fields<__half><<<blocks, 256, 0, st>>>(s, pop_par, gmode, u_full, rho_full, to_ufield);
            break;
        case LBIB_POP_BF16S:
            k_fields<__nv_bfloat16><<<blocks, 256, 0, st>>>(s, pop_par, gmode, u_full, rho_full, to_ufield);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Coupling force of buffer gpar (live entries only) into a full-box array.
__global__ void k_read_coupling(SimDev s, int gpar, float *g) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= s.nf) return;
    if (!((s.amask[f >> 5] >> (f & 31)) & 1u)) return;
    const float4 v = s.G[gpar][f];
    const int64_t c = full_index(s, f);
    const int64_t ncell = (int64_t)s.nx * s.ny * s.nz;
    g[c] = v.x;
    g[ncell + c] = v.y;
    g[2 * ncell + c] = v.z;
}

cudaError_t launch_read_coupling(const SimDev &s, int gpar, float *g, cudaStream_t st) {
    k_read_coupling<<<(s.nf + 255) / 256, 256, 0, st>>>(s, gpar, g);
    return cudaGetLastError();
}

__global__ void k_set_coupling(SimDev s, int gpar, const float *g) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= s.nf) return;
    const int64_t c = full_index(s, f);
    const int64_t ncell = (int64_t)s.nx * s.ny * s.nz;
    const float4 v = make_float4(g[c], g[ncell + c], g[2 * ncell + c], 0.f);
    s.G[gpar][f] = v;
    if (v.x != 0.f || v.y != 0.f || v.z != 0.f) atomicOr(s.amask + (f >> 5), 1u << (f & 31));
}

cudaError_t launch_set_coupling(const SimDev &s, int gpar, const float *g, cudaStream_t st) {
    k_set_coupling<<<(s.nf + 255) / 256, 256, 0, st>>>(s, gpar, g);
    return cudaGetLastError();
}

template <typename T>
__global__ void k_read_pops(SimDev s, int par, double *h) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= s.nf) return;
    const int64_t c = full_index(s, f);
    const int64_t ncell = (int64_t)s.nx * s.ny * s.nz;
    const T *src = (const T *)s.pop[par];
    for (int q = 0; q < NQ; ++q) {
        const float v = (float)PopIO<T>::ld(src + (size_t)q * s.nfp + f, 1.0f);
        h[q * ncell + c] = (double)v * (double)s.inv_scale;
    }
}

template <typename T>
__global__ void k_set_pops(SimDev s, int par, const double *h) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= s.nf) return;
    const int64_t c = full_index(s, f);
    const int64_t ncell = (int64_t)s.nx * s.ny * s.nz;
    T *dst = (T *)s.pop[par];
    for (int q = 0; q < NQ; ++q) {
        const double v = h[q * ncell + c] * (double)s.scale;
        if constexpr (sizeof(T) == 4) {
            dst[(size_t)q * s.nfp + f] = (float)v;
        } else {
            if constexpr (sizeof(T) == 2 && std::is_same<T, __half>::value)
                dst[(size_t)q * s.nfp + f] = __float2half_rn((float)v);
            else
                dst[(size_t)q * s.nfp + f] = __float2bfloat16_rn((float)v);
        }
    }
}

cudaError_t launch_read_pops(const SimDev &s, int par, double *h, cudaStream_t st) {
    const int blocks = (s.nf + 255) / 256;
    switch (s.prec) {
        case LBIB_POP_F32: k_read_pops<float><<<blocks, 256, 0, st>>>(s, par, h); break;
        case LBIB_POP_F16S: k_read_pops<__half><<<blocks, 256, 0, st>>>(s, par, h); break;
        case LBIB_POP_BF16S: k_read_pops<__nv_bfloat16><<<blocks, 256, 0, st>>>(s, par, h); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_set_pops(const SimDev &s, int par, const double *h, cudaStream_t st) {
    const int blocks = (s.nf + 255) / 256;
    switch (s.prec) {
        case LBIB_POP_F32: k_set_pops<float><<<blocks, 256, 0, st>>>(s, par, h); break;
        case LBIB_POP_F16S: k_set_pops<__half><<<blocks, 256, 0, st>>>(s, par, h); break;
        case LBIB_POP_BF16S: k_set_pops<__nv_bfloat16><<<blocks, 256, 0, st>>>(s, par, h); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- mass (FP64)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of all deviations h over fluid cells, FP64: each thread sums its
// cells' 19 values in FP64, a warp shuffle and a shared-memory pass reduce
// the block, one FP64 atomic per block adds it to *acc.
template <typename T>
__global__ void __launch_bounds__(256) k_mass(SimDev s, int par, double *acc) {
    double local = 0.0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < s.nf; f += gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) local += (double)ld_pop<T>(s, par, q, f);
    }
    local = warp_sum(local);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < 8 ? part[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) atomicAdd(acc, v);
    }
}

// Allocation-free variant: each block writes its FP64 partial sum to its own
// slot of a fixed scratch array in the library's static device memory, and
// the host adds the slots in block order (so the result is also
// independent of scheduling).  One scratch array per device per process.
static __device__ __align__(256) double g_mass_scratch[MASS_SCRATCH_SLOTS];

template <typename T>
__global__ void __launch_bounds__(256) k_mass_partials(SimDev s, int par, double *part) {
    double local = 0.0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < s.nf; f += gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) local += (double)ld_pop<T>(s, par, q, f);
    }
    local = warp_sum(local);
    __shared__ double wpart[8];
    if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += wpart[w];
        part[blockIdx.x] = v;  // every slot below gridDim.x is written: nothing to clear
    }
}

cudaError_t mass_scratch(double **ptr) {
    // resolved once per device, with that device current (the caller's)
    static std::mutex mu;
    static double *addr[MASS_SCRATCH_DEVICES] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MASS_SCRATCH_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = (double *)p;
    }
    *ptr = addr[dev];
    return cudaSuccess;
}

cudaError_t launch_mass_partials(const SimDev &s, int par, double *part, int blocks, cudaStream_t st) {
    switch (s.prec) {
        case LBIB_POP_F32: k_mass_partials<float><<<blocks, 256, 0, st>>>(s, par, part); break;
        case LBIB_POP_F16S: k_mass_partials<__half><<<blocks, 256, 0, st>>>(s, par, part); break;
        case LBIB_POP_BF16S: k_mass_partials<__nv_bfloat16><<<blocks, 256, 0, st>>>(s, par, part); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_mass(const SimDev &s, int par, double *acc, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int blocks = sms * 4;
    const int need = (s.nf + 255) / 256;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    switch (s.prec) {
        case LBIB_POP_F32: k_mass<float><<<blocks, 256, 0, st>>>(s, par, acc); break;
        case LBIB_POP_F16S: k_mass<__half><<<blocks, 256, 0, st>>>(s, par, acc); break;
        case LBIB_POP_BF16S: k_mass<__nv_bfloat16><<<blocks, 256, 0, st>>>(s, par, acc); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace lbib
