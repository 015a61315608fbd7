// Warp-specialised two-cells fluid kernel for 16-bit storage (Eq.
// lbequation; the update is the one of fluid_pair in fluid_core.cuh, bit for
// bit): one producer warp streams the populations a tile of cells pulls
// into a ring of shared-memory stages with bulk asynchronous copies, and
// four consumer warps collide and store.  The consumers never wait for DRAM
// directly, and the copies of the next stages are in flight while they
// compute.
//
// Tile: a segment of W cells (W divides nx, W <= 256, W % 8 == 0) of one
// fluid row (y', z).  For each direction q the cells of the segment pull
// from one contiguous segment of plane q: row (y' - e_y, z - e_z) (z, and y
// without walls, periodic), shifted by -e_x; at a wall the population is
// the cell's own opposite one (plane opp(q), the tile's own row, no shift).
// Stage layout, per direction: [8 elements left halo][W elements][8
// elements right halo] (16-bit), the halos being the 16 bytes before and
// after the segment in the row, wrapped at the row ends (periodic x).
// Every copy starts and ends on a 16-byte boundary because nx % 8 == 0.
// Copies per tile: 19 segments and 2 halos for each of the 10 directions
// with e_x != 0; bytes per tile 19 * 2W + 10 * 32, the same for every tile.
//
// Pipeline: full[s] completes when a stage's bytes have landed (producer
// arrive + transaction count); empty[s] completes when the 4 consumer warps
// have read their pairs out of it.  Every wait is bounded (about 2 s by the
// global timer); a wait that runs out sets ST_TIMEOUT in the simulation's
// status word and the thread leaves its loop.  Before the kernel ends the
// producer waits (bounded again) for the copies it issued, so no copy is
// in flight into shared memory when the block exits.
#include <cstdint>
#include <mutex>

#include "fluid_core.cuh"

namespace lbib {

constexpr int TMA_STAGES = 4;
constexpr int TMA_CONSUMERS = 128;  // consumer threads, one cell pair each
constexpr int TMA_THREADS = TMA_CONSUMERS + 32;
constexpr int TMA_MAX_W = 2 * TMA_CONSUMERS;
constexpr int TMA_HALO = 8;  // 16-bit elements (16 bytes)
constexpr int TMA_TILES_PER_BLOCK = 32;
constexpr unsigned long long TMA_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the phase with the given parity of *bar has completed; false
// when the bound (ns of the global timer) ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint64_t bound_ns = TMA_WAIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 255u && global_ns() - t0 > bound_ns) return false;
    }
}

// Check of the bounded wait itself: one thread waits on a barrier that
// nothing arrives at; when the bound runs out it sets ST_TIMEOUT in *status
// and returns, and the context stays usable.  arrive != 0: the thread
// arrives first, so the wait completes at once (the control case).
__global__ void k_wait_probe(uint32_t *status, unsigned long long bound_ns, int arrive) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) mbar_arrive(&bar);
    if (!mbar_wait(&bar, 0, bound_ns)) atomicOr(status, ST_TIMEOUT);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&bar)) : "memory");
}

cudaError_t run_wait_probe(uint32_t *status, unsigned long long bound_ns, int arrive, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(status, bound_ns, arrive);
    return cudaGetLastError();
}

// One bulk copy of `bytes` (a multiple of 16) from global to this block's
// shared memory, completing on *bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

struct TmaTiles {
    int W, segs, ntiles;
    uint32_t tile_bytes;
};

__host__ __device__ constexpr int tma_row_elems(int W) { return W + 2 * TMA_HALO; }

// Producer: lane q < 19 issues the copies of direction q for tile `tile`
// into stage buffer `buf`.
__device__ __forceinline__ void tma_issue(const SimDev &s, const TmaTiles &tt, const uint16_t *src, uint16_t *buf,
                                          int tile, uint64_t *full, int lane) {
    if (lane == 0) mbar_arrive_expect_tx(full, tt.tile_bytes);
    __syncwarp();
    if (lane >= NQ) return;
    const int q = lane;
    constexpr unsigned long long PX = pack_e(0), PY = pack_e(1), PZ = pack_e(2);
    const int ex = unpack_e(PX, q), ey = unpack_e(PY, q), ez = unpack_e(PZ, q);
    const int seg = tile % tt.segs, row = tile / tt.segs;
    const int y = row % s.nyf, z = row / s.nyf;
    const int x0 = seg * tt.W;
    int plane = q, sy = y, sz = z;
    const bool bounce = s.walls && ((ey == 1 && y == 0) || (ey == -1 && y == s.nyf - 1));
    if (bounce) {
        plane = d3q19_opp(q);
    } else {
        sy = y - ey;
        if (sy < 0) sy += s.nyf;  // only without walls
        if (sy >= s.nyf) sy -= s.nyf;
        sz = z - ez;
        if (sz < 0) sz += s.nz;
        if (sz >= s.nz) sz -= s.nz;
    }
    const uint16_t *prow = src + (size_t)plane * s.nfp + (size_t)s.nx * (sy + (size_t)s.nyf * sz);
    uint16_t *dq = buf + q * tma_row_elems(tt.W);
    bulk_g2s(dq + TMA_HALO, prow + x0, 2u * tt.W, full);
    if (ex != 0) {
        const int xl = x0 > 0 ? x0 - TMA_HALO : s.nx - TMA_HALO;
        const int xr = x0 + tt.W < s.nx ? x0 + tt.W : 0;
        bulk_g2s(dq, prow + xl, 2u * TMA_HALO, full);
        bulk_g2s(dq + TMA_HALO + tt.W, prow + xr, 2u * TMA_HALO, full);
    }
}

// Consumer: the packed pair of direction Q for local cells (x, x+1), x even.
template <int Q>
__device__ __forceinline__ uint32_t tma_pull(const uint16_t *buf, int re, int x, bool ylo, bool yhi) {
    constexpr int ex = d3q19_ex(Q), ey = d3q19_ey(Q);
    const uint16_t *r = buf + Q * re + TMA_HALO;
    const bool bounce = (ey == 1 && ylo) || (ey == -1 && yhi);
    if (ex == 0 || bounce) return *(const uint32_t *)(r + x);
    if (ex == 1) return __byte_perm(*(const uint32_t *)(r + x - 2), *(const uint32_t *)(r + x), 0x5432);
    return __byte_perm(*(const uint32_t *)(r + x), *(const uint32_t *)(r + x + 2), 0x5432);
}

template <typename T>
__global__ void __launch_bounds__(TMA_THREADS, 4) k_fluid_pair_tma(SimDev s, int par, uint32_t seed, TmaTiles tt) {
    extern __shared__ __align__(128) unsigned char tma_smem[];
    uint64_t *full = (uint64_t *)tma_smem;
    uint64_t *empty = full + TMA_STAGES;
    uint16_t *stage0 = (uint16_t *)(tma_smem + 128);
    const int re = tma_row_elems(tt.W);
    const int stage_elems = NQ * re;
    const int t0 = blockIdx.x * TMA_TILES_PER_BLOCK;
    const int nt = min(TMA_TILES_PER_BLOCK, tt.ntiles - t0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < TMA_STAGES; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, TMA_CONSUMERS / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const uint16_t *src = (const uint16_t *)s.pop[par];

    if (warp == TMA_CONSUMERS / 32) {  // producer
        int issued = 0;
        for (int i = 0; i < nt; ++i) {
            const int st = i % TMA_STAGES;
            // every lane waits; the warp goes on only together (the copies
            // of a stage are issued by 19 lanes after one warp barrier)
            const bool ok = i < TMA_STAGES || mbar_wait(empty + st, (uint32_t)((i / TMA_STAGES) - 1) & 1u);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) atomicOr(s.status, ST_TIMEOUT);
                break;
            }
            tma_issue(s, tt, src, stage0 + st * stage_elems, t0 + i, full + st, lane);
            issued = i + 1;
        }
        // every copy issued has landed before the block may exit
        for (int i = max(0, issued - TMA_STAGES); i < issued; ++i)
            if (!__all_sync(0xffffffffu, mbar_wait(full + i % TMA_STAGES, (uint32_t)(i / TMA_STAGES) & 1u))) {
                if (lane == 0) atomicOr(s.status, ST_TIMEOUT);
                break;
            }
        return;
    }

    // consumers
    const int x = 2 * (int)threadIdx.x;  // local cell pair (x, x + 1)
    const bool mine = x < tt.W;
    // active-cell bits of the pair of the first tile; the next tile's are
    // read while the current one is computed
    auto active_bits = [&](int tile) -> uint32_t {
        if (!mine || tile >= t0 + nt) return 0u;
        const uint32_t f = (uint32_t)((tile % tt.segs) * tt.W + x + s.nx * (tile / tt.segs));
        return __ldcg(s.amask + (f >> 5)) >> (f & 31);
    };
    uint32_t act_next = active_bits(t0);
    for (int i = 0; i < nt; ++i) {
        const int st = i % TMA_STAGES;
        const uint32_t act = act_next & 3u;
        act_next = active_bits(t0 + i + 1);
        if (!__all_sync(0xffffffffu, mbar_wait(full + st, (uint32_t)(i / TMA_STAGES) & 1u))) {
            if (lane == 0) atomicOr(s.status, ST_TIMEOUT);
            return;
        }
        const int tile = t0 + i;
        const int seg = tile % tt.segs, row = tile / tt.segs;
        const int y = row % s.nyf;
        const bool ylo = s.walls && y == 0, yhi = s.walls && y == s.nyf - 1;
        const uint16_t *buf = stage0 + st * stage_elems;
        uint32_t P[NQ];
        if (mine) {
#define LBIB_TPULL(q) P[q] = tma_pull<q>(buf, re, x, ylo, yhi);
            LBIB_TPULL(0) LBIB_TPULL(1) LBIB_TPULL(2) LBIB_TPULL(3) LBIB_TPULL(4) LBIB_TPULL(5) LBIB_TPULL(6)
            LBIB_TPULL(7) LBIB_TPULL(8) LBIB_TPULL(9) LBIB_TPULL(10) LBIB_TPULL(11) LBIB_TPULL(12)
            LBIB_TPULL(13) LBIB_TPULL(14) LBIB_TPULL(15) LBIB_TPULL(16) LBIB_TPULL(17) LBIB_TPULL(18)
#undef LBIB_TPULL
        }
        // the stage may be refilled once every consumer warp has read it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + st);
        if (mine) pair_update_act<T>(s, par, (uint32_t)(seg * tt.W + x + s.nx * row), P, seed, act);
    }
}

// Tile width of a row of nx cells: the largest multiple of 8 that divides
// nx and is at most 256; 0 when nx is not a multiple of 8.
static int tma_width(int nx) {
    if (nx % 8) return 0;
    for (int W = TMA_MAX_W; W >= 8; W -= 8)
        if (nx % W == 0) return W;
    return 0;
}

bool fluid_tma_shape(const SimDev &s) {
    return s.prec != LBIB_POP_F32 && !s.solid && !s.in_on && tma_width(s.nx) >= 64;
}

static size_t tma_smem_bytes(int W) { return 128 + (size_t)TMA_STAGES * NQ * tma_row_elems(W) * 2; }

template <typename T>
static cudaError_t launch_tma_t(const SimDev &s, int par, uint32_t seed, cudaStream_t st) {
    TmaTiles tt;
    tt.W = tma_width(s.nx);
    tt.segs = s.nx / tt.W;
    tt.ntiles = tt.segs * s.nyf * s.nz;
    tt.tile_bytes = (uint32_t)(NQ * 2 * tt.W + 10 * 2 * 2 * TMA_HALO);
    const size_t smem = tma_smem_bytes(tt.W);
    static SmemAttr attr;
    cudaError_t e = attr.ensure((const void *)k_fluid_pair_tma<T>, tma_smem_bytes(TMA_MAX_W), false);
    if (e != cudaSuccess) return e;
    const int blocks = (tt.ntiles + TMA_TILES_PER_BLOCK - 1) / TMA_TILES_PER_BLOCK;
    k_fluid_pair_tma<T><<<blocks, TMA_THREADS, smem, st>>>(s, par, seed, tt);
    return cudaGetLastError();
}

cudaError_t launch_fluid_tma(const SimDev &s, int par, uint32_t seed, cudaStream_t st) {
    if (!fluid_tma_shape(s)) return cudaErrorInvalidValue;
    if (s.prec == LBIB_POP_F16S) return launch_tma_t<__half>(s, par, seed, st);
    return launch_tma_t<__nv_bfloat16>(s, par, seed, st);
}

}  // namespace lbib
