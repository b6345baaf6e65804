// glbe_tile.cuh -- the fused step with TMA-staged gathers (sm_100+ tensor
// memory accelerator, mbarrier pipeline), for x-periodic grids with nx a
// multiple of 128 and FP32 / BF16 / FP16 storage.
//
// The arithmetic is the one of glbe_kernels.cuh (node_from_sources); only the
// gather changes.  A persistent block holds one producer warp and four
// consumer warps.  Work is cut into tiles of 128 consecutive x nodes of one
// fluid (y, z) row.  For a tile the producer warp issues one 2-D tensor copy
// per population array (19 for f, 21 more for g; lane r takes array r and
// r + 32): the row the direction
// streams from, (y - e_y, z - e_z), over x in [x0 - 8, x0 + 136), into a
// stage of shared memory, all completing on the stage's mbarrier.  Where that
// row is a wall plane, the link is bounced and the copy takes instead the
// node row's own opposite population (the half-way bounce-back source).  The
// consumer thread of node x reads its 19 (+21) values at x - e_x from the
// stage, releases the stage, and runs the node update.  Four stages per block
// keep the copies of the next tiles in flight while the current one is
// computed, so the compute warps do not wait on DRAM latency.
//
// Periodic wrap in x: the copies read zeros outside [0, nx); the one thread at
// x = 0 (x = nx - 1) takes its sources from x = nx - 1 (x = 0) with plain
// loads.  Every mbarrier wait is bounded in time; a wait that runs out records
// an error flag (reported by glbe_sync) and the block leaves its loop.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

namespace glbe {

constexpr int TILE_W = 128;                          // nodes per tile (one per consumer thread)
constexpr int TILE_HALO = 8;                         // copied halo on each side (16-byte aligned start)
constexpr int TILE_BOX = TILE_W + 2 * TILE_HALO;     // elements per row copy
// Pipeline depth: four stages for the flow lattice; two when the 21 D3Q7
// rows are staged as well (a stage then holds 40 rows).
template <bool MHD>
constexpr int tile_stages() { return MHD ? 2 : 3; }
// Warps per block: one node per thread (4 warps), or two x-adjacent nodes per
// thread with packed FP32x2 arithmetic (2 warps).
template <bool PAIR>
constexpr int tile_consumer_warps() { return PAIR ? TILE_W / 64 : TILE_W / 32; }
template <bool PAIR>
constexpr int tile_threads() { return 32 * tile_consumer_warps<PAIR>(); }
// Resident blocks the register allocation is held to: the paired flow-only
// form fits 96 registers (10 blocks of 64 threads per SM); the other forms
// are left to the compiler.
template <bool PAIR, bool MHD>
constexpr int tile_min_blocks() { return PAIR && !MHD ? 10 : 1; }
constexpr unsigned long long TILE_WAIT_NS = 2000000000ull;   // 2 s per wait at most
// Hint for the time a waiting thread may be suspended inside one try_wait
// (it resumes when the phase completes): waiting warps then take no issue
// slots from the working ones.
constexpr uint32_t TILE_SUSPEND_NS = 100000u;

// Tile decomposition of the fluid rows of a grid.
struct TileGeom {
    uint32_t ntiles;     // xtiles * nyf * nzf
    uint32_t xtiles;     // nx / TILE_W
    uint32_t y0, nyf;    // fluid rows y in [y0, y0 + nyf)
    uint32_t z0, nzf;
    uint32_t plane;      // ny * nz: rows of one population array
};

// Set when a bounded wait of the tile kernel ran out (one flag per
// translation unit; read through tile_wait_error_t).
static __device__ int g_tile_wait_error;

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(TILE_SUSPEND_NS)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long tile_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of the given parity; false (and the error flag set)
// when TILE_WAIT_NS passed first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = tile_clock_ns();
    for (;;) {
        for (int k = 0; k < 4; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (tile_clock_ns() - t0 > TILE_WAIT_NS) {
            atomicExch(&g_tile_wait_error, 1);
            return false;
        }
    }
}

// 2-D tensor copy global -> shared, completing on bar (any lane may issue).
__device__ __forceinline__ void tma_load_row(void* dst, const CUtensorMap* map, int x, int row, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(row), "r"(smem_addr(bar))
        : "memory");
}

template <int ST>
__device__ __forceinline__ float smem_pop(const typename Store<ST>::T* p)
{
    if constexpr (ST == ST_BF16) return __bfloat162float(*p);
    else if constexpr (ST == ST_F16) return __half2float(*p);
    else return *p;
}

// Elements i and i + 1 of a staged row as two FP32 lanes (raw stored values).
// i even: one aligned 4- or 8-byte load; i odd: two element loads.
template <int ST>
__device__ __forceinline__ F2 smem_pair(const typename Store<ST>::T* row, int i, bool aligned)
{
    if (aligned) {
        if constexpr (ST == ST_BF16) return F2(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(row + i)));
        else if constexpr (ST == ST_F16) return F2(__half22float2(*reinterpret_cast<const __half2*>(row + i)));
        else return F2(*reinterpret_cast<const float2*>(row + i));
    }
    return F2(smem_pop<ST>(row + i), smem_pop<ST>(row + i + 1));
}

// Shared-memory row pitch (elements): each row copy starts 128-byte aligned.
template <int ST>
constexpr int tile_pitch()
{
    return (int)(((TILE_BOX * sizeof(typename Store<ST>::T) + 127) / 128) * 128 / sizeof(typename Store<ST>::T));
}

template <int ST, bool MHD>
constexpr size_t tile_smem_bytes()
{
    return 128 + (size_t)tile_stages<MHD>() * (MHD ? 40 : 19) * tile_pitch<ST>() * sizeof(typename Store<ST>::T);
}

// (e_x, e_y, e_z) and opposite of the D3Q19 directions (ordering of glbe.h).
__device__ __forceinline__ void dir19(int a, int& ex, int& ey, int& ez)
{
    constexpr int E[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                              {1, 1, 0},  {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1}, {1, 0, -1},
                              {-1, 0, -1}, {0, 1, 1}, {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};
    ex = E[a][0];
    ey = E[a][1];
    ez = E[a][2];
}

// What a consumer needs of its tile's row: the staged rows and the
// neighbouring planes (with their wall flags) of the fluid row (y, z).
template <class T>
struct TileRowT {
    const T* st;      // stage: row r of the 19 (+21) copies at st + r * pitch
    int pitch;
    int y, z, ym, yp, zm, zp;
    bool sym, syp, szm, szp;
};

// Gather of one node (x = x0 + t) from the stage.  Rows without walls above
// or below read every source at its x-shift; the node at the periodic seam
// (x = 0 or nx - 1) takes the sources across it with plain loads.  Rows next
// to a wall read a bounced link's source unshifted (the stage holds the
// node row's opposite population there) and negate g's (anti-bounce-back).
template <int ST, bool MHD>
__device__ __forceinline__ void tile_gather_one(const StepParams& p, const TileRowT<typename Store<ST>::T>& R, int t,
                                                int x, const typename Store<ST>::T* __restrict__ fs,
                                                const typename Store<ST>::T* __restrict__ gs, float (&d)[19],
                                                float (&q)[21])
{
    const size_t N = p.N;
    const int ny = p.ny;
    const bool wrap_lo = x == 0, wrap_hi = x == p.nx - 1;
    const bool wall_row = R.sym || R.syp || R.szm || R.szp;
    if (!wall_row && !wrap_lo && !wrap_hi) {
        // the common case: no bounced link, no seam; every source at its x-shift
#pragma unroll
        for (int a = 0; a < 19; ++a) {
            int ex, ey, ez;
            dir19(a, ex, ey, ez);
            d[a] = unscale<ST>(p, smem_pop<ST>(R.st + a * R.pitch + TILE_HALO + t - ex));
        }
        if (MHD) {
#pragma unroll
            for (int i = 0; i < 21; ++i) {
                int ex, ey, ez;
                dir19(i % 7, ex, ey, ez);
                q[i] = unscale<ST>(p, smem_pop<ST>(R.st + (19 + i) * R.pitch + TILE_HALO + t - ex));
            }
        }
        return;
    }
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        int ex, ey, ez;
        dir19(a, ex, ey, ez);
        const bool sol = wall_row && ((ey > 0 && R.sym) || (ey < 0 && R.syp) || (ez > 0 && R.szm) || (ez < 0 && R.szp));
        d[a] = unscale<ST>(p, smem_pop<ST>(R.st + a * R.pitch + TILE_HALO + t - (sol ? 0 : ex)));
        if (!sol && ((ex > 0 && wrap_lo) || (ex < 0 && wrap_hi))) {
            const int ys = ey > 0 ? R.ym : (ey < 0 ? R.yp : R.y), zs = ez > 0 ? R.zm : (ez < 0 ? R.zp : R.z);
            const int xw = ex > 0 ? p.nx - 1 : 0;
            d[a] = unscale<ST>(p, Store<ST>::ld(fs + (size_t)a * N + ((size_t)zs * ny + ys) * p.nx + xw));
        }
    }
    if (MHD) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float wall = 0.25f * p.bwall_dev[j];
#pragma unroll
            for (int a = 0; a < 7; ++a) {
                int ex, ey, ez;
                dir19(a, ex, ey, ez);
                const bool sol =
                    wall_row && ((ey > 0 && R.sym) || (ey < 0 && R.syp) || (ez > 0 && R.szm) || (ez < 0 && R.szp));
                float v = unscale<ST>(p, smem_pop<ST>(R.st + (19 + j * 7 + a) * R.pitch + TILE_HALO + t - (sol ? 0 : ex)));
                if (!sol && ((ex > 0 && wrap_lo) || (ex < 0 && wrap_hi))) {
                    const int xw = ex > 0 ? p.nx - 1 : 0;
                    v = unscale<ST>(p, Store<ST>::ld(gs + (size_t)(j * 7 + a) * N + ((size_t)R.z * ny + R.y) * p.nx + xw));
                }
                q[j * 7 + a] = sol ? wall - v : v;
            }
        }
    }
}

// Gather of the node pair (x, x + 1), x = x0 + 2t, as FP32x2 lanes; the same
// rules, with aligned pair reads where the x-shift is 0 and lane patches at
// the periodic seam.
template <int ST, bool MHD>
__device__ __forceinline__ void tile_gather_pair(const StepParams& p, const TileRowT<typename Store<ST>::T>& R, int t,
                                                 int x, const typename Store<ST>::T* __restrict__ fs,
                                                 const typename Store<ST>::T* __restrict__ gs, F2 (&d)[19],
                                                 F2 (&q)[21])
{
    const size_t N = p.N;
    const int ny = p.ny;
    const bool wrap_lo = x == 0, wrap_hi = x + 1 == p.nx - 1;
    const bool wall_row = R.sym || R.syp || R.szm || R.szp;
    if (!wall_row && !wrap_lo && !wrap_hi) {
        // the common case: no bounced link, no seam; aligned pairs where e_x = 0
#pragma unroll
        for (int a = 0; a < 19; ++a) {
            int ex, ey, ez;
            dir19(a, ex, ey, ez);
            d[a] = unscale<ST>(p, smem_pair<ST>(R.st + a * R.pitch, TILE_HALO + 2 * t - ex, ex == 0));
        }
        if (MHD) {
#pragma unroll
            for (int i = 0; i < 21; ++i) {
                int ex, ey, ez;
                dir19(i % 7, ex, ey, ez);
                q[i] = unscale<ST>(p, smem_pair<ST>(R.st + (19 + i) * R.pitch, TILE_HALO + 2 * t - ex, ex == 0));
            }
        }
        return;
    }
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        int ex, ey, ez;
        dir19(a, ex, ey, ez);
        const bool sol = wall_row && ((ey > 0 && R.sym) || (ey < 0 && R.syp) || (ez > 0 && R.szm) || (ez < 0 && R.szp));
        const bool shifted = !sol && ex != 0;
        F2 v = smem_pair<ST>(R.st + a * R.pitch, TILE_HALO + 2 * t - (shifted ? ex : 0), !shifted);
        if (shifted && ((ex > 0 && wrap_lo) || (ex < 0 && wrap_hi))) {
            const int ys = ey > 0 ? R.ym : (ey < 0 ? R.yp : R.y), zs = ez > 0 ? R.zm : (ez < 0 ? R.zp : R.z);
            const int xw = ex > 0 ? p.nx - 1 : 0;
            const float w = Store<ST>::ld(fs + (size_t)a * N + ((size_t)zs * ny + ys) * p.nx + xw);
            if (ex > 0) v.v.x = w; else v.v.y = w;
        }
        d[a] = unscale<ST>(p, v);
    }
    if (MHD) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const F2 wall(0.25f * p.bwall_dev[j]);
#pragma unroll
            for (int a = 0; a < 7; ++a) {
                int ex, ey, ez;
                dir19(a, ex, ey, ez);
                const bool sol =
                    wall_row && ((ey > 0 && R.sym) || (ey < 0 && R.syp) || (ez > 0 && R.szm) || (ez < 0 && R.szp));
                const bool shifted = !sol && ex != 0;
                F2 v = smem_pair<ST>(R.st + (19 + j * 7 + a) * R.pitch, TILE_HALO + 2 * t - (shifted ? ex : 0),
                                     !shifted);
                if (shifted && ((ex > 0 && wrap_lo) || (ex < 0 && wrap_hi))) {
                    const int xw = ex > 0 ? p.nx - 1 : 0;
                    const float w =
                        Store<ST>::ld(gs + (size_t)(j * 7 + a) * N + ((size_t)R.z * ny + R.y) * p.nx + xw);
                    if (ex > 0) v.v.x = w; else v.v.y = w;
                }
                v = unscale<ST>(p, v);
                q[j * 7 + a] = sol ? wall - v : v;
            }
        }
    }
}

// The same tables for run-time indices (the producer lanes): e_y, e_z and
// the opposite direction.
static __constant__ int c_tile_ey[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
static __constant__ int c_tile_ez[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
static __constant__ int c_tile_opp[19] = {0, 2, 1, 4, 3, 6, 5, 10, 9, 8, 7, 14, 13, 12, 11, 18, 17, 16, 15};

template <int ST, bool MHD, int MODE, bool PAIR>
__global__ void __launch_bounds__(tile_threads<PAIR>(), tile_min_blocks<PAIR, MHD>())
    tile_kernel(const StepParams p, const StepBuffers b, const TileGeom tg, const __grid_constant__ CUtensorMap tmf,
                const __grid_constant__ CUtensorMap tmg)
{
    using S = Store<ST>;
    using T = typename S::T;
    constexpr int Q = MHD ? 40 : 19;
    constexpr int RP = tile_pitch<ST>();
    constexpr uint32_t TILE_STAGES = (uint32_t)tile_stages<MHD>();
    constexpr uint32_t STAGE_TX = (uint32_t)(Q * TILE_BOX * sizeof(T));
    constexpr int TILE_WARPS = tile_consumer_warps<PAIR>();
    constexpr int TILE_THREADS = tile_threads<PAIR>();
    if (b.stop != nullptr && *b.stop) return;

    extern __shared__ __align__(128) unsigned char tile_smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(tile_smem);
    uint64_t* empty = full + TILE_STAGES;
    T* stages = reinterpret_cast<T*>(tile_smem + 128);
    if (threadIdx.x == 0) {
        for (uint32_t s = 0; s < TILE_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TILE_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = threadIdx.x;
    const int ny = p.ny, nz = p.nz;
    const T* __restrict__ fs = static_cast<const T*>(b.fsrc);
    const T* __restrict__ gs = static_cast<const T*>(b.gsrc);
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

    // Warp 0 fills a stage with the rows of a tile: lane r issues row copy r
    // (and r + 32), all completing on the stage's full barrier.
    auto issue = [&](uint32_t tile, uint32_t s) {
        if (lane == 0) mbar_arrive_expect_tx(&full[s], STAGE_TX);
        __syncwarp();
        const uint32_t xt = tile % tg.xtiles, r = tile / tg.xtiles;
        const int y = (int)(tg.y0 + r % tg.nyf), z = (int)(tg.z0 + r / tg.nyf);
        const int xs = (int)(xt * TILE_W) - TILE_HALO;
        T* st = stages + (size_t)s * Q * RP;
        for (int rr = lane; rr < Q; rr += 32) {
            // row rr of the stage: f direction rr, or g component j, direction a
            const int a = rr < 19 ? rr : (rr - 19) % 7;
            const int arr = rr < 19 ? rr : rr - 19;   // population array index within f or g
            const int ey = c_tile_ey[a], ez = c_tile_ez[a];
            const int ys = y - ey < 0 ? ny - 1 : (y - ey >= ny ? 0 : y - ey);
            const int zs = z - ez < 0 ? nz - 1 : (z - ez >= nz ? 0 : z - ez);
            const bool sol = plane_solid(ys, ny, p.wlo[1], p.whi[1]) || plane_solid(zs, nz, p.wlo[2], p.whi[2]);
            const int src_arr = sol ? arr - a + c_tile_opp[a] : arr;   // bounced: the opposite population
            const int row = sol ? src_arr * (int)tg.plane + z * ny + y : src_arr * (int)tg.plane + zs * ny + ys;
            tma_load_row(st + rr * RP, rr < 19 ? &tmf : &tmg, xs, row, &full[s]);
        }
    };

    uint32_t issued = 0;   // tiles issued by warp 0
    if (warp == 0) {
        for (uint32_t j = 0; j < TILE_STAGES; ++j) {
            const uint32_t tile = blockIdx.x + j * gridDim.x;
            if (tile >= tg.ntiles) break;
            issue(tile, j);
            ++issued;
        }
    }
    bool ok = true;
    uint32_t k = 0;
    for (uint32_t tile = blockIdx.x; tile < tg.ntiles; tile += gridDim.x, ++k) {
        const uint32_t s = k % TILE_STAGES;
        const uint32_t par = (k / TILE_STAGES) & 1u;
        const uint32_t xt = tile % tg.xtiles, r = tile / tg.xtiles;
        const int y = (int)(tg.y0 + r % tg.nyf), z = (int)(tg.z0 + r / tg.nyf);
        const int x = (int)(xt * TILE_W) + (PAIR ? 2 * t : t);
        const uint32_t n = ((uint32_t)z * (uint32_t)ny + (uint32_t)y) * (uint32_t)p.nx + (uint32_t)x;
        using V = typename std::conditional<PAIR, F2, float>::type;
        // the node's other inputs, loaded while the stage may still be in flight
        NodeIn<V> in;
        if constexpr (PAIR) in = pair_inputs<MHD, MODE>(p, b, n);
        else in = node_inputs<MHD, MODE>(p, b, n);
        if (!mbar_wait(&full[s], par)) { ok = false; break; }
        const T* st = stages + (size_t)s * Q * RP;
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        const bool sym = plane_solid(ym, ny, p.wlo[1], p.whi[1]), syp = plane_solid(yp, ny, p.wlo[1], p.whi[1]);
        const bool szm = plane_solid(zm, nz, p.wlo[2], p.whi[2]), szp = plane_solid(zp, nz, p.wlo[2], p.whi[2]);
        V d[19], dl[19], q[21], ql[21];
        const TileRowT<T> row{st, RP, y, z, ym, yp, zm, zp, sym, syp, szm, szp};
        if constexpr (PAIR) tile_gather_pair<ST, MHD>(p, row, t, x, fs, gs, d, q);
        else tile_gather_one<ST, MHD>(p, row, t, x, fs, gs, d, q);
        // the stage is no longer needed: release it; warp 0 refills it with
        // the tile TILE_STAGES ahead once every warp has released it
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (warp == 0) {
            const uint32_t next = tile + TILE_STAGES * gridDim.x;
            if (next < tg.ntiles) {
                int got = 0;
                if (lane == 0) got = mbar_wait(&empty[s], par) ? 1 : 0;
                if (!__shfl_sync(0xffffffffu, got, 0)) { ok = false; break; }
                issue(next, s);
                ++issued;
            }
        }
        if constexpr (PAIR) pair_from_sources<ST, MHD, MODE>(p, b, n, d, dl, q, ql, in, acc);
        else node_from_sources<ST, MHD, MODE>(p, b, FieldOut{nullptr, nullptr, nullptr}, n, d, dl, q, ql, in, acc);
    }
    if (!ok && warp == 0 && lane == 0) {
        // leave no copy in flight: wait (bounded) for the tiles issued but not consumed
        for (uint32_t kk = k; kk < issued; ++kk) mbar_wait(&full[kk % TILE_STAGES], (kk / TILE_STAGES) & 1u);
    }
    if (MODE == MODE_STEP_RESID) block_partials<TILE_THREADS>(acc, b.partials);
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
inline bool tile_eligible(const StepParams& p, int mode)
{
    if (mode == MODE_FIELDS) return false;
    if (p.storage != ST_F32 && p.storage != ST_BF16 && p.storage != ST_F16) return false;
    if (p.wlo[0] || p.whi[0]) return false;                 // x periodic
    if (p.glo_z || p.ghi_z) return false;                   // no ghost planes
    if (p.nx % TILE_W != 0) return false;
    if (p.ny - p.wlo[1] - p.whi[1] < 1 || p.nz - p.wlo[2] - p.whi[2] < 1) return false;
    const unsigned long long rows = 21ull * (unsigned long long)p.ny * (unsigned long long)p.nz;
    return rows < (1ull << 31);
}

inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// Row-copy tensor map over a population buffer: dims (nx, rows), one row
// per copy of TILE_BOX elements.
template <int ST>
inline bool make_row_map(CUtensorMap* map, const void* base, int nx, unsigned long long rows)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = ST == ST_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : (ST == ST_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    const size_t es = sizeof(typename Store<ST>::T);
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)nx * es};
    const cuuint32_t box[2] = {(cuuint32_t)TILE_BOX, 1u};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int ST, bool MHD, int MODE, bool PAIR>
cudaError_t launch_tile(const StepParams& p, const StepBuffers& b, cudaStream_t st, unsigned* nblocks)
{
    constexpr int TILE_THREADS = tile_threads<PAIR>();
    static int max_blocks = 0;   // resident blocks for the whole GPU (per instantiation, first device used)
    constexpr size_t smem = tile_smem_bytes<ST, MHD>();
    if (max_blocks == 0) {
        cudaError_t e = cudaFuncSetAttribute(tile_kernel<ST, MHD, MODE, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_kernel<ST, MHD, MODE, PAIR>, TILE_THREADS, smem);
        if (e != cudaSuccess) return e;
        max_blocks = sms * (per_sm > 0 ? per_sm : 1);
    }
    TileGeom tg;
    tg.xtiles = (uint32_t)(p.nx / TILE_W);
    tg.y0 = (uint32_t)p.wlo[1];
    tg.nyf = (uint32_t)(p.ny - p.wlo[1] - p.whi[1]);
    tg.z0 = (uint32_t)p.wlo[2];
    tg.nzf = (uint32_t)(p.nz - p.wlo[2] - p.whi[2]);
    tg.ntiles = tg.xtiles * tg.nyf * tg.nzf;
    tg.plane = (uint32_t)(p.ny * p.nz);
    CUtensorMap mf, mg;
    if (!make_row_map<ST>(&mf, b.fsrc, p.nx, 19ull * tg.plane)) return cudaErrorInvalidValue;
    if (MHD) {
        if (!make_row_map<ST>(&mg, b.gsrc, p.nx, 21ull * tg.plane)) return cudaErrorInvalidValue;
    } else {
        mg = mf;
    }
    // at most one block per tile, per resident slot, and per residual partial
    // the context holds (one per 256 nodes)
    unsigned grid = (unsigned)(tg.ntiles < (uint32_t)max_blocks ? tg.ntiles : (uint32_t)max_blocks);
    const unsigned partial_cap = (unsigned)(((size_t)p.N + STEP_THREADS - 1) / STEP_THREADS);
    if (grid > partial_cap) grid = partial_cap;
    tile_kernel<ST, MHD, MODE, PAIR><<<grid, TILE_THREADS, smem, st>>>(p, b, tg, mf, mg);
    if (nblocks) *nblocks = grid;
    return cudaGetLastError();
}

// Reads and clears this translation unit's wait-error flag.
inline int tile_wait_error_read()
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tile_wait_error, sizeof v) != cudaSuccess) return 0;
    if (v) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_tile_wait_error, &zero, sizeof zero);
    }
    return v;
}

}  // namespace glbe
