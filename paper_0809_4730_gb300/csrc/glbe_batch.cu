// glbe_batch.cu -- many independent steady solves in one persistent launch.
//
// A batch holds up to GLBE_BATCH_MAX_DOMAINS independent lattices (own grid,
// walls, gamma, rates, induction coupling or not).  One cooperative kernel,
// resident on every SM for the whole solve, marches all unconverged domains
// together: each step its blocks walk a flattened list of 256-node (or
// 128-node) tiles of all active domains with the one-node-per-thread update of
// glbe_kernels.cuh, then meet at a grid barrier.  Every 10 levels each tile
// leaves its residual sums, a second phase reduces them per domain in a fixed
// order, and a domain whose r(t) <= tol (or whose velocity became non-finite)
// leaves the march; its convergence level and the device time since the start
// of the launch are recorded.  The launch is captured once in a CUDA graph.
//
// The grid barrier is this file's own: a block that waits longer than
// BARRIER_SPIN_LIMIT polls raises an error flag and the whole kernel returns;
// the host reports GLBE_ERR_TIMEOUT.  The launch is cooperative, so all blocks
// are resident and the barrier can complete.
//
// The block size and the number of resident blocks per SM are chosen by
// glbe_batch_autotune, which times a few steps of each candidate on the batch
// itself and then restores the rest state.
#include <cstring>
#include <new>
#include <vector>

#include "glbe.h"
#include "glbe_internal.h"
#include "glbe_kernels.cuh"

using namespace glbe;

namespace {

constexpr long long BARRIER_SPIN_LIMIT = 1ll << 26;   // default polls of ~64 ns: about 4 s

struct BatchDomain {
    StepParams p;
    void* f[2];
    void* g[2];
    float* FL;
    float* usnap;
    uint32_t nodes;
    int mhd;
    double mass0;
};

struct BatchState {
    unsigned barrier_count;
    unsigned barrier_gen;
    int error;
    int n_active;
    unsigned long long t_start_ns;
};

struct BatchDomainState {
    int active;
    int nonfinite;
    long long conv_level;      // level t with r(t) <= tol, -1 while marching
    double conv_seconds;       // device time from the start of the launch
    double r;                  // last residual
    long long last_level;      // level of the last residual
};

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Sense-reversing grid barrier with a bounded wait.  Returns false (for every
// block) once any block gave up.
__device__ bool grid_barrier(BatchState* st, long long spin_limit)
{
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &st->barrier_gen;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&st->barrier_count, 1u);
        if (arrived == gridDim.x - 1) {
            st->barrier_count = 0;
            __threadfence();
            atomicAdd(&st->barrier_gen, 1u);
        } else {
            long long spins = 0;
            while (*gen == g0) {
                if (++spins > spin_limit || *(volatile int*)&st->error) {
                    atomicExch(&st->error, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = *(volatile int*)&st->error == 0;
    }
    __syncthreads();
    return ok;
}

template <int ST, int BT>
__global__ void __launch_bounds__(BT, 512 / BT) batch_kernel(const BatchDomain* __restrict__ doms, int ndom,
                                                   const uint32_t* __restrict__ tile_start, uint32_t ntiles,
                                                   double* __restrict__ partials, BatchState* st,
                                                   BatchDomainState* ds, long long t0, long long nsteps,
                                                   long long snap_level, double tol, long long spin_limit,
                                                   int absent_block)
{
    // absent_block >= 0 (failure-detection tests only): that block leaves at
    // once, so the others' first barrier wait runs out and the launch ends
    // with the error flag set instead of hanging
    if ((int)blockIdx.x == absent_block) return;
    __shared__ StepParams sp;
    // the domain whose parameters sp holds: the same in every thread (a tile
    // belongs to one domain), so the check needs no shared flag and a block
    // synchronises only when it moves to another domain
    int cur_dom = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->t_start_ns = globaltimer_ns();
    long long last_snap = snap_level;
    for (long long s = 0; s < nsteps; ++s) {
        const long long t = t0 + s;
        const bool resid = (t % 10) == 0;
        const bool have_snap = resid && last_snap >= 0 && last_snap == t - 10;
        const int par = (int)(t & 1);
        // the block's tiles ascend, and so do the domains' tile ranges: the
        // domain of the next tile is found by advancing a cursor, and the
        // domain's buffers and active flag (which changes only between
        // levels) are read once per domain and level
        int d = 0, lvl_dom = -1;
        bool active = false;
        StepBuffers b{};
        uint32_t tile0 = 0;
        bool mhd = false;
        for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            while (__ldg(tile_start + d + 1) <= tile) ++d;
            if (d != lvl_dom) {
                lvl_dom = d;
                const BatchDomain& D = doms[d];
                active = __ldcg(&ds[d].active) != 0;
                b.fsrc = D.f[par];
                b.fdst = D.f[par ^ 1];
                b.gsrc = D.g[par];
                b.gdst = D.g[par ^ 1];
                b.FL = D.FL;
                b.usnap = D.usnap;
                b.snap_lo = 1;
                b.have_snap = have_snap ? 1 : 0;
                tile0 = __ldg(tile_start + d);
                mhd = D.mhd != 0;
            }
            float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (active) {
                if (cur_dom != d) {
                    // the block's copy of the domain's step parameters (after
                    // every thread is done with the previous domain's)
                    __syncthreads();
                    const int words = (int)(sizeof(StepParams) / 4);
                    for (int w = threadIdx.x; w < words; w += BT)
                        reinterpret_cast<int*>(&sp)[w] = reinterpret_cast<const int*>(&doms[d].p)[w];
                    __syncthreads();
                    cur_dom = d;
                }
                const FieldOut fo{nullptr, nullptr, nullptr};
                const uint32_t i = (tile - tile0) * BT + threadIdx.x;
                // populations written by other blocks earlier in this launch:
                // coherent loads (CG), cached in L1 within a level.  A coupled
                // node is updated in two passes
                // (induction, then flow with this step's Lorentz force), each
                // within the kernel's register budget; the one-pass update
                // spilled over a kilobyte per thread.
                if (mhd) {
                    coupled_induction_pass<ST, true>(sp, b, i);
                    if (resid) scalar_node_step<ST, false, MODE_STEP_RESID, true, false, true>(sp, b, fo, i, acc);
                    else scalar_node_step<ST, false, MODE_STEP, true, false, true>(sp, b, fo, i, acc);
                } else {
                    if (resid) scalar_node_step<ST, false, MODE_STEP_RESID, true>(sp, b, fo, i, acc);
                    else scalar_node_step<ST, false, MODE_STEP, true>(sp, b, fo, i, acc);
                }
            }
            if (resid) {
                // partials[k][tile]; converged domains leave zeros
                __shared__ double sh[BT / 32][7];
                const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
                for (int k = 0; k < 7; ++k) {
                    const float v = warp_sum(acc[k]);
                    if (lane == 0) sh[warp][k] = (double)v;
                }
                __syncthreads();
                if (threadIdx.x < 7) {
                    double sum = 0.0;
#pragma unroll
                    for (int w = 0; w < BT / 32; ++w) sum += sh[w][threadIdx.x];
                    partials[(size_t)threadIdx.x * ntiles + tile] = sum;
                }
                __syncthreads();
            }
        }
        if (!grid_barrier(st, spin_limit)) return;
        if (resid) {
            if (have_snap) {
                // per-domain residual: block b reduces domains b, b + G, ... in a fixed order
                __shared__ double red[7][BT];
                for (int d = blockIdx.x; d < ndom; d += gridDim.x) {
                    if (!__ldcg(&ds[d].active)) continue;
                    const uint32_t t0d = tile_start[d], t1d = tile_start[d + 1];
                    for (int k = 0; k < 7; ++k) {
                        double sum = 0.0;
                        for (uint32_t tt = t0d + threadIdx.x; tt < t1d; tt += BT)
                            sum += __ldcg(&partials[(size_t)k * ntiles + tt]);
                        red[k][threadIdx.x] = sum;
                    }
                    __syncthreads();
                    for (int w = BT / 2; w > 0; w >>= 1) {
                        if ((int)threadIdx.x < w)
                            for (int k = 0; k < 7; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
                        __syncthreads();
                    }
                    if (threadIdx.x == 0) {
                        const double num = red[0][0], den = red[1][0];
                        const double r = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
                        BatchDomainState& S = ds[d];
                        S.r = r;
                        S.last_level = t;
                        const bool bad = red[6][0] > 0.0 || !isfinite(r);
                        if (bad) S.nonfinite = 1;
                        if (bad || r <= tol) {
                            S.active = 0;
                            S.conv_level = bad ? -1 : t;
                            S.conv_seconds = (double)(globaltimer_ns() - st->t_start_ns) * 1e-9;
                            atomicSub(&st->n_active, 1);
                        }
                    }
                    __syncthreads();
                }
            }
            last_snap = t;
            if (!grid_barrier(st, spin_limit)) return;
            if (*(volatile int*)&st->n_active == 0) return;
        }
    }
}

__global__ void batch_reset_kernel(BatchState* st, BatchDomainState* ds, int ndom)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        st->barrier_count = 0;
        st->barrier_gen = 0;
        st->error = 0;
        st->n_active = ndom;
        st->t_start_ns = 0;
    }
    if (i < ndom) {
        ds[i].active = 1;
        ds[i].nonfinite = 0;
        ds[i].conv_level = -1;
        ds[i].conv_seconds = 0.0;
        ds[i].r = 0.0;
        ds[i].last_level = -1;
    }
}

size_t align_up(size_t x) { return (x + 255) / 256 * 256; }

struct DomLayout {
    size_t f[2], g[2], FL, usnap, end;
};

size_t storage_bytes(int st) { return st == GLBE_F32 ? 4 : (st == GLBE_F32C ? 6 : 2); }

}  // namespace

struct glbe_batch {
    int n;
    int storage;
    std::vector<glbe_params> prm;
    std::vector<BatchDomain> host_doms;
    char* ws;
    size_t ws_bytes;
    BatchDomain* d_doms;
    uint32_t* d_tile_start;
    double* d_partials;
    BatchState* d_state;
    BatchDomainState* d_dstate;
    size_t partial_doubles;
    cudaStream_t stream;
    int block_threads;     // 128 or 256
    int blocks_per_sm;     // resident blocks of the persistent launch
    int num_sms;
    long long t;           // level of all domains
    long long snap_level;
    std::vector<long long> level;   // level each domain's state is at after a solve
    long long spin_limit;           // polls before a barrier wait gives up
    int absent_block;               // failure-detection tests: block that skips the march
    size_t state_bytes_end;   // bytes of the population region (for the reset)
};

namespace {

glbe_status batch_layout(const glbe_params* doms, int n, std::vector<DomLayout>* lay, size_t* misc_off,
                         size_t* total, size_t* partial_doubles)
{
    if (!doms || n < 1 || n > GLBE_BATCH_MAX_DOMAINS)
        return fail(GLBE_ERR_ARG, "batch needs 1..%d domains", GLBE_BATCH_MAX_DOMAINS);
    const int st = doms[0].storage;
    if (st != GLBE_F32 && st != GLBE_F32C) return fail(GLBE_ERR_ARG, "batch storage must be GLBE_F32 or GLBE_F32C");
    size_t off = 0, tiles128 = 0;
    lay->resize(n);
    for (int d = 0; d < n; ++d) {
        glbe_status s = validate_params(&doms[d]);
        if (s != GLBE_OK) return fail(s, "domain %d: %s", d, glbe_last_error());
        if (doms[d].storage != st) return fail(GLBE_ERR_ARG, "all domains of a batch share one storage type");
        if (doms[d].force_field) return fail(GLBE_ERR_ARG, "batch domains take a uniform force (force_field = 0)");
        if (doms[d].ghost_lo || doms[d].ghost_hi) return fail(GLBE_ERR_ARG, "batch domains have no ghost planes");
        if (doms[d].collision) return fail(GLBE_ERR_ARG, "batch domains use the MRT collision");
        if (make_step_params(&doms[d]).cavity) return fail(GLBE_ERR_ARG, "batch domains have no box or lid");
        const size_t N = (size_t)doms[d].nx * doms[d].ny * doms[d].nz;
        const size_t ss = storage_bytes(st);
        DomLayout& L = (*lay)[d];
        auto take = [&](size_t b) { size_t o = off; off = align_up(off + b); return o; };
        L.f[0] = take(19 * N * ss);
        L.f[1] = take(19 * N * ss);
        if (doms[d].induction) {
            L.g[0] = take(21 * N * ss);
            L.g[1] = take(21 * N * ss);
            L.FL = take(3 * N * sizeof(float));
        } else {
            L.g[0] = L.g[1] = L.FL = (size_t)-1;
        }
        L.usnap = take(6 * N * sizeof(float));   // double-float velocity snapshot (F32, F32C)
        L.end = off;
        tiles128 += (N + 127) / 128;
    }
    *misc_off = off;
    *partial_doubles = 8 * tiles128;
    off = align_up(off + sizeof(BatchDomain) * n);
    off = align_up(off + sizeof(uint32_t) * (n + 1));
    off = align_up(off + sizeof(double) * *partial_doubles);
    off = align_up(off + sizeof(BatchState));
    off = align_up(off + sizeof(BatchDomainState) * n);
    *total = off;
    return GLBE_OK;
}

cudaError_t upload_tiles(glbe_batch* b)
{
    std::vector<uint32_t> ts(b->n + 1);
    uint32_t acc = 0;
    for (int d = 0; d < b->n; ++d) {
        ts[d] = acc;
        acc += (b->host_doms[d].nodes + b->block_threads - 1) / b->block_threads;
    }
    ts[b->n] = acc;
    return cudaMemcpyAsync(b->d_tile_start, ts.data(), sizeof(uint32_t) * (b->n + 1), cudaMemcpyHostToDevice,
                           b->stream);
}

uint32_t total_tiles(const glbe_batch* b)
{
    uint32_t acc = 0;
    for (int d = 0; d < b->n; ++d) acc += (b->host_doms[d].nodes + b->block_threads - 1) / b->block_threads;
    return acc;
}

template <int ST, int BT>
void* kernel_ptr()
{
    return reinterpret_cast<void*>(&batch_kernel<ST, BT>);
}

void* batch_kernel_for(int storage, int bt)
{
    if (storage == GLBE_F32) return bt == 128 ? kernel_ptr<ST_F32, 128>() : kernel_ptr<ST_F32, 256>();
    return bt == 128 ? kernel_ptr<ST_F32C, 128>() : kernel_ptr<ST_F32C, 256>();
}

glbe_status max_blocks_per_sm(glbe_batch* b, int bt, int* out)
{
    int nb = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel_for(b->storage, bt), bt, 0);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "occupancy query: %s", cudaGetErrorString(e));
    *out = nb;
    return GLBE_OK;
}

// Enqueues one persistent cooperative launch of nsteps levels.
glbe_status launch_batch(glbe_batch* b, long long nsteps, double tol, cudaStream_t stream)
{
    const uint32_t ntiles = total_tiles(b);
    int maxb = 0;
    glbe_status s = max_blocks_per_sm(b, b->block_threads, &maxb);
    if (s != GLBE_OK) return s;
    if (maxb < 1) return fail(GLBE_ERR_CUDA, "batch kernel cannot be resident (block %d)", b->block_threads);
    const int bps = b->blocks_per_sm < 1 ? 1 : (b->blocks_per_sm > maxb ? maxb : b->blocks_per_sm);
    const unsigned grid = (unsigned)(bps * b->num_sms);
    long long t0 = b->t, snap = b->snap_level;
    long long spin = b->spin_limit;
    int absent = b->absent_block;
    void* args[] = {&b->d_doms, &b->n, &b->d_tile_start, (void*)&ntiles, &b->d_partials, &b->d_state, &b->d_dstate,
                    &t0, &nsteps, &snap, &tol, &spin, &absent};
    cudaError_t e = cudaLaunchCooperativeKernel(batch_kernel_for(b->storage, b->block_threads), dim3(grid),
                                                dim3(b->block_threads), args, 0, stream);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "cooperative batch launch: %s", cudaGetErrorString(e));
    return GLBE_OK;
}

glbe_status reset_state(glbe_batch* b, bool populations)
{
    cudaError_t e = cudaSuccess;
    if (populations) e = cudaMemsetAsync(b->ws, 0, b->state_bytes_end, b->stream);
    if (e == cudaSuccess) {
        batch_reset_kernel<<<(b->n + 255) / 256, 256, 0, b->stream>>>(b->d_state, b->d_dstate, b->n);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "batch reset: %s", cudaGetErrorString(e));
    if (populations) {
        b->t = 0;
        b->snap_level = -1;
        b->level.clear();
    }
    return GLBE_OK;
}

}  // namespace

extern "C" {

glbe_status glbe_batch_workspace_bytes(const glbe_params* doms, int n, size_t* bytes)
{
    if (!bytes) return fail(GLBE_ERR_ARG, "bytes is NULL");
    std::vector<DomLayout> lay;
    size_t misc = 0, total = 0, pd = 0;
    glbe_status s = batch_layout(doms, n, &lay, &misc, &total, &pd);
    if (s != GLBE_OK) return s;
    *bytes = total;
    return GLBE_OK;
}

glbe_status glbe_batch_init(const glbe_params* doms, int n, void* d_workspace, size_t bytes, void* stream,
                            glbe_batch** out)
{
    if (!out) return fail(GLBE_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::vector<DomLayout> lay;
    size_t misc = 0, total = 0, pd = 0;
    glbe_status s = batch_layout(doms, n, &lay, &misc, &total, &pd);
    if (s != GLBE_OK) return s;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u))
        return fail(GLBE_ERR_ARG, "workspace must be a 256-byte aligned device pointer");
    if (bytes < total) return fail(GLBE_ERR_ARG, "workspace of %zu bytes is smaller than the %zu needed", bytes, total);
    glbe_batch* b = new (std::nothrow) glbe_batch();
    if (!b) return fail(GLBE_ERR_ARG, "out of host memory");
    b->n = n;
    b->storage = doms[0].storage;
    b->prm.assign(doms, doms + n);
    b->ws = static_cast<char*>(d_workspace);
    b->ws_bytes = bytes;
    b->stream = static_cast<cudaStream_t>(stream);
    b->state_bytes_end = misc;
    size_t off = misc;
    b->d_doms = reinterpret_cast<BatchDomain*>(b->ws + off);
    off = align_up(off + sizeof(BatchDomain) * n);
    b->d_tile_start = reinterpret_cast<uint32_t*>(b->ws + off);
    off = align_up(off + sizeof(uint32_t) * (n + 1));
    b->d_partials = reinterpret_cast<double*>(b->ws + off);
    b->partial_doubles = pd;
    off = align_up(off + sizeof(double) * pd);
    b->d_state = reinterpret_cast<BatchState*>(b->ws + off);
    off = align_up(off + sizeof(BatchState));
    b->d_dstate = reinterpret_cast<BatchDomainState*>(b->ws + off);
    b->block_threads = 256;
    b->blocks_per_sm = 1;
    b->spin_limit = BARRIER_SPIN_LIMIT;
    b->absent_block = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess || !coop) {
        delete b;
        return fail(GLBE_ERR_CUDA, "device attributes / cooperative launch unavailable");
    }
    b->host_doms.resize(n);
    for (int d = 0; d < n; ++d) {
        const glbe_params& p = doms[d];
        BatchDomain& D = b->host_doms[d];
        std::memset(&D, 0, sizeof D);
        D.p = make_step_params(&p);
        D.f[0] = b->ws + lay[d].f[0];
        D.f[1] = b->ws + lay[d].f[1];
        D.g[0] = p.induction ? b->ws + lay[d].g[0] : nullptr;
        D.g[1] = p.induction ? b->ws + lay[d].g[1] : nullptr;
        D.FL = p.induction ? reinterpret_cast<float*>(b->ws + lay[d].FL) : nullptr;
        D.usnap = reinterpret_cast<float*>(b->ws + lay[d].usnap);
        D.nodes = (uint32_t)((size_t)p.nx * p.ny * p.nz);
        D.mhd = p.induction;
        const long long fluid = fluid_nodes(&p);
        D.mass0 = p.rho0 * (double)fluid;
    }
    e = cudaMemcpyAsync(b->d_doms, b->host_doms.data(), sizeof(BatchDomain) * n, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = upload_tiles(b);
    if (e != cudaSuccess) {
        delete b;
        return fail(GLBE_ERR_CUDA, "batch upload: %s", cudaGetErrorString(e));
    }
    s = reset_state(b, true);
    if (s != GLBE_OK) {
        delete b;
        return s;
    }
    e = cudaStreamSynchronize(b->stream);   // the host-side tables above must outlive their copies
    if (e != cudaSuccess) {
        delete b;
        return fail(GLBE_ERR_CUDA, "batch init sync: %s", cudaGetErrorString(e));
    }
    *out = b;
    return GLBE_OK;
}

glbe_status glbe_batch_set_launch(glbe_batch* b, int block_threads, int blocks_per_sm)
{
    if (!b) return fail(GLBE_ERR_ARG, "batch is NULL");
    if (block_threads != 128 && block_threads != 256) return fail(GLBE_ERR_ARG, "block_threads must be 128 or 256");
    int maxb = 0;
    b->block_threads = block_threads;
    glbe_status s = max_blocks_per_sm(b, block_threads, &maxb);
    if (s != GLBE_OK) return s;
    if (blocks_per_sm < 1 || blocks_per_sm > maxb)
        return fail(GLBE_ERR_ARG, "blocks_per_sm must be in 1..%d for %d threads", maxb, block_threads);
    b->blocks_per_sm = blocks_per_sm;
    cudaError_t e = upload_tiles(b);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "tile table: %s", cudaGetErrorString(e));
    return GLBE_OK;
}

glbe_status glbe_batch_autotune(glbe_batch* b, int steps_per_trial, int* block_threads_out, int* blocks_per_sm_out,
                                double* seconds_per_step_out)
{
    if (!b) return fail(GLBE_ERR_ARG, "batch is NULL");
    if (steps_per_trial < 2) steps_per_trial = 2;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(GLBE_ERR_CUDA, "event create");
    double best = 1e30;
    int best_bt = 256, best_bps = 1;
    glbe_status st = GLBE_OK;
    for (int bt : {128, 256}) {
        int maxb = 0;
        b->block_threads = bt;
        st = max_blocks_per_sm(b, bt, &maxb);
        if (st != GLBE_OK) break;
        for (int bps = 1; bps <= maxb; ++bps) {
            st = glbe_batch_set_launch(b, bt, bps);
            if (st != GLBE_OK) break;
            st = reset_state(b, false);
            if (st != GLBE_OK) break;
            // trial steps start at an odd level so that no residual is taken
            b->t = 1;
            cudaEventRecord(e0, b->stream);
            st = launch_batch(b, steps_per_trial, 0.0, b->stream);
            if (st != GLBE_OK) break;
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = fail(GLBE_ERR_CUDA, "autotune trial");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double sps = ms * 1e-3 / steps_per_trial;
            if (sps < best) {
                best = sps;
                best_bt = bt;
                best_bps = bps;
            }
        }
        if (st != GLBE_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GLBE_OK) return st;
    st = glbe_batch_set_launch(b, best_bt, best_bps);
    if (st != GLBE_OK) return st;
    st = reset_state(b, true);   // the trials advanced the state: back to rest
    if (st != GLBE_OK) return st;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(GLBE_ERR_CUDA, "autotune reset");
    if (block_threads_out) *block_threads_out = best_bt;
    if (blocks_per_sm_out) *blocks_per_sm_out = best_bps;
    if (seconds_per_step_out) *seconds_per_step_out = best;
    return GLBE_OK;
}

glbe_status glbe_batch_solve(glbe_batch* b, double tol, long max_steps, int use_graph, glbe_batch_result* res,
                             double* seconds_out)
{
    NvtxRange range_("glbe_batch_solve");
    if (!b || !res) return fail(GLBE_ERR_ARG, "batch or results is NULL");
    if (!(tol > 0.0) || max_steps < 1) return fail(GLBE_ERR_ARG, "tol must be > 0 and max_steps >= 1");
    if (b->t != 0) return fail(GLBE_ERR_STATE, "a batch solves once from the rest state: call glbe_batch_reset");
    glbe_status st = reset_state(b, false);
    if (st != GLBE_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(GLBE_ERR_CUDA, "event create");
    cudaEventRecord(e0, b->stream);
    if (use_graph) {
        cudaStream_t cap = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = launch_batch(b, max_steps, tol, cap);
            e = cudaStreamEndCapture(cap, &graph);
        }
        if (e == cudaSuccess && st == GLBE_OK) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess && st == GLBE_OK) e = cudaGraphLaunch(exec, b->stream);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
        if (st == GLBE_OK && e != cudaSuccess) st = fail(GLBE_ERR_CUDA, "batch graph: %s", cudaGetErrorString(e));
    } else {
        st = launch_batch(b, max_steps, tol, b->stream);
    }
    cudaEventRecord(e1, b->stream);
    cudaError_t es = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GLBE_OK) return st;
    if (es != cudaSuccess) return fail(GLBE_ERR_CUDA, "batch solve: %s", cudaGetErrorString(es));
    if (seconds_out) *seconds_out = ms * 1e-3;
    BatchState hs;
    std::vector<BatchDomainState> hd(b->n);
    cudaError_t e = cudaMemcpy(&hs, b->d_state, sizeof hs, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hd.data(), b->d_dstate, sizeof(BatchDomainState) * b->n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "batch results: %s", cudaGetErrorString(e));
    // levels reached: a converged domain stopped after the step that took its
    // residual; the others after max_steps
    long long last = -1;
    b->level.assign(b->n, b->t + max_steps);
    for (int d = 0; d < b->n; ++d) {
        if (!hd[d].active && hd[d].nonfinite == 0) b->level[d] = hd[d].conv_level + 1;
        res[d].converged = hd[d].active == 0 && hd[d].nonfinite == 0;
        res[d].steps = hd[d].active ? -1 : (long)hd[d].conv_level;
        res[d].r = hd[d].r;
        res[d].seconds = hd[d].active ? -1.0 : hd[d].conv_seconds;
        res[d].nonfinite = hd[d].nonfinite;
        if (hd[d].last_level > last) last = hd[d].last_level;
    }
    b->t = b->t + max_steps;   // marks the batch as solved (glbe_batch_reset restarts it)
    b->snap_level = last;
    if (hs.error) return fail(GLBE_ERR_TIMEOUT, "batch grid barrier timed out");
    for (int d = 0; d < b->n; ++d)
        if (hd[d].nonfinite) return fail(GLBE_ERR_DIVERGED, "domain %d: non-finite velocity", d);
    if (hs.n_active > 0) return fail(GLBE_ERR_TIMEOUT, "%d domains above tol after %ld steps", hs.n_active, max_steps);
    return GLBE_OK;
}

glbe_status glbe_batch_fields(glbe_batch* b, int d, float* d_rho, float* d_u, float* d_B)
{
    if (!b || d < 0 || d >= b->n) return fail(GLBE_ERR_ARG, "bad batch or domain");
    const BatchDomain& D = b->host_doms[d];
    StepBuffers sb{};
    const long long lvl = b->level.empty() ? b->t : b->level[d];
    const int par = (int)(lvl & 1);
    sb.fsrc = D.f[par];
    sb.gsrc = D.g[par];
    sb.FL = D.FL;
    sb.usnap = D.usnap;
    const FieldOut fo{d_rho, d_u, D.mhd ? d_B : nullptr};
    cudaError_t e;
    if (b->storage == GLBE_F32) e = launch_step_t<ST_F32>(D.mhd, MODE_FIELDS, D.p, sb, fo, b->stream, nullptr);
    else e = launch_step_t<ST_F32C>(D.mhd, MODE_FIELDS, D.p, sb, fo, b->stream, nullptr);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "batch fields: %s", cudaGetErrorString(e));
    return GLBE_OK;
}

glbe_status glbe_batch_reset(glbe_batch* b)
{
    if (!b) return fail(GLBE_ERR_ARG, "batch is NULL");
    b->level.clear();
    glbe_status st = reset_state(b, true);
    if (st != GLBE_OK) return st;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return fail(GLBE_ERR_CUDA, "batch reset sync");
    return GLBE_OK;
}

glbe_status glbe_batch_set_barrier_test(glbe_batch* b, long long spin_limit, int absent_block)
{
    if (!b) return fail(GLBE_ERR_ARG, "batch is NULL");
    if (spin_limit < 1) return fail(GLBE_ERR_ARG, "spin_limit must be >= 1");
    b->spin_limit = spin_limit;
    b->absent_block = absent_block;
    return GLBE_OK;
}

void glbe_batch_destroy(glbe_batch* b) { delete b; }

}  // extern "C"
