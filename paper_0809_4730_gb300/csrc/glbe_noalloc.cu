// glbe_noalloc.cu -- the allocation-free entry point glbe_step_residual_noalloc.
//
// Every other entry point of this library works on a workspace the caller
// allocated (glbe_workspace_bytes); part of that workspace is scratch: the
// per-block FP64 partial sums of the residual step and the record its finalize
// kernel writes.  Some callers cannot provide that: an application whose
// device memory is owned by another allocator (a framework's pool, a fixed
// arena) and that may not call cudaMalloc itself, for instance because an
// allocation would synchronise the device or fall outside the pool's budget.
// They hold the population and velocity buffers they already own and need one
// time step with the residual without any further device memory.
//
// For them the scratch lives in a file-scope static device array of fixed size
// (SCRATCH_DOUBLES doubles, a little over 1 MiB), which every GPU that loads
// this library holds until the process exits.  Host code cannot use the
// array's name as a device address (on the host it names a host-side stand-in;
// a kernel given it would fault or, where the GPU can reach host memory,
// silently use the wrong memory), so the address is looked up once per device
// with cudaGetSymbolAddress while that device is current.  The lookup is keyed
// on the device's current driver context as well: after cudaDeviceReset (or a
// primary context that was released and created again) the module is loaded
// anew and the array may sit elsewhere, so a new context triggers a new
// lookup.  Nothing here calls cudaMalloc, cudaFree or any allocating library
// routine.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "glbe.h"
#include "glbe_internal.h"

using namespace glbe;

namespace {

constexpr unsigned NOALLOC_MAX_BLOCKS = 16384;                       // step blocks of 256 nodes
constexpr size_t NOALLOC_MAX_NODES = (size_t)NOALLOC_MAX_BLOCKS * STEP_THREADS;
constexpr size_t PARTIAL_DOUBLES = (size_t)NOALLOC_MAX_BLOCKS * PARTIAL_STRIDE;
// partials [8][blocks], then one record, a one-record history, and the
// finalize kernel's counters (history count, residual level, tol, stop flag)
constexpr size_t SCRATCH_DOUBLES = PARTIAL_DOUBLES + 2 * RECORD_STRIDE + 8;

static __device__ __align__(256) double g_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_scratch_addr[MAX_DEVICES] = {};
CUcontext g_scratch_ctx[MAX_DEVICES] = {};   // driver context the address belongs to

// cuCtxGetCurrent through the runtime's driver entry point (the library links
// the static CUDA runtime only, not libcuda directly).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    return fn;
}

// Device address of g_scratch on the current device: looked up on the first
// call per device, and again whenever the device's current driver context is
// not the one the cached address was taken in.
glbe_status scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(GLBE_ERR_ARG, "device ordinal %d out of range", dev);
    // make the device's primary context current on this thread (a no-op when
    // it already is)
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    CUcontext ctx = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (!get || get(&ctx) != CUDA_SUCCESS || !ctx)
        return fail(GLBE_ERR_CUDA, "cuCtxGetCurrent is unavailable: cannot key the static scratch on its context");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(GLBE_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<double*>(ptr);
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return GLBE_OK;
}

// The array keeps the previous call's contents: reset the finalize kernel's
// counters, flag and tolerance before every use.
__global__ void reset_counters(unsigned long long* hist_count, long long* t_dev, double* tol, int* stop, long long t)
{
    *hist_count = 0;
    *t_dev = t;
    *tol = 0.0;
    *stop = 0;
}

}  // namespace

extern "C" glbe_status glbe_step_residual_noalloc(const glbe_params* p, const void* d_src, void* d_dst,
                                                  const float* d_force, float* d_u, int have_prev, long t,
                                                  glbe_residual_info* out)
{
    glbe_status st = validate_params(p);
    if (st != GLBE_OK) return st;
    if (p->induction) return fail(GLBE_ERR_ARG, "the allocation-free step covers the D3Q19 flow lattice only");
    if (make_step_params(p).cavity)
        return fail(GLBE_ERR_ARG, "the allocation-free step takes no fluid box or moving lid");
    if (!d_src || !d_dst || !d_u || !out) return fail(GLBE_ERR_ARG, "src, dst, u or out is NULL");
    if (d_src == d_dst) return fail(GLBE_ERR_ARG, "src and dst must be different buffers");
    if (p->force_field && !d_force) return fail(GLBE_ERR_ARG, "force_field > 0 needs a force field");
    // the step moves node pairs as 8-byte vectors: every buffer must be 16-byte aligned
    auto misaligned = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) != 0; };
    if (misaligned(d_src) || misaligned(d_dst) || misaligned(d_u) || (d_force && misaligned(d_force)))
        return fail(GLBE_ERR_ARG, "src, dst, u and force must be 16-byte aligned");
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    if (N > NOALLOC_MAX_NODES)
        return fail(GLBE_ERR_ARG, "grid of %zu nodes exceeds the allocation-free limit of %zu nodes", N,
                    NOALLOC_MAX_NODES);
    double* scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != GLBE_OK) return st;

    double* partials = scratch;
    double* record = scratch + PARTIAL_DOUBLES;
    double* hist = record + RECORD_STRIDE;
    double* misc = hist + RECORD_STRIDE;
    auto* hist_count = reinterpret_cast<unsigned long long*>(misc);
    auto* t_dev = reinterpret_cast<long long*>(misc + 1);
    double* tol = misc + 2;
    int* stop = reinterpret_cast<int*>(misc + 3);

    cudaStream_t stream = static_cast<cudaStream_t>(p->stream);
    const StepParams sp = make_step_params(p);
    StepBuffers b{};
    b.fsrc = d_src;
    b.fdst = d_dst;
    b.Ffield = p->force_field ? d_force : nullptr;
    b.usnap = d_u;
    b.partials = partials;
    b.have_snap = have_prev ? 1 : 0;
    b.stop = nullptr;
    b.sr_ctr = nullptr;              // stochastic rounding (the _SR forms) seeded by the time level
    b.sr_seed = (unsigned)t;
    const FieldOut fo{nullptr, nullptr, nullptr};

    unsigned grid = 0;   // blocks of the step launch (at most NOALLOC_MAX_BLOCKS for N within the limit)
    reset_counters<<<1, 1, 0, stream>>>(hist_count, t_dev, tol, stop, (long long)t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        switch (p->storage) {
        case GLBE_F32: e = launch_step_t<ST_F32>(false, MODE_STEP_RESID, sp, b, fo, stream, &grid); break;
        case GLBE_BF16: e = launch_step_t<ST_BF16>(false, MODE_STEP_RESID, sp, b, fo, stream, &grid); break;
        case GLBE_F16: e = launch_step_t<ST_F16>(false, MODE_STEP_RESID, sp, b, fo, stream, &grid); break;
        case GLBE_BF16_SR: e = launch_step_t<ST_BF16_SR>(false, MODE_STEP_RESID, sp, b, fo, stream, &grid); break;
        case GLBE_F16_SR: e = launch_step_t<ST_F16_SR>(false, MODE_STEP_RESID, sp, b, fo, stream, &grid); break;
        default: e = launch_step_t<ST_F32C>(false, MODE_STEP_RESID, sp, b, fo, stream, &grid); break;
        }
    }
    const long long fluid = fluid_nodes(p);
    if (e == cudaSuccess && have_prev)
        e = launch_finalize(partials, grid, p->rho0 * (double)fluid, t_dev, record, hist, hist_count, 1, stop, tol,
                            stream);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "allocation-free step: %s", cudaGetErrorString(e));
    // the record is read on the caller's stream (no device-wide synchronisation)
    double rec[RECORD_STRIDE];
    if (have_prev) {
        e = cudaMemcpyAsync(rec, record, sizeof rec, cudaMemcpyDeviceToHost, stream);
        if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "allocation-free record read: %s", cudaGetErrorString(e));
    }
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "allocation-free step sync: %s", cudaGetErrorString(e));
    // the TMA-staged tile kernel (variants 3 and 4) returns early when one of
    // its bounded pipeline waits runs out; its outputs are then incomplete
    int waited_out = 0;
    if (p->variant >= 3) switch (p->storage) {
    case GLBE_F32: waited_out = tile_wait_error_t<ST_F32>(); break;
    case GLBE_BF16: waited_out = tile_wait_error_t<ST_BF16>(); break;
    case GLBE_F16: waited_out = tile_wait_error_t<ST_F16>(); break;
    default: break;
    }
    if (waited_out) return fail(GLBE_ERR_TIMEOUT, "a pipeline wait of the TMA-staged step kernel ran out");

    std::memset(out, 0, sizeof *out);
    out->t = -1;
    if (!have_prev) return GLBE_OK;
    out->t = (long)rec[0];
    out->r = rec[1];
    out->num = rec[2];
    out->den = rec[3];
    out->mass = rec[4];
    out->momentum[0] = rec[5];
    out->momentum[1] = rec[6];
    out->momentum[2] = rec[7];
    out->nonfinite = (int)rec[8];
    if (out->nonfinite > 0 || !(out->r == out->r))
        return fail(GLBE_ERR_DIVERGED, "non-finite velocity at time level %ld", t);
    return GLBE_OK;
}
