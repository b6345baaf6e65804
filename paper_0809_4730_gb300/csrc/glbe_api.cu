// glbe_api.cu -- host side of the C-ABI declared in include/glbe.h.
//
// The library owns no device memory: glbe_init carves the caller's workspace
// into the two population buffers (ping-pong of the pull scheme), the lagged
// Lorentz force, the body-force field, the velocity snapshot of the residual,
// per-block FP64 partial sums and a small record/history area.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "glbe.h"
#include "glbe_internal.h"

using namespace glbe;

namespace {

thread_local std::string g_last_error;

}  // namespace

glbe_status glbe::fail(glbe_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

namespace {

glbe_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(GLBE_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define GLBE_CUDA(call, what)                         \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr double THETA_M = 0.25;        // theta_m = 1/N_m, N_m = 4 (Sec. 4)
constexpr unsigned HIST_CAP = 4096;     // residual records kept on the device
constexpr size_t ALIGN = 256;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    size_t f[2], g[2], FL, Ffield, usnap, partials, record, hist, misc, Fstage, total;
};

size_t storage_bytes(int st) { return st == GLBE_F32 ? 4 : (st == GLBE_F32C ? 6 : 2); }   // the others: 16 bits

unsigned step_grid(size_t N) { return (unsigned)((N + STEP_THREADS - 1) / STEP_THREADS); }

// Rows of the velocity snapshot: the FP32 and compensated forms keep u as a
// double-float pair (high and low parts), the 16-bit forms the high part.
size_t snap_rows(int st) { return (st == GLBE_F32 || st == GLBE_F32C) ? 6 : 3; }

Layout make_layout(const glbe_params* p)
{
    Layout L{};
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    const size_t ss = storage_bytes(p->storage);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    L.f[0] = take(19 * N * ss);
    L.f[1] = take(19 * N * ss);
    if (p->induction) {
        L.g[0] = take(21 * N * ss);
        L.g[1] = take(21 * N * ss);
        L.FL = take(3 * N * sizeof(float));
    } else {
        L.g[0] = L.g[1] = L.FL = (size_t)-1;
    }
    L.Ffield = p->force_field ? take((size_t)p->force_field * N * sizeof(float)) : (size_t)-1;
    L.usnap = take(snap_rows(p->storage) * N * sizeof(float));
    L.partials = take((size_t)step_grid(N) * PARTIAL_STRIDE * sizeof(double));
    L.record = take(RECORD_STRIDE * sizeof(double));
    L.hist = take((size_t)HIST_CAP * RECORD_STRIDE * sizeof(double));
    L.misc = take(64);
    // staging buffer of glbe_set_force_host (last, outside the region the
    // initial memset clears)
    L.Fstage = p->force_field ? take((size_t)p->force_field * N * sizeof(float)) : (size_t)-1;
    L.total = off;
    return L;
}

}  // namespace

glbe_status glbe::validate_params(const glbe_params* p)
{
    if (!p) return fail(GLBE_ERR_ARG, "params is NULL");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(GLBE_ERR_ARG, "grid sizes must be >= 1");
    const unsigned long long N = (unsigned long long)p->nx * p->ny * p->nz;
    if (N >= (1ull << 31)) return fail(GLBE_ERR_ARG, "nx*ny*nz = %llu must be < 2^31", N);
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int d = 0; d < 3; ++d) {
        if ((p->wall_lo[d] | p->wall_hi[d]) & ~1) return fail(GLBE_ERR_ARG, "wall flags must be 0 or 1");
        if (n[d] - p->wall_lo[d] - p->wall_hi[d] < 1)
            return fail(GLBE_ERR_ARG, "axis %d has no fluid plane between its walls", d);
    }
    if (!(p->rho0 > 0.0)) return fail(GLBE_ERR_ARG, "rho0 must be > 0");
    if (!(p->gamma > 0.0 && p->gamma <= 1.0)) return fail(GLBE_ERR_ARG, "gamma must be in (0, 1]");
    if (!(p->nu > 0.0)) return fail(GLBE_ERR_ARG, "nu must be > 0");
    for (int k = 0; k < 19; ++k)
        if (!(p->s[k] > 0.0 && p->s[k] < 2.0)) return fail(GLBE_ERR_ARG, "s[%d] = %g must be in (0, 2)", k, p->s[k]);
    if (p->force_field != 0 && p->force_field != 1 && p->force_field != 3)
        return fail(GLBE_ERR_ARG, "force_field must be 0, 1 or 3");
    if (p->induction != 0 && p->induction != 1) return fail(GLBE_ERR_ARG, "induction must be 0 or 1");
    if (p->induction) {
        if (!(p->gamma_m > 0.0 && p->gamma_m <= 1.0)) return fail(GLBE_ERR_ARG, "gamma_m must be in (0, 1]");
        if (!(p->eta > 0.0)) return fail(GLBE_ERR_ARG, "eta must be > 0");
        if (!(p->chi > 0.0)) return fail(GLBE_ERR_ARG, "chi must be > 0");
        if (!(p->mu > 0.0)) return fail(GLBE_ERR_ARG, "mu must be > 0");
    }
    if (p->storage < GLBE_F32 || p->storage > GLBE_F16_SR)
        return fail(GLBE_ERR_ARG, "storage must be GLBE_F32, GLBE_BF16, GLBE_F16, GLBE_F32C, GLBE_BF16_SR or GLBE_F16_SR");
    if (p->variant < 0 || p->variant > 4) return fail(GLBE_ERR_ARG, "variant must be 0 ... 4");
    if (p->storage_scale < 0.0 || !std::isfinite(p->storage_scale))
        return fail(GLBE_ERR_ARG, "storage_scale must be >= 0 and finite");
    if ((p->ghost_lo | p->ghost_hi) & ~1) return fail(GLBE_ERR_ARG, "ghost flags must be 0 or 1");
    if (p->collision < 0 || p->collision > 2) return fail(GLBE_ERR_ARG, "collision must be 0 (MRT), 1 or 2 (SRT)");
    if (p->collision && p->storage != GLBE_F32 && p->storage != GLBE_F32C && p->storage != GLBE_BF16)
        return fail(GLBE_ERR_ARG, "the SRT collision takes F32, F32C or BF16 storage");
    if (p->box != 0 && p->box != 1) return fail(GLBE_ERR_ARG, "box must be 0 or 1");
    const bool lid = p->U_lid[0] != 0.0 || p->U_lid[1] != 0.0 || p->U_lid[2] != 0.0;
    if (p->box || lid) {
        if (p->storage != GLBE_F32 && p->storage != GLBE_F32C && p->storage != GLBE_BF16)
            return fail(GLBE_ERR_ARG, "a fluid box or a moving lid takes F32, F32C or BF16 storage");
        if (p->collision == 2 || (p->collision == 1 && p->storage != GLBE_F32))
            return fail(GLBE_ERR_ARG, "the cavity kernel runs the MRT or, with F32 storage, the SRT collision");
        if (p->ghost_lo || p->ghost_hi) return fail(GLBE_ERR_ARG, "a cavity is not split into slabs");
        if (p->box)
            for (int d = 0; d < 3; ++d)
                if (p->box_lo[d] < 0 || p->box_hi[d] >= n[d] || p->box_lo[d] > p->box_hi[d])
                    return fail(GLBE_ERR_ARG, "box axis %d: need 0 <= box_lo <= box_hi < n", d);
        if (fluid_nodes(p) < 1) return fail(GLBE_ERR_ARG, "the fluid box holds no node off the walls");
        for (int d = 0; d < 3; ++d)
            if (!std::isfinite(p->U_lid[d])) return fail(GLBE_ERR_ARG, "U_lid must be finite");
    }
    if ((p->ghost_lo && p->wall_lo[2]) || (p->ghost_hi && p->wall_hi[2]))
        return fail(GLBE_ERR_ARG, "a z face has either a wall or a ghost plane");
    if (p->nz - p->wall_lo[2] - p->wall_hi[2] - p->ghost_lo - p->ghost_hi < 1)
        return fail(GLBE_ERR_ARG, "no computed z plane between the ghost and wall planes");
    return GLBE_OK;
}

StepParams glbe::make_step_params(const glbe_params* p)
{
    StepParams s{};
    s.nx = p->nx;
    s.ny = p->ny;
    s.nz = p->nz;
    s.N = (uint32_t)((size_t)p->nx * p->ny * p->nz);
    s.div_nx = make_fastdiv((uint32_t)p->nx);
    s.div_nxy = make_fastdiv((uint32_t)(p->nx * p->ny));
    s.glo_z = p->ghost_lo;
    s.ghi_z = p->ghost_hi;
    s.box = p->box;
    for (int d = 0; d < 3; ++d) {
        s.blo[d] = p->box ? p->box_lo[d] : 0;
        s.bhi[d] = p->box ? p->box_hi[d] : (d == 0 ? p->nx : d == 1 ? p->ny : p->nz) - 1;
    }
    s.top_z = p->box ? p->box_hi[2] : (p->wall_hi[2] ? p->nz - 2 : p->nz - 1);
    {
        // moving-wall term of the lid, 6 w_a rho0 (e_a . U_lid), in the ordering of include/glbe.h
        static const int E[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                     {1, 1, 0},  {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1}, {1, 0, -1},
                                     {-1, 0, -1}, {0, 1, 1}, {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};
        for (int a = 0; a < 19; ++a) {
            const double w = a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
            const double eU = E[a][0] * p->U_lid[0] + E[a][1] * p->U_lid[1] + E[a][2] * p->U_lid[2];
            s.lid_corr[a] = (float)(6.0 * w * p->rho0 * eU);
        }
        const bool lid = p->U_lid[0] != 0.0 || p->U_lid[1] != 0.0 || p->U_lid[2] != 0.0;
        s.cavity = (p->box || lid) ? 1 : 0;
    }
    for (int d = 0; d < 3; ++d) {
        s.wlo[d] = p->wall_lo[d];
        s.whi[d] = p->wall_hi[d];
        s.F[d] = (float)p->F[d];
        s.B0[d] = (float)p->B0[d];
        s.bwall_dev[d] = 0.f;
    }
    s.rho0 = (float)p->rho0;
    s.inv_gamma = (float)(1.0 / p->gamma);
    s.inv_gamma2 = (float)(1.0 / (p->gamma * p->gamma));
    // Lambda*: 1/s_nu* = 3 nu / gamma + 1/2 on the viscous rows (Sec. 3)
    const double snu = 1.0 / (3.0 * p->nu / p->gamma + 0.5);
    for (int k = 0; k < 19; ++k) s.s[k] = (float)p->s[k];
    s.s[9] = s.s[11] = s.s[13] = s.s[14] = s.s[15] = (float)snu;
    {
        // folded relaxation per row (App. A tables): |row_k|^2, P_S,k and the
        // constant c_k of S_k = c_k R_k
        static const double norm2[19] = {19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8};
        const double ig = 1.0 / p->gamma, ig2 = ig * ig;
        const double ps[19] = {1, ig2, ig2, ig, ig, ig, ig, ig, ig, ig2, ig2, ig2, ig2, ig2, ig2, ig2, 1, 1, 1};
        const double ck[19] = {0, 38, -11, 0, -2.0 / 3.0, 0, -2.0 / 3.0, 0, -2.0 / 3.0, 2, -1, 2, -1, 1, 1, 1, 0, 0, 0};
        for (int k = 0; k < 19; ++k) {
            const double sk = (k == 9 || k == 11 || k == 13 || k == 14 || k == 15) ? snu : p->s[k];
            s.rl_a[k] = (float)(-sk / norm2[k]);
            s.rl_b[k] = (float)((1.0 - 0.5 * sk) * ps[k] * ck[k] / norm2[k]);
            s.rl_c[k] = (float)((1.0 - sk) / norm2[k]);
        }
        s.rl_cons = (float)(ig / 10.0);
    }
    s.force_ncomp = p->force_field;
    if (p->induction) {
        // tau_m* = eta / (gamma_m theta_m) + 1/2 (Eq. mrelaxationtime)
        const double tau_m = p->eta / (p->gamma_m * THETA_M) + 0.5;
        s.conv_coef = (float)(p->chi / p->gamma_m);
        s.omega_m = (float)(1.0 / tau_m);
        s.J_coef = (float)(-1.0 / (p->mu * p->chi * tau_m * THETA_M));
    }
    double scale = p->storage_scale;
    if (p->storage != GLBE_F16 && p->storage != GLBE_F16_SR) scale = 1.0;   // only FP16 stores scaled deviations
    else if (scale == 0.0) scale = 4096.0;
    s.scale = (float)scale;
    s.inv_scale = (float)(1.0 / scale);
    s.variant = p->variant;
    s.collision = p->collision;
    s.storage = p->storage;
    // interior nodes: on each axis lo = 1 + wall_lo, hi = n - 2 - wall_hi
    // (neighbours neither on a wall plane nor across the periodic seam); on
    // an x axis without walls the whole axis, since the gather corrects the
    // sources that cross the x seam (a warp covers x-consecutive nodes, so
    // the seam nodes would otherwise split their warps between two paths)
    s.interior_ok = 1;
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int d = 0; d < 3; ++d) {
        int lo = 1 + p->wall_lo[d], hi = n[d] - 2 - p->wall_hi[d];
        if (d == 0 && !p->wall_lo[0] && !p->wall_hi[0]) { lo = 0; hi = n[0] - 1; }
        if (hi < lo) s.interior_ok = 0;
        s.ilo[d] = (uint32_t)lo;
        s.ispan[d] = hi >= lo ? (uint32_t)(hi - lo) : 0u;
    }
    if (s.cavity) {
        // interior nodes of a cavity: inside the box with a margin of one node
        // (no bounced link, none to the lid); on an axis the box spans whole
        // without walls the periodic-seam rule of the plain grid stays
        const int n[3] = {p->nx, p->ny, p->nz};
        s.interior_ok = 1;
        for (int d = 0; d < 3; ++d) {
            if (p->box && p->box_lo[d] == 0 && p->box_hi[d] == n[d] - 1 && !p->wall_lo[d] && !p->wall_hi[d]) continue;
            int lo = (p->box ? p->box_lo[d] : 0) + 1, hi = (p->box ? p->box_hi[d] : n[d] - 1) - 1;
            if (lo < 1 + p->wall_lo[d]) lo = 1 + p->wall_lo[d];
            if (hi > n[d] - 2 - p->wall_hi[d]) hi = n[d] - 2 - p->wall_hi[d];
            if (d == 2 && hi > s.top_z - 1) hi = s.top_z - 1;
            if (hi < lo) s.interior_ok = 0;
            s.ilo[d] = (uint32_t)lo;
            s.ispan[d] = hi >= lo ? (uint32_t)(hi - lo) : 0u;
        }
    }
    // D3Q19 directions in the order of include/glbe.h
    static const int E[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                 {1, 1, 0},  {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0}, {1, 0, 1},  {-1, 0, 1}, {1, 0, -1},
                                 {-1, 0, -1}, {0, 1, 1}, {0, -1, 1}, {0, 1, -1}, {0, -1, -1}};
    const long long Nn = (long long)p->nx * p->ny * p->nz, sx = 1, sy = p->nx, sz = (long long)p->nx * p->ny;
    for (int a = 0; a < 19; ++a) {
        s.doff[a] = a * Nn - (E[a][0] * sx + E[a][1] * sy + E[a][2] * sz);
        s.toff[a] = a * Nn + (E[a][0] * sx + E[a][1] * sy + E[a][2] * sz);
    }
    return s;
}

namespace {

constexpr int FIN_THREADS = 1024;

__global__ void __launch_bounds__(FIN_THREADS) finalize_kernel(const double* __restrict__ partials, unsigned nblocks,
                                                               double mass0, long long* t_dev, double* record,
                                                               double* hist, unsigned long long* hist_count,
                                                               unsigned hist_cap, int* stop, const double* tol)
{
    if (*stop) return;   // a solve already converged: the chunk's remaining work is skipped
    __shared__ double sh[7][FIN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 7; ++k) {
        // partials are [k][block]: consecutive threads read consecutive blocks
        const double* pk = partials + (size_t)k * nblocks;
        double s = 0.0;
        for (unsigned b = threadIdx.x; b < nblocks; b += FIN_THREADS) s += pk[b];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[k][warp] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[7];
        for (int k = 0; k < 7; ++k) {
            double s = 0.0;
            for (int w = 0; w < FIN_THREADS / 32; ++w) s += sh[k][w];
            tot[k] = s;
        }
        const double num = tot[0], den = tot[1];
        const double r = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
        const long long t = *t_dev;
        double rec[RECORD_STRIDE] = {0};
        rec[0] = (double)t;
        rec[1] = r;
        rec[2] = num;
        rec[3] = den;
        rec[4] = mass0 + tot[2];
        rec[5] = tot[3];
        rec[6] = tot[4];
        rec[7] = tot[5];
        rec[8] = tot[6];
        for (int k = 0; k < RECORD_STRIDE; ++k) record[k] = rec[k];
        const unsigned long long c = *hist_count;
        double* h = hist + (size_t)(c % hist_cap) * RECORD_STRIDE;
        for (int k = 0; k < RECORD_STRIDE; ++k) h[k] = rec[k];
        *hist_count = c + 1;
        *t_dev = t + 10;
        if ((*tol > 0.0 && r <= *tol) || rec[8] > 0.0 || !isfinite(r)) *stop = 1;
    }
}

// First stage of the residual reduction for large grids: block b sums the
// partials of blocks [b*chunk, (b+1)*chunk) of the step (fixed order) into
// row 7 of the partials, which the step leaves unused: out[k][b].
constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS) partial_reduce_kernel(const double* __restrict__ partials,
                                                                     unsigned nblocks, unsigned fb, double* out,
                                                                     const int* stop)
{
    if (*stop) return;
    __shared__ double sh[RED_THREADS / 32];
    const unsigned chunk = (nblocks + fb - 1) / fb;
    const unsigned b0 = blockIdx.x * chunk, b1 = b0 + chunk < nblocks ? b0 + chunk : nblocks;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 7; ++k) {
        const double* pk = partials + (size_t)k * nblocks;
        double s = 0.0;
        for (unsigned b = b0 + threadIdx.x; b < b1; b += RED_THREADS) s += pk[b];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < RED_THREADS / 32; ++w) t += sh[w];
            out[(size_t)k * fb + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

__global__ void misc_set_kernel(long long* t_dev, long long t, int* stop, int stop_v, double* tol, double tol_v,
                                double* record, unsigned long long* hist_count, int reset_record)
{
    if (t_dev) *t_dev = t;
    if (stop) *stop = stop_v;
    if (tol) *tol = tol_v;
    if (reset_record) {
        for (int k = 0; k < RECORD_STRIDE; ++k) record[k] = 0.0;
        record[0] = -1.0;
        *hist_count = 0;
    }
}

}  // namespace

struct glbe_ctx {
    glbe_params prm;
    StepParams sp;
    Layout L;
    size_t N;
    unsigned grid;
    char* ws;
    void* f[2];
    void* g[2];
    float* FL;
    float* Ffield;
    float* usnap;
    double* partials;
    double* record;
    double* hist;
    unsigned long long* hist_count;
    long long* t_dev;
    int* stop_dev;
    double* tol_dev;
    unsigned* sr_ctr;   // [2] seeds of stochastic rounding, read by the step of parity t & 1
    double mass0;   // rho0 x number of fluid nodes
    long t;         // current time level
    long t_snap;    // level of the velocity snapshot, -1 if none
    cudaStream_t stream;
    cudaStream_t cap_stream;
    cudaGraphExec_t chunk;
    // host force uploads: staged on their own stream (created on first use)
    float* Fstage;
    cudaStream_t copy_stream;
    cudaEvent_t ev_staged;       // the host copy into Fstage is complete
    cudaEvent_t ev_stage_free;   // the hand-over from Fstage to Ffield is complete
};

namespace {

cudaError_t launch_step_any(glbe_ctx* c, int mode, const StepBuffers& b, const FieldOut& fo, cudaStream_t st,
                            unsigned* nblocks)
{
    switch (c->prm.storage) {
    case GLBE_F32: return launch_step_t<ST_F32>(c->prm.induction, mode, c->sp, b, fo, st, nblocks);
    case GLBE_BF16: return launch_step_t<ST_BF16>(c->prm.induction, mode, c->sp, b, fo, st, nblocks);
    case GLBE_F16: return launch_step_t<ST_F16>(c->prm.induction, mode, c->sp, b, fo, st, nblocks);
    case GLBE_BF16_SR: return launch_step_t<ST_BF16_SR>(c->prm.induction, mode, c->sp, b, fo, st, nblocks);
    case GLBE_F16_SR: return launch_step_t<ST_F16_SR>(c->prm.induction, mode, c->sp, b, fo, st, nblocks);
    default: return launch_step_t<ST_F32C>(c->prm.induction, mode, c->sp, b, fo, st, nblocks);
    }
}

StepBuffers buffers_for(glbe_ctx* c, long t)
{
    StepBuffers b{};
    const int s = (int)(t & 1);
    b.fsrc = c->f[s];
    b.fdst = c->f[s ^ 1];
    b.gsrc = c->prm.induction ? c->g[s] : nullptr;
    b.gdst = c->prm.induction ? c->g[s ^ 1] : nullptr;
    b.FL = c->FL;
    b.Ffield = c->Ffield;
    b.usnap = c->usnap;
    b.partials = c->partials;
    b.have_snap = 0;
    b.stop = nullptr;
    b.snap_lo = snap_rows(c->prm.storage) == 6 ? 1 : 0;
    b.sr_ctr = c->sr_ctr;
    b.sr_par = s;
    b.sr_seed = 0;
    return b;
}

// Enqueues the step from level c->t to c->t + 1 on stream st.
glbe_status enqueue_step(glbe_ctx* c, cudaStream_t st, const int* stop)
{
    StepBuffers b = buffers_for(c, c->t);
    b.stop = stop;
    const FieldOut fo{nullptr, nullptr, nullptr};
    if (c->t % 10 == 0) {
        b.have_snap = (c->t_snap >= 0 && c->t_snap == c->t - 10) ? 1 : 0;
        unsigned nb = 0;
        GLBE_CUDA(launch_step_any(c, MODE_STEP_RESID, b, fo, st, &nb), "step kernel (residual)");
        if (b.have_snap) {
            GLBE_CUDA(launch_finalize(c->partials, nb, c->mass0, c->t_dev, c->record, c->hist, c->hist_count,
                                      HIST_CAP, c->stop_dev, c->tol_dev, st),
                      "residual finalize");
        } else {
            misc_set_kernel<<<1, 1, 0, st>>>(c->t_dev, (long long)c->t + 10, nullptr, 0, nullptr, 0.0, nullptr,
                                             nullptr, 0);
            GLBE_CUDA(cudaGetLastError(), "set residual level");
        }
        c->t_snap = c->t;
    } else {
        GLBE_CUDA(launch_step_any(c, MODE_STEP, b, fo, st, nullptr), "step kernel");
    }
    c->t += 1;
    return GLBE_OK;
}

}  // namespace

namespace glbe {
size_t storage_value_bytes(int storage) { return storage_bytes(storage); }

glbe_status ctx_view(glbe_ctx* c, CtxView* v)
{
    if (!c || !v) return fail(GLBE_ERR_ARG, "ctx or view is NULL");
    const int s = (int)(c->t & 1);
    v->prm = c->prm;
    v->sp = c->sp;
    v->N = c->N;
    v->t = c->t;
    v->fsrc = c->f[s];
    v->gsrc = c->prm.induction ? c->g[s] : nullptr;
    v->FL = c->FL;
    v->Ffield = c->Ffield;
    v->f_bytes = 19 * c->N * storage_bytes(c->prm.storage);
    v->g_bytes = c->prm.induction ? 21 * c->N * storage_bytes(c->prm.storage) : 0;
    v->stream = c->stream;
    return GLBE_OK;
}

cudaError_t launch_finalize(const double* partials, unsigned nblocks, double mass0, long long* t_dev, double* record,
                            double* hist, unsigned long long* hist_count, unsigned hist_cap, int* stop,
                            const double* tol, cudaStream_t st)
{
    // large grids: a first stage over many blocks (one SM alone reads the
    // 7 x nblocks partials at a fraction of the HBM bandwidth), its results
    // in the unused row 7 of the partials; then the one-block finalize
    constexpr unsigned PER_BLOCK = 512;
    if (nblocks >= 2 * PER_BLOCK) {
        unsigned fb = nblocks / PER_BLOCK;
        if (7 * fb > nblocks) fb = nblocks / 7;
        double* row7 = const_cast<double*>(partials) + (size_t)7 * nblocks;
        partial_reduce_kernel<<<fb, RED_THREADS, 0, st>>>(partials, nblocks, fb, row7, stop);
        finalize_kernel<<<1, FIN_THREADS, 0, st>>>(row7, fb, mass0, t_dev, record, hist, hist_count, hist_cap, stop,
                                                   tol);
    } else {
        finalize_kernel<<<1, FIN_THREADS, 0, st>>>(partials, nblocks, mass0, t_dev, record, hist, hist_count,
                                                   hist_cap, stop, tol);
    }
    return cudaGetLastError();
}
}  // namespace glbe

extern "C" {

int glbe_abi_version(void) { return GLBE_ABI_VERSION; }

void glbe_struct_sizes(size_t* params_bytes, size_t* info_bytes)
{
    if (params_bytes) *params_bytes = sizeof(glbe_params);
    if (info_bytes) *info_bytes = sizeof(glbe_residual_info);
}

const char* glbe_last_error(void) { return g_last_error.c_str(); }

void glbe_params_default(glbe_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->rho0 = 1.0;
    p->gamma = 1.0;
    for (int k = 0; k < 19; ++k) p->s[k] = 1.0;
    // kinetic rates of the D3Q19 model quoted in Sec. 3
    p->s[1] = 1.19;
    p->s[2] = p->s[10] = p->s[12] = 1.4;
    p->s[4] = p->s[6] = p->s[8] = 1.2;
    p->s[16] = p->s[17] = p->s[18] = 1.98;
    p->gamma_m = 1.0;
    p->eta = 0.0;
    p->chi = 1.0;
    p->mu = 1.0;
    p->storage = GLBE_F32;
    p->storage_scale = 0.0;
    p->stream = nullptr;
}

glbe_status glbe_workspace_bytes(const glbe_params* p, size_t* bytes)
{
    if (!bytes) return fail(GLBE_ERR_ARG, "bytes is NULL");
    glbe_status s = validate_params(p);
    if (s != GLBE_OK) return s;
    *bytes = make_layout(p).total;
    return GLBE_OK;
}

glbe_status glbe_init(const glbe_params* p, void* d_workspace, size_t bytes, glbe_ctx** out)
{
    if (!out) return fail(GLBE_ERR_ARG, "out is NULL");
    *out = nullptr;
    glbe_status s = validate_params(p);
    if (s != GLBE_OK) return s;
    if (!d_workspace) return fail(GLBE_ERR_ARG, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(d_workspace) % ALIGN) != 0)
        return fail(GLBE_ERR_ARG, "workspace must be %zu-byte aligned", ALIGN);
    const Layout L = make_layout(p);
    if (bytes < L.total) return fail(GLBE_ERR_ARG, "workspace of %zu bytes is smaller than the %zu needed", bytes, L.total);

    glbe_ctx* c = new (std::nothrow) glbe_ctx();
    if (!c) return fail(GLBE_ERR_ARG, "out of host memory");
    c->prm = *p;
    c->sp = make_step_params(p);
    c->L = L;
    c->N = (size_t)p->nx * p->ny * p->nz;
    c->grid = step_grid(c->N);
    c->ws = static_cast<char*>(d_workspace);
    c->f[0] = c->ws + L.f[0];
    c->f[1] = c->ws + L.f[1];
    c->g[0] = p->induction ? c->ws + L.g[0] : nullptr;
    c->g[1] = p->induction ? c->ws + L.g[1] : nullptr;
    c->FL = p->induction ? reinterpret_cast<float*>(c->ws + L.FL) : nullptr;
    c->Ffield = p->force_field ? reinterpret_cast<float*>(c->ws + L.Ffield) : nullptr;
    c->Fstage = p->force_field ? reinterpret_cast<float*>(c->ws + L.Fstage) : nullptr;
    c->usnap = reinterpret_cast<float*>(c->ws + L.usnap);
    c->partials = reinterpret_cast<double*>(c->ws + L.partials);
    c->record = reinterpret_cast<double*>(c->ws + L.record);
    c->hist = reinterpret_cast<double*>(c->ws + L.hist);
    char* misc = c->ws + L.misc;
    c->hist_count = reinterpret_cast<unsigned long long*>(misc);
    c->t_dev = reinterpret_cast<long long*>(misc + 8);
    c->tol_dev = reinterpret_cast<double*>(misc + 16);
    c->stop_dev = reinterpret_cast<int*>(misc + 24);
    c->sr_ctr = reinterpret_cast<unsigned*>(misc + 32);
    c->mass0 = p->rho0 * (double)fluid_nodes(p);   // planes on walls and ghost planes excluded
    c->t = 0;
    c->t_snap = -1;
    c->stream = static_cast<cudaStream_t>(p->stream);
    c->cap_stream = nullptr;
    c->chunk = nullptr;
    c->copy_stream = nullptr;
    c->ev_staged = c->ev_stage_free = nullptr;

    // rest state: all deviations zero (all-zero bits in every storage type)
    cudaError_t e = cudaMemsetAsync(c->ws, 0, L.usnap, c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->ws + L.usnap, 0, snap_rows(p->storage) * c->N * sizeof(float), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->sr_ctr, 0, 2 * sizeof(unsigned), c->stream);
    if (e == cudaSuccess && c->sp.cavity) {   // the lid's links of the first gather (see lid_init_kernel)
        if (p->storage == GLBE_F32) e = launch_lid_init_t<ST_F32>(c->sp, c->f[0], c->stream);
        else if (p->storage == GLBE_F32C) e = launch_lid_init_t<ST_F32C>(c->sp, c->f[0], c->stream);
        else e = launch_lid_init_t<ST_BF16>(c->sp, c->f[0], c->stream);
    }
    if (e == cudaSuccess) {
        misc_set_kernel<<<1, 1, 0, c->stream>>>(c->t_dev, 10, c->stop_dev, 0, c->tol_dev, 0.0, c->record,
                                                c->hist_count, 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "glbe_init");
    }
    *out = c;
    return GLBE_OK;
}

void glbe_destroy(glbe_ctx* c)
{
    if (!c) return;
    if (c->chunk) cudaGraphExecDestroy(c->chunk);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    if (c->ev_staged) cudaEventDestroy(c->ev_staged);
    if (c->ev_stage_free) cudaEventDestroy(c->ev_stage_free);
    delete c;
}

glbe_status glbe_set_force(glbe_ctx* c, const float* d_F)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    if (!c->prm.force_field) return fail(GLBE_ERR_STATE, "context was created with force_field = 0");
    if (!d_F) return fail(GLBE_ERR_ARG, "force field is NULL");
    GLBE_CUDA(cudaMemcpyAsync(c->Ffield, d_F, (size_t)c->prm.force_field * c->N * sizeof(float),
                              cudaMemcpyDeviceToDevice, c->stream),
              "glbe_set_force");
    return GLBE_OK;
}

glbe_status glbe_set_force_host(glbe_ctx* c, const float* h_F)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    if (!c->prm.force_field) return fail(GLBE_ERR_STATE, "context was created with force_field = 0");
    if (!h_F) return fail(GLBE_ERR_ARG, "force field is NULL");
    const size_t bytes = (size_t)c->prm.force_field * c->N * sizeof(float);
    if (!c->copy_stream) {
        // all three or none: a failed creation leaves the context as it was
        cudaStream_t cs = nullptr;
        cudaEvent_t e1 = nullptr, e2 = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&e2, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            if (e2) cudaEventDestroy(e2);
            if (e1) cudaEventDestroy(e1);
            if (cs) cudaStreamDestroy(cs);
            return cuda_fail(e, "glbe_set_force_host");
        }
        c->copy_stream = cs;
        c->ev_staged = e1;
        c->ev_stage_free = e2;
    }
    // The host copy runs on the copy stream into the staging buffer, so it
    // overlaps the steps already enqueued on the context's stream (they read
    // Ffield); the context's stream then waits for it and hands the field
    // over with a device copy (Ffield keeps its address: captured graphs stay
    // valid).  A second upload waits until the first hand-over is done.
    GLBE_CUDA(cudaStreamWaitEvent(c->copy_stream, c->ev_stage_free, 0), "glbe_set_force_host");
    GLBE_CUDA(cudaMemcpyAsync(c->Fstage, h_F, bytes, cudaMemcpyHostToDevice, c->copy_stream), "glbe_set_force_host");
    GLBE_CUDA(cudaEventRecord(c->ev_staged, c->copy_stream), "glbe_set_force_host");
    GLBE_CUDA(cudaStreamWaitEvent(c->stream, c->ev_staged, 0), "glbe_set_force_host");
    GLBE_CUDA(cudaMemcpyAsync(c->Ffield, c->Fstage, bytes, cudaMemcpyDeviceToDevice, c->stream), "glbe_set_force_host");
    GLBE_CUDA(cudaEventRecord(c->ev_stage_free, c->stream), "glbe_set_force_host");
    return GLBE_OK;
}

glbe_status glbe_step_n(glbe_ctx* c, long n)
{
    NvtxRange range_("glbe_step_n");
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    if (n < 0) return fail(GLBE_ERR_ARG, "n must be >= 0");
    for (long k = 0; k < n; ++k) {
        glbe_status s = enqueue_step(c, c->stream, nullptr);
        if (s != GLBE_OK) return s;
    }
    return GLBE_OK;
}

glbe_status glbe_sync(glbe_ctx* c)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    GLBE_CUDA(cudaStreamSynchronize(c->stream), "glbe_sync");
    int waited_out = 0;
    switch (c->prm.storage) {
    case GLBE_F32: waited_out = tile_wait_error_t<ST_F32>(); break;
    case GLBE_BF16: waited_out = tile_wait_error_t<ST_BF16>(); break;
    case GLBE_F16: waited_out = tile_wait_error_t<ST_F16>(); break;
    default: break;
    }
    if (waited_out) return fail(GLBE_ERR_TIMEOUT, "a pipeline wait of the TMA-staged step kernel ran out");
    return GLBE_OK;
}

static glbe_status read_record(glbe_ctx* c, glbe_residual_info* out)
{
    double rec[RECORD_STRIDE];
    GLBE_CUDA(cudaStreamSynchronize(c->stream), "residual sync");
    GLBE_CUDA(cudaMemcpy(rec, c->record, sizeof rec, cudaMemcpyDeviceToHost), "residual read");
    out->t = (long)rec[0];
    out->r = rec[1];
    out->num = rec[2];
    out->den = rec[3];
    out->mass = rec[4];
    out->momentum[0] = rec[5];
    out->momentum[1] = rec[6];
    out->momentum[2] = rec[7];
    out->nonfinite = (int)rec[8];
    if (out->t >= 0 && (out->nonfinite > 0 || !std::isfinite(out->r)))
        return fail(GLBE_ERR_DIVERGED, "non-finite velocity at time level %ld", out->t);
    return GLBE_OK;
}

glbe_status glbe_history(glbe_ctx* c, glbe_residual_info* out, long cap, long* n)
{
    if (!c || !n || (cap > 0 && !out)) return fail(GLBE_ERR_ARG, "ctx, out or n is NULL");
    *n = 0;
    if (cap <= 0) return GLBE_OK;
    unsigned long long count = 0;
    GLBE_CUDA(cudaStreamSynchronize(c->stream), "history sync");
    GLBE_CUDA(cudaMemcpy(&count, c->hist_count, sizeof count, cudaMemcpyDeviceToHost), "history count");
    const unsigned long long kept = count < HIST_CAP ? count : HIST_CAP;
    const unsigned long long take = kept < (unsigned long long)cap ? kept : (unsigned long long)cap;
    double rec[RECORD_STRIDE];
    for (unsigned long long i = 0; i < take; ++i) {
        const unsigned long long k = count - take + i;
        GLBE_CUDA(cudaMemcpy(rec, c->hist + (size_t)(k % HIST_CAP) * RECORD_STRIDE, sizeof rec,
                             cudaMemcpyDeviceToHost), "history read");
        glbe_residual_info& o = out[i];
        o.t = (long)rec[0];
        o.r = rec[1];
        o.num = rec[2];
        o.den = rec[3];
        o.mass = rec[4];
        o.momentum[0] = rec[5];
        o.momentum[1] = rec[6];
        o.momentum[2] = rec[7];
        o.nonfinite = (int)rec[8];
    }
    *n = (long)take;
    return GLBE_OK;
}

glbe_status glbe_residual(glbe_ctx* c, glbe_residual_info* out)
{
    NvtxRange range_("glbe_residual");
    if (!c || !out) return fail(GLBE_ERR_ARG, "ctx or out is NULL");
    return read_record(c, out);
}

// Builds the graph of one 10-step chunk starting at an even level that is a
// multiple of 10 with a snapshot at the previous multiple of 10:
// residual step + finalize, then nine plain steps, each honouring stop_dev.
static glbe_status build_chunk(glbe_ctx* c)
{
    if (c->chunk) return GLBE_OK;
    if (!c->cap_stream) GLBE_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
    const long t_save = c->t, snap_save = c->t_snap;
    c->t = 10;
    c->t_snap = 0;
    GLBE_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    glbe_status s = GLBE_OK;
    for (int k = 0; k < 10 && s == GLBE_OK; ++k) s = enqueue_step(c, c->cap_stream, c->stop_dev);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->t = t_save;
    c->t_snap = snap_save;
    if (s != GLBE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&c->chunk, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->chunk = nullptr;
        return cuda_fail(e, "graph instantiate");
    }
    return GLBE_OK;
}

glbe_status glbe_solve(glbe_ctx* c, double tol, long max_steps, long* steps_out, double* r_out)
{
    NvtxRange range_("glbe_solve");
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    if (!(tol > 0.0)) return fail(GLBE_ERR_ARG, "tol must be > 0");
    if (max_steps < 0) return fail(GLBE_ERR_ARG, "max_steps must be >= 0");
    const long t_end = c->t + max_steps;
    // align: level a multiple of 10 with a snapshot of the previous multiple of 10
    while (!(c->t % 10 == 0 && c->t_snap >= 0 && c->t_snap == c->t - 10) && c->t < t_end) {
        glbe_status s = enqueue_step(c, c->stream, nullptr);
        if (s != GLBE_OK) return s;
    }
    glbe_status s = build_chunk(c);
    if (s != GLBE_OK) return s;
    misc_set_kernel<<<1, 1, 0, c->stream>>>(nullptr, 0, c->stop_dev, 0, c->tol_dev, tol, nullptr, nullptr, 0);
    GLBE_CUDA(cudaGetLastError(), "solve setup");
    const long batch = 16;       // chunks between host checks
    int stop = 0;
    while (c->t + 10 <= t_end) {
        long nb = 0;
        for (; nb < batch && c->t + 10 * (nb + 1) <= t_end; ++nb)
            GLBE_CUDA(cudaGraphLaunch(c->chunk, c->stream), "graph launch");
        GLBE_CUDA(cudaStreamSynchronize(c->stream), "solve sync");
        GLBE_CUDA(cudaMemcpy(&stop, c->stop_dev, sizeof(int), cudaMemcpyDeviceToHost), "solve read");
        if (stop) {
            glbe_residual_info info;
            glbe_status rs = read_record(c, &info);
            c->t = info.t + 1;          // the residual step of level info.t completed
            c->t_snap = info.t;
            if (steps_out) *steps_out = info.t;
            if (r_out) *r_out = info.r;
            misc_set_kernel<<<1, 1, 0, c->stream>>>(nullptr, 0, c->stop_dev, 0, c->tol_dev, 0.0, nullptr, nullptr, 0);
            GLBE_CUDA(cudaGetLastError(), "solve reset");
            return rs;
        }
        c->t += 10 * nb;
        c->t_snap = c->t - 10;
    }
    // finish with plain steps if max_steps is not a multiple of 10
    while (c->t < t_end) {
        s = enqueue_step(c, c->stream, nullptr);
        if (s != GLBE_OK) return s;
    }
    glbe_residual_info info;
    s = read_record(c, &info);
    if (steps_out) *steps_out = c->t;
    if (r_out) *r_out = info.t >= 0 ? info.r : NAN;
    if (s != GLBE_OK) return s;
    if (info.t >= 0 && info.r <= tol) return GLBE_OK;
    return fail(GLBE_ERR_TIMEOUT, "residual %g > tol %g after %ld steps", info.r, tol, max_steps);
}

glbe_status glbe_fields(glbe_ctx* c, float* d_rho, float* d_u, float* d_B)
{
    NvtxRange range_("glbe_fields");
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    StepBuffers b = buffers_for(c, c->t);
    const FieldOut fo{d_rho, d_u, c->prm.induction ? d_B : nullptr};
    GLBE_CUDA(launch_step_any(c, MODE_FIELDS, b, fo, c->stream, nullptr), "fields kernel");
    return GLBE_OK;
}

glbe_status glbe_get_state(glbe_ctx* c, float* d_df, float* d_dg, float* d_FL)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    if (c->sp.cavity) return fail(GLBE_ERR_STATE, "state transfer does not take a fluid box or a moving lid");
    const int s = (int)(c->t & 1);
    const bool mhd = c->prm.induction;
    cudaError_t e;
    switch (c->prm.storage) {
    case GLBE_F32: e = launch_get_state_t<ST_F32>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    case GLBE_BF16: e = launch_get_state_t<ST_BF16>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    case GLBE_F16: e = launch_get_state_t<ST_F16>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    case GLBE_BF16_SR: e = launch_get_state_t<ST_BF16_SR>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    case GLBE_F16_SR: e = launch_get_state_t<ST_F16_SR>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    default: e = launch_get_state_t<ST_F32C>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    }
    GLBE_CUDA(e, "get_state kernel");
    return GLBE_OK;
}

glbe_status glbe_set_state(glbe_ctx* c, const float* d_df, const float* d_dg, const float* d_FL, long t)
{
    if (c && c->sp.cavity) return fail(GLBE_ERR_STATE, "state transfer does not take a fluid box or a moving lid");
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    if (t < 0) return fail(GLBE_ERR_ARG, "t must be >= 0");
    const int s = (int)(t & 1);
    const bool mhd = c->prm.induction;
    cudaError_t e;
    switch (c->prm.storage) {
    case GLBE_F32: e = launch_set_state_t<ST_F32>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    case GLBE_BF16: e = launch_set_state_t<ST_BF16>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    case GLBE_F16: e = launch_set_state_t<ST_F16>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    case GLBE_BF16_SR: e = launch_set_state_t<ST_BF16_SR>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    case GLBE_F16_SR: e = launch_set_state_t<ST_F16_SR>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    default: e = launch_set_state_t<ST_F32C>(mhd, c->sp, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL, c->stream); break;
    }
    GLBE_CUDA(e, "set_state kernel");
    // a replaced state starts a fresh residual history
    misc_set_kernel<<<1, 1, 0, c->stream>>>(c->t_dev, (long long)t + 10, c->stop_dev, 0, c->tol_dev, 0.0, c->record,
                                            c->hist_count, 1);
    GLBE_CUDA(cudaGetLastError(), "set_state reset");
    c->t = t;
    c->t_snap = -1;
    return GLBE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint / resume: the raw state (populations in the storage type, the
// lagged Lorentz force, the force field, the velocity snapshot, the residual
// record and counters) in one host buffer, so that a resumed march is bit for
// bit the uninterrupted one.
// ---------------------------------------------------------------------------
namespace {

struct CkptHeader {
    char magic[8];                 // "GLBECKP1"
    uint32_t version, header_bytes;
    int32_t nx, ny, nz, storage, induction, force_field;
    int64_t t, t_snap, t_dev;
    uint64_t N, f_bytes, g_bytes, total;
    uint64_t reserved[4];
};

size_t ckpt_total(const glbe_ctx* c)
{
    const size_t fb = 19 * c->N * storage_bytes(c->prm.storage);
    const size_t gb = c->prm.induction ? 21 * c->N * storage_bytes(c->prm.storage) : 0;
    return sizeof(CkptHeader) + fb + gb + (c->prm.induction ? 3 * c->N * sizeof(float) : 0) +
           (size_t)c->prm.force_field * c->N * sizeof(float) + snap_rows(c->prm.storage) * c->N * sizeof(float) +
           RECORD_STRIDE * sizeof(double);
}

}  // namespace

extern "C" glbe_status glbe_checkpoint_bytes(const glbe_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(GLBE_ERR_ARG, "ctx or bytes is NULL");
    *bytes = ckpt_total(c);
    return GLBE_OK;
}

extern "C" glbe_status glbe_checkpoint_save(glbe_ctx* c, void* h_buf, size_t bytes)
{
    if (!c || !h_buf) return fail(GLBE_ERR_ARG, "ctx or buffer is NULL");
    const size_t total = ckpt_total(c);
    if (bytes < total) return fail(GLBE_ERR_ARG, "checkpoint buffer of %zu bytes is smaller than %zu", bytes, total);
    GLBE_CUDA(cudaStreamSynchronize(c->stream), "checkpoint sync");
    CkptHeader h{};
    std::memcpy(h.magic, "GLBECKP1", 8);
    h.version = 1;
    h.header_bytes = sizeof(CkptHeader);
    h.nx = c->prm.nx;
    h.ny = c->prm.ny;
    h.nz = c->prm.nz;
    h.storage = c->prm.storage;
    h.induction = c->prm.induction;
    h.force_field = c->prm.force_field;
    h.t = c->t;
    h.t_snap = c->t_snap;
    long long tdev = 0;
    GLBE_CUDA(cudaMemcpy(&tdev, c->t_dev, sizeof tdev, cudaMemcpyDeviceToHost), "checkpoint t");
    h.t_dev = tdev;
    unsigned seed = 0;   // stochastic-rounding seed of the step from level t
    GLBE_CUDA(cudaMemcpy(&seed, c->sr_ctr + (c->t & 1), sizeof seed, cudaMemcpyDeviceToHost), "checkpoint seed");
    h.reserved[0] = seed;
    h.N = c->N;
    h.f_bytes = 19 * c->N * storage_bytes(c->prm.storage);
    h.g_bytes = c->prm.induction ? 21 * c->N * storage_bytes(c->prm.storage) : 0;
    h.total = total;
    char* o = static_cast<char*>(h_buf);
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    const int s = (int)(c->t & 1);
    GLBE_CUDA(cudaMemcpy(o, c->f[s], h.f_bytes, cudaMemcpyDeviceToHost), "checkpoint f");
    o += h.f_bytes;
    if (c->prm.induction) {
        GLBE_CUDA(cudaMemcpy(o, c->g[s], h.g_bytes, cudaMemcpyDeviceToHost), "checkpoint g");
        o += h.g_bytes;
        GLBE_CUDA(cudaMemcpy(o, c->FL, 3 * c->N * sizeof(float), cudaMemcpyDeviceToHost), "checkpoint F_L");
        o += 3 * c->N * sizeof(float);
    }
    if (c->prm.force_field) {
        const size_t fb = (size_t)c->prm.force_field * c->N * sizeof(float);
        GLBE_CUDA(cudaMemcpy(o, c->Ffield, fb, cudaMemcpyDeviceToHost), "checkpoint force");
        o += fb;
    }
    const size_t snap_bytes = snap_rows(c->prm.storage) * c->N * sizeof(float);
    GLBE_CUDA(cudaMemcpy(o, c->usnap, snap_bytes, cudaMemcpyDeviceToHost), "checkpoint snapshot");
    o += snap_bytes;
    GLBE_CUDA(cudaMemcpy(o, c->record, RECORD_STRIDE * sizeof(double), cudaMemcpyDeviceToHost), "checkpoint record");
    return GLBE_OK;
}

extern "C" glbe_status glbe_checkpoint_load(glbe_ctx* c, const void* h_buf, size_t bytes)
{
    if (!c || !h_buf) return fail(GLBE_ERR_ARG, "ctx or buffer is NULL");
    CkptHeader h;
    if (bytes < sizeof h) return fail(GLBE_ERR_ARG, "checkpoint buffer too small");
    std::memcpy(&h, h_buf, sizeof h);
    if (std::memcmp(h.magic, "GLBECKP1", 8) != 0 || h.version != 1 || h.header_bytes != sizeof h)
        return fail(GLBE_ERR_ARG, "not a checkpoint of this library version");
    if (h.nx != c->prm.nx || h.ny != c->prm.ny || h.nz != c->prm.nz || h.storage != c->prm.storage ||
        h.induction != c->prm.induction || h.force_field != c->prm.force_field)
        return fail(GLBE_ERR_ARG, "checkpoint of another grid, storage or coupling");
    if (h.total != ckpt_total(c) || bytes < h.total) return fail(GLBE_ERR_ARG, "checkpoint size mismatch");
    if (h.t < 0) return fail(GLBE_ERR_ARG, "checkpoint time level < 0");
    GLBE_CUDA(cudaStreamSynchronize(c->stream), "restore sync");
    const char* in = static_cast<const char*>(h_buf) + sizeof h;
    const int s = (int)(h.t & 1);
    GLBE_CUDA(cudaMemcpy(c->f[s], in, h.f_bytes, cudaMemcpyHostToDevice), "restore f");
    in += h.f_bytes;
    if (c->prm.induction) {
        GLBE_CUDA(cudaMemcpy(c->g[s], in, h.g_bytes, cudaMemcpyHostToDevice), "restore g");
        in += h.g_bytes;
        GLBE_CUDA(cudaMemcpy(c->FL, in, 3 * c->N * sizeof(float), cudaMemcpyHostToDevice), "restore F_L");
        in += 3 * c->N * sizeof(float);
    }
    if (c->prm.force_field) {
        const size_t fb = (size_t)c->prm.force_field * c->N * sizeof(float);
        GLBE_CUDA(cudaMemcpy(c->Ffield, in, fb, cudaMemcpyHostToDevice), "restore force");
        in += fb;
    }
    const size_t snap_bytes = snap_rows(c->prm.storage) * c->N * sizeof(float);
    GLBE_CUDA(cudaMemcpy(c->usnap, in, snap_bytes, cudaMemcpyHostToDevice), "restore snapshot");
    in += snap_bytes;
    GLBE_CUDA(cudaMemcpy(c->record, in, RECORD_STRIDE * sizeof(double), cudaMemcpyHostToDevice), "restore record");
    // residual level counter as saved; a fresh history; no pending stop
    misc_set_kernel<<<1, 1, 0, c->stream>>>(c->t_dev, (long long)h.t_dev, c->stop_dev, 0, c->tol_dev, 0.0, nullptr,
                                            nullptr, 0);
    GLBE_CUDA(cudaGetLastError(), "restore counters");
    GLBE_CUDA(cudaMemsetAsync(c->hist_count, 0, sizeof(unsigned long long), c->stream), "restore history");
    const unsigned seed = (unsigned)h.reserved[0];
    GLBE_CUDA(cudaMemcpyAsync(c->sr_ctr + (h.t & 1), &seed, sizeof seed, cudaMemcpyHostToDevice, c->stream),
              "restore seed");
    GLBE_CUDA(cudaStreamSynchronize(c->stream), "restore sync");
    c->t = (long)h.t;
    c->t_snap = (long)h.t_snap;
    return GLBE_OK;
}

// ---------------------------------------------------------------------------
// Halo of the slab decomposition along z
// ---------------------------------------------------------------------------
namespace {

constexpr int HALO_MAX_ROWS = 16;   // (5 + 3) rows, twice for the compensated low parts

// Rows of one face: row i copies P elements of esz[i] bytes from src[i] to dst[i].
struct HaloRows {
    const char* src[HALO_MAX_ROWS];
    char* dst[HALO_MAX_ROWS];
    int esz[HALO_MAX_ROWS];
    int n;
};

__global__ void halo_copy_kernel(const HaloRows rows, size_t P)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    for (int r = 0; r < rows.n; ++r) {
        if (rows.esz[r] == 4)
            reinterpret_cast<uint32_t*>(rows.dst[r])[i] = reinterpret_cast<const uint32_t*>(rows.src[r])[i];
        else
            reinterpret_cast<uint16_t*>(rows.dst[r])[i] = reinterpret_cast<const uint16_t*>(rows.src[r])[i];
    }
}

// D3Q19 directions with e_z = +1 and -1 (the ordering of include/glbe.h:
// 5 = (0,0,1), 11 = (1,0,1), 12 = (-1,0,1), 15 = (0,1,1), 16 = (0,-1,1); their
// opposites); D3Q7: 5 (+z) and 6 (-z).
const int EZ_PLUS[5] = {5, 11, 12, 15, 16};
const int EZ_MINUS[5] = {6, 13, 14, 17, 18};

size_t halo_bytes_of(const glbe_ctx* c)
{
    const size_t P = (size_t)c->prm.nx * c->prm.ny;
    const size_t rows = 5 + (c->prm.induction ? 3 : 0);
    size_t b = rows * P * (c->prm.storage == GLBE_F32C ? 4 : storage_bytes(c->prm.storage));
    if (c->prm.storage == GLBE_F32C) b += rows * P * 2;
    return b;
}

// Row table between plane z of the current population buffers and a packed
// buffer: directions `dirs` (e_z = +1 or -1) and, with induction, the D3Q7
// direction of the same sign of each component.  to_buf: plane -> buffer.
HaloRows halo_rows(glbe_ctx* c, int z, bool up, char* buf, bool to_buf)
{
    HaloRows r{};
    const size_t N = c->N, P = (size_t)c->prm.nx * c->prm.ny, plane = (size_t)z * P;
    const int s = (int)(c->t & 1);
    const bool comp = c->prm.storage == GLBE_F32C;
    const size_t es = comp ? 4 : storage_bytes(c->prm.storage);
    const int* dirs = up ? EZ_PLUS : EZ_MINUS;
    const int a7 = up ? 5 : 6;
    char* f = static_cast<char*>(c->f[s]);
    char* g = c->prm.induction ? static_cast<char*>(c->g[s]) : nullptr;
    size_t off = 0;
    auto add = [&](char* base, size_t row_elem, size_t esz) {
        char* pl = base + (row_elem + plane) * esz;
        char* bf = buf + off;
        r.src[r.n] = to_buf ? pl : bf;
        r.dst[r.n] = to_buf ? bf : pl;
        r.esz[r.n] = (int)esz;
        ++r.n;
        off += P * esz;
    };
    for (int k = 0; k < 5; ++k) add(f, (size_t)dirs[k] * N, es);
    if (g)
        for (int j = 0; j < 3; ++j) add(g, (size_t)(j * 7 + a7) * N, es);
    if (comp) {   // low parts: FP16 rows after the 19N (21N) high parts
        char* fl = f + 19 * N * 4;
        for (int k = 0; k < 5; ++k) add(fl, (size_t)dirs[k] * N, 2);
        if (g) {
            char* gl = g + 21 * N * 4;
            for (int j = 0; j < 3; ++j) add(gl, (size_t)(j * 7 + a7) * N, 2);
        }
    }
    return r;
}

glbe_status halo_launch(glbe_ctx* c, const HaloRows& r)
{
    const size_t P = (size_t)c->prm.nx * c->prm.ny;
    const unsigned grid = (unsigned)((P + 255) / 256);
    halo_copy_kernel<<<grid, 256, 0, c->stream>>>(r, P);
    GLBE_CUDA(cudaGetLastError(), "halo copy");
    return GLBE_OK;
}

}  // namespace

extern "C" glbe_status glbe_halo_bytes(const glbe_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(GLBE_ERR_ARG, "ctx or bytes is NULL");
    *bytes = halo_bytes_of(c);
    return GLBE_OK;
}

extern "C" glbe_status glbe_halo_pack(glbe_ctx* c, int face, void* d_buf)
{
    if (!c || !d_buf) return fail(GLBE_ERR_ARG, "ctx or buffer is NULL");
    if (face != 0 && face != 1) return fail(GLBE_ERR_ARG, "face must be 0 (low z) or 1 (high z)");
    if (!(face ? c->prm.ghost_hi : c->prm.ghost_lo)) return fail(GLBE_ERR_STATE, "face %d has no ghost plane", face);
    // face 1: e_z = +1 populations of the top computed plane; face 0: e_z = -1 of the bottom one
    const int z = face ? c->prm.nz - 2 : 1;
    return halo_launch(c, halo_rows(c, z, face == 1, static_cast<char*>(d_buf), true));
}

extern "C" glbe_status glbe_halo_unpack(glbe_ctx* c, int face, const void* d_buf)
{
    if (!c || !d_buf) return fail(GLBE_ERR_ARG, "ctx or buffer is NULL");
    if (face != 0 && face != 1) return fail(GLBE_ERR_ARG, "face must be 0 (low z) or 1 (high z)");
    if (!(face ? c->prm.ghost_hi : c->prm.ghost_lo)) return fail(GLBE_ERR_STATE, "face %d has no ghost plane", face);
    // the low ghost plane receives what streams upward (e_z = +1), the high one what streams down
    const int z = face ? c->prm.nz - 1 : 0;
    return halo_launch(c, halo_rows(c, z, face == 0, const_cast<char*>(static_cast<const char*>(d_buf)), false));
}

extern "C" glbe_status glbe_residual_combine(const glbe_residual_info* parts, int n, glbe_residual_info* out)
{
    if (!parts || !out || n < 1) return fail(GLBE_ERR_ARG, "parts, out or n");
    glbe_residual_info o{};
    o.t = parts[0].t;
    for (int i = 0; i < n; ++i) {
        if (parts[i].t != o.t) return fail(GLBE_ERR_ARG, "records of levels %ld and %ld", o.t, parts[i].t);
        o.num += parts[i].num;
        o.den += parts[i].den;
        o.mass += parts[i].mass;
        for (int k = 0; k < 3; ++k) o.momentum[k] += parts[i].momentum[k];
        o.nonfinite += parts[i].nonfinite;
    }
    o.r = o.den > 0.0 ? std::sqrt(o.num / o.den) : (o.num > 0.0 ? INFINITY : 0.0);
    *out = o;
    return GLBE_OK;
}

extern "C" {

glbe_status glbe_time(const glbe_ctx* c, long* t)
{
    if (!c || !t) return fail(GLBE_ERR_ARG, "ctx or t is NULL");
    *t = c->t;
    return GLBE_OK;
}

}  // extern "C"
