// glbe_internal.h -- structures shared by the host side of the C-ABI
// (glbe_api.cu) and the kernel translation units (glbe_step_*.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "glbe.h"

namespace glbe {

// Unsigned division by a run-time constant d >= 1 for dividends n < 2^31:
// q = (umulhi(n, m) + n) >> s with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1 (Granlund & Montgomery, PLDI 1994).
struct FastDiv {
    uint32_t d, m, s;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    f.s = s;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << s) - d)) / d) + 1);
    return f;
}

// Per-launch constants of the fused step (passed by value: kernel parameter
// space, uniform across the grid).
struct StepParams {
    int nx, ny, nz;
    uint32_t N;
    FastDiv div_nx, div_nxy;
    int wlo[3], whi[3];
    int glo_z, ghi_z;     // ghost planes at z = 0 / z = nz - 1 (slab decomposition): not collided,
                          // gathered from as fluid
    int cavity;           // 1: box and / or lid (the cavity kernel)
    int box;              // the flow lattice is fluid only inside [blo, bhi]
    int blo[3], bhi[3];
    int top_z;            // highest fluid z plane of the flow lattice
    float lid_corr[19];   // 6 w_a rho0 (e_a . U_lid): added to a link bounced above top_z
    float rho0;
    float inv_gamma;      // 1/gamma
    float inv_gamma2;     // 1/gamma^2
    float s[19];          // Lambda* diagonal
    // relaxation folded per moment row k (host, FP64 -> FP32): the collision
    // change of row k is rl_a[k] n_k + rl_b[k] R_k (see flow_collide)
    float rl_a[19];       // -s_k / |row_k|^2
    float rl_b[19];       // (1 - s_k/2) P_S,k c_k / |row_k|^2
    float rl_cons;        // 1 / (10 gamma): rows 3, 5, 7
    float rl_c[19];       // (1 - s_k) / |row_k|^2 = rl_a[k] + 1/|row_k|^2: row k of the
                          // post-collision moments over |row_k|^2 (16-bit storage forms)
    float F[3];           // uniform force
    int force_ncomp;      // 0, 1 (F_x field), 3
    // D3Q7 vector lattice
    float conv_coef;      // chi / gamma_m
    float omega_m;        // 1 / tau_m*
    float J_coef;         // -1 / (mu chi tau_m* theta_m)
    float B0[3];
    float bwall_dev[3];   // B_wall - B0 (0: insulating walls at the applied field)
    // storage of deviations
    float scale, inv_scale;
    int variant;          // 0 automatic, 1 one node per thread, 2 two nodes per thread, 3 TMA-staged tiles
    int collision;        // 0 MRT-GLBE; 1 preconditioned SRT-LBE; 2 SRT with the naive source
    int storage;          // Storage of the buffers (for the automatic choice)
    // interior nodes (no solid node among the 18 neighbours, no periodic wrap
    // on y and z; on an x axis without walls every x, the sources across the
    // x seam corrected by -+nx): x - ilo[0] <= ispan[0] (unsigned) and
    // likewise y, z; interior_ok = 0 if none
    int interior_ok;
    uint32_t ilo[3], ispan[3];
    long long doff[19];   // a N - (e_ax + e_ay nx + e_az nx ny): offset of the source of direction a
    long long toff[19];   // o N + (e_ox + e_oy nx + e_oz nx ny): offset of the slot o the post-collision
                          // population o of a node streams into (the transposed pull of the adjoint)
};

// Buffers of one launch.  Populations are deviations in the storage type,
// layout [a][N] (f) and [j*7 + a][N] (g).
struct StepBuffers {
    const void* fsrc;
    void* fdst;
    const void* gsrc;
    void* gdst;
    float* FL;            // [3][N] Lorentz force of the previous step (in place)
    const float* Ffield;  // [force_ncomp][N] or null
    float* usnap;         // [3][N] velocity snapshot of the last residual level; with snap_lo
                          // [6][N], rows 3..5 the low parts of u (double-float snapshot)
    double* partials;     // [8][gridDim.x] per-block residual sums
    int have_snap;        // 1: usnap holds u(t-10)
    int snap_lo;          // 1: usnap is [6][N] (FP32 and compensated storage)
    const int* stop;      // null, or a device flag: when set the launch does nothing
    // Per-direction addresses of the population buffers, filled by the
    // launcher from fsrc, fdst and StepParams::doff (kernels launched
    // otherwise do not read them): fsrc_dir[a] = fsrc + doff[a] (the
    // interior source of direction a of node n is fsrc_dir[a] + n) and
    // fdst_dir[a] = fdst + a N (slot a of node n is fdst_dir[a] + n), in
    // elements of the storage type (F32C: its high parts).
    const void* fsrc_dir[19];
    void* fdst_dir[19];
    // L2 prefetch distance in blocks, filled by the launcher (0: none): a
    // flow-step block prefetches the f rows and the force row that the block
    // pf_ahead positions later will gather -- one resident wave of the
    // launched kernel ahead
    long long pf_ahead;
    // Stochastic rounding (storage forms BF16_SR, F16_SR): the step's seed is
    // sr_ctr[sr_par] (a device counter pair; the step writes the next step's
    // seed, sr_ctr[sr_par ^ 1] = seed + 1, which no block of this step
    // reads), or sr_seed when sr_ctr is null.
    unsigned* sr_ctr;
    int sr_par;
    unsigned sr_seed;
};

// Storage forms of the population deviations.  The _SR forms store BF16 /
// FP16 like ST_BF16 / ST_F16 but round each stored value stochastically.
enum Storage { ST_F32 = 0, ST_BF16 = 1, ST_F16 = 2, ST_F32C = 3, ST_BF16_SR = 4, ST_F16_SR = 5 };
// The layout (and load path) a storage form shares
constexpr int base_storage(int st) { return st == ST_BF16_SR ? ST_BF16 : (st == ST_F16_SR ? ST_F16 : st); }
enum Mode { MODE_STEP = 0, MODE_STEP_RESID = 1, MODE_FIELDS = 2 };

constexpr int STEP_THREADS = 256;   // scalar kernel: one node per thread
constexpr int PAIR_THREADS = 128;   // paired kernel: two nodes per thread (the same 256 nodes per block)
constexpr int PARTIAL_STRIDE = 8;   // per block: num, den, sum drho, Mx, My, Mz, nonfinite, and a row the
                                    // finalize uses for its first-stage sums; stored [k][block]

// Outputs of MODE_FIELDS.
struct FieldOut {
    float* rho;
    float* u;
    float* B;
};

// Launchers, explicitly instantiated per storage type in glbe_step_<storage>.cu.
// Launches the fused step over the whole grid -- the paired kernel on
// x-periodic grids with an even nx (except for MODE_FIELDS), else the scalar
// one -- and reports the number of blocks (= residual partials) in *nblocks.
template <int ST>
cudaError_t launch_step_t(bool mhd, int mode, const StepParams& p, const StepBuffers& b, const FieldOut& fo,
                          cudaStream_t st, unsigned* nblocks);
template <int ST>
cudaError_t launch_get_state_t(bool mhd, const StepParams& p, const void* fsrc, const void* gsrc, const float* FL,
                               float* df, float* dg, float* dFL, cudaStream_t st);
// 1 if a bounded wait of the TMA-staged step kernel (variant 3) ran out since
// the last call (the flag is then cleared); one flag per storage type.
template <int ST>
int tile_wait_error_t();
// Initial state of a context with a moving lid (F32, F32C and BF16 storage):
// see lid_init_kernel.
template <int ST>
cudaError_t launch_lid_init_t(const StepParams& p, void* fbuf, cudaStream_t st);
template <int ST>
cudaError_t launch_set_state_t(bool mhd, const StepParams& p, void* fsrc, void* gsrc, float* FL, const float* df,
                               const float* dg, const float* dFL, cudaStream_t st);

// Reduces the per-block partials of a residual step in a fixed order into
// record[0..8] = (t, r, num, den, mass, Mx, My, Mz, nonfinite), with t read
// from *t_dev and then advanced by 10, mass = mass0 + sum drho, and appends
// the record to the history ring hist[(count % cap) * RECORD_STRIDE].
constexpr int RECORD_STRIDE = 16;
// The reduction also raises *stop when r <= *tol (tol > 0) or a velocity is
// non-finite, and does nothing once *stop is set.
cudaError_t launch_finalize(const double* partials, unsigned nblocks, double mass0, long long* t_dev,
                            double* record, double* hist, unsigned long long* hist_count, unsigned hist_cap,
                            int* stop, const double* tol, cudaStream_t st);

// Host helpers shared by the C-ABI translation units (glbe_api.cu).
glbe_status fail(glbe_status s, const char* fmt, ...);       // sets the thread-local message
glbe_status validate_params(const glbe_params* p);
// Fluid nodes of a grid: planes on walls and ghost planes excluded.
inline long long fluid_nodes(const glbe_params* p)
{
    const int n[3] = {p->nx, p->ny, p->nz};
    long long count = 1;
    for (int d = 0; d < 3; ++d) {
        int lo = p->wall_lo[d], hi = n[d] - 1 - p->wall_hi[d];
        if (d == 2) {
            lo += p->ghost_lo;
            hi -= p->ghost_hi;
        }
        if (p->box) {
            lo = lo > p->box_lo[d] ? lo : p->box_lo[d];
            hi = hi < p->box_hi[d] ? hi : p->box_hi[d];
        }
        count *= hi >= lo ? hi - lo + 1 : 0;
    }
    return count;
}
StepParams make_step_params(const glbe_params* p);

// What another translation unit (the adjoint) needs of a context: its
// parameters and the buffers of the current time level t (the populations the
// next step gathers from, the lagged Lorentz force, the force field).
struct CtxView {
    glbe_params prm;
    StepParams sp;
    size_t N;
    long t;
    void* fsrc;           // population deviations entering the step from t (storage type)
    void* gsrc;           // null without induction
    float* FL;            // [3][N] Lorentz force of the step that led to t (null without induction)
    const float* Ffield;  // [force_field][N] or null
    size_t f_bytes;       // bytes of one f buffer (19N values, F32C: plus the 19N low parts)
    size_t g_bytes;       // bytes of one g buffer (0 without induction)
    cudaStream_t stream;
};
glbe_status ctx_view(glbe_ctx* c, CtxView* v);

// NVTX range around a C-ABI call (visible in Nsight tools; header-only NVTX 3,
// a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
size_t storage_value_bytes(int storage);   // bytes per population value (F32C: 4 + 2)

}  // namespace glbe
