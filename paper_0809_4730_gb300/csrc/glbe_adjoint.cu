// glbe_adjoint.cu -- gradient of a velocity objective with respect to the
// body-force field: the transposed (adjoint) collide-stream step, the steady
// adjoint fixed point and the checkpointed reverse sweep of an unrolled march.
//
// The paper (arXiv:0809.4730) has no adjoint.  What is differentiated is its
// time step: the state s_t per node (pre-collision f, g and the lagged Lorentz
// force) evolves as s_{t+1} = P Y(s_t, F), Y the node update of Secs. 2-4
// (glbe_kernels.cuh), P the streaming of Eqs. pstreaming/mstreaming with
// bounce-back (f) and anti-bounce-back (g).  The objective is
// Q = sum_x w(x) . u(x) with u = j/rho (Eq. precondhydrofields).
//
// One adjoint step at level t takes the cotangent lam_{t+1} of the next
// state and forms, per fluid node x (one thread, no atomics):
//   v(x)  = (P^t lam_{t+1})(x): the pull of the forward step run backwards,
//           v_o(x) = lam_{t+1,o}(x - e_a) for the link a = opp(o) of the
//           forward gather, or lam_{t+1,a}(x) where that link was bounced
//           (with a minus sign for g, whose wall reflection is negated);
//   lam_t(x) = Y_s(x)^t v(x) + U_s(x)^t w(x),  dQ/dF(x) += Y_F^t v + U_F^t w
// (node_reverse in glbe_adjoint.cuh).  The steady adjoint iterates this map
// at the fixed point s*: its spectrum is the one of the forward step, so the
// gamma preconditioning accelerates it the same way.  Its convergence is
// measured on the gradient field itself,
// r = ||dQdF_k - dQdF_{k-10}|| / ||dQdF_k||, every 10 iterations.  The map is
// linear in lam with coefficients from 16 forward quantities per node
// (NodeLin: 1/rho, j, F, B, u0, J), and s* does not change: the steady
// adjoint writes them once and every iteration reads them in place of the
// gathered state; the unrolled sweep, whose state changes every level,
// gathers it.
#include <cstring>

#include "glbe.h"
#include "glbe_internal.h"
#include "glbe_adjoint.cuh"

using namespace glbe;

// The forward steps are instantiated in glbe_step_f32.cu / glbe_step_f32c.cu.
namespace glbe {
extern template cudaError_t launch_step_t<ST_F32>(bool, int, const StepParams&, const StepBuffers&, const FieldOut&,
                                                  cudaStream_t, unsigned*);
extern template cudaError_t launch_step_t<ST_F32C>(bool, int, const StepParams&, const StepBuffers&,
                                                   const FieldOut&, cudaStream_t, unsigned*);
}  // namespace glbe

namespace {

constexpr size_t ALIGN = 256;
constexpr unsigned HIST_CAP = 64;
// One node per thread; 128-thread blocks held to 128 registers (4 resident
// blocks per SM; the reverse step needs ~160 registers unconstrained, which
// leaves one 256-thread block per SM).
constexpr int ADJ_THREADS = 128;
size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Buffers of one adjoint step.
struct AdjArgs {
    // forward state at level t (the gather of the forward step)
    const void* fsrc;
    const void* gsrc;
    const float* FL;          // [3][N] lagged Lorentz force at level t
    const float* Ffield;      // [force_ncomp][N] or null
    // linearisation rows of the same state ([LIN_ROWS][N], NodeLin order);
    // read by the LIN launches in place of fsrc, gsrc, FL and Ffield
    const float* lin;
    // cotangents: in = level t+1, out = level t; [19][N] f, [21][N] g, [3][N] F_L
    const float* lam_in;
    float* lam_out;
    // objective weights applied at this level (objective = 0: none)
    int objective;
    const float* w;           // [3][N] or null: then w_uniform on fluid nodes
    float w_uniform[3];
    float* dQdF;              // [3][N]
    int accumulate;           // 1: dQdF += ..., 0: dQdF = ...
    // convergence of the steady iteration (RESID launches)
    float* dsnap;             // [3][N] gradient of the previous evaluation
    double* partials;         // [8][blocks]
    int have_snap;
    const int* stop;          // null or a device flag: when set the launch does nothing
};

// One adjoint step.  LIN: the linearisation point comes from a.lin (the
// steady adjoint, whose state is fixed); else from the forward gather of the
// state at fsrc/gsrc/FL.
template <int ST, bool MHD, bool RESID, bool LIN>
__global__ void __launch_bounds__(ADJ_THREADS, 4) adjoint_kernel(const StepParams p, const AdjArgs a)
{
    using S = Store<ST>;
    using T = typename S::T;
    if (a.stop != nullptr && *a.stop) return;
    const uint32_t i = blockIdx.x * ADJ_THREADS + threadIdx.x;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const size_t N = p.N;
    const bool inb = i < p.N;
    const uint32_t n = inb ? i : 0u;
    const float* __restrict__ lf = a.lam_in;
    const float* __restrict__ lg = a.lam_in + 19 * N;
    const float* __restrict__ lk = a.lam_in + 40 * N;
    float* __restrict__ of = a.lam_out;
    float* __restrict__ og = a.lam_out + 19 * N;
    float* __restrict__ ok = a.lam_out + 40 * N;
    // linearisation point (the forward gather of level t: d, q) and
    // v = P^t lam_{t+1} (vf, vg): the forward pull of slot a from (src, a),
    // or from the node's own opposite slot o when bounced, read backwards
    float d[19], dl[19], q[21], ql[21], vf[19], vg[21];
    // compensated storage: the node update is linearised at high + low part
    const auto fold_lo = [](auto& v, const auto& lo) {
        if constexpr (S::COMP) {
#pragma unroll
            for (int k = 0; k < (int)(sizeof(v) / sizeof(v[0])); ++k) v[k] += lo[k];
        }
    };
    bool fluid = inb;
    int wp = 0, wm = 0;
    if (inb && is_interior(p, n, wp, wm)) {
        // every link is a plain one: slot o of the node x + e_o at the fixed
        // offset toff[o] (x-seam targets corrected like the sources of opp(o))
        if (!LIN) {
            load_f_interior<ST>(p, static_cast<const T*>(a.fsrc), n, wp, wm, d, dl);
            fold_lo(d, dl);
            if (MHD) {
                load_g_interior<ST>(p, static_cast<const T*>(a.gsrc), n, wp, wm, q, ql);
                fold_lo(q, ql);
            }
        }
        const float* __restrict__ l0 = lf + n;
#pragma unroll
        for (int o = 0; o < 19; ++o) vf[o] = *(seam_src(dir_opp(o), l0, l0 + wp, l0 + wm) + p.toff[o]);
        if (MHD) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float* __restrict__ b0 = lg + (size_t)(j * 7) * N + n;
#pragma unroll
                for (int o = 0; o < 7; ++o) vg[j * 7 + o] = *(seam_src(dir_opp(o), b0, b0 + wp, b0 + wm) + p.toff[o]);
            }
        }
    } else {
        const Geo g = make_geo(p, n);
        fluid = inb && !g.solid;
        if (fluid) {
            if (!LIN) {
                load_f<ST>(p, static_cast<const T*>(a.fsrc), g, d, dl);
                fold_lo(d, dl);
                if (MHD) {
                    load_g<ST>(p, static_cast<const T*>(a.gsrc), g, q, ql);
                    fold_lo(q, ql);
                }
            }
            vf[0] = lf[n];
#define GLBE_ADJF(a_, o_, src, sol) vf[o_] = (sol) ? lf[(size_t)(a_) * N + n] : lf[(size_t)(o_) * N + (src)];
            GLBE_DIRS(GLBE_ADJF)
#undef GLBE_ADJF
            if (MHD) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float* __restrict__ b = lg + (size_t)(j * 7) * N;
                    vg[j * 7] = b[n];
#define GLBE_ADJG(a_, o_, src, sol) \
    vg[j * 7 + o_] = (sol) ? -b[(size_t)(a_) * N + n] : b[(size_t)(o_) * N + (src)];
                    GLBE_DIRS7(GLBE_ADJG)
#undef GLBE_ADJG
                }
            }
        }
    }
    if (!fluid) {
        if (inb) {
            for (int k = 0; k < 19; ++k) of[(size_t)k * N + n] = 0.f;
            if (MHD) {
                for (int k = 0; k < 21; ++k) og[(size_t)k * N + n] = 0.f;
                for (int k = 0; k < 3; ++k) ok[(size_t)k * N + n] = 0.f;
            }
            if (!a.accumulate)
                for (int k = 0; k < 3; ++k) a.dQdF[(size_t)k * N + n] = 0.f;
            if (RESID)
                for (int k = 0; k < 3; ++k) a.dsnap[(size_t)k * N + n] = 0.f;
        }
    } else {
        NodeLin lp;
        if (LIN) {
            const float* __restrict__ ln = a.lin + n;
            lp.ri = ln[0];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lp.j[c] = ln[(size_t)(1 + c) * N];
                lp.F[c] = ln[(size_t)(4 + c) * N];
                lp.B[c] = MHD ? ln[(size_t)(7 + c) * N] : 0.f;
                lp.u0[c] = MHD ? ln[(size_t)(10 + c) * N] : 0.f;
                lp.Jv[c] = MHD ? ln[(size_t)(13 + c) * N] : 0.f;
            }
        } else {
            float FLp[3] = {0.f, 0.f, 0.f};
            if (MHD) {
                FLp[0] = a.FL[n];
                FLp[1] = a.FL[N + n];
                FLp[2] = a.FL[2 * N + n];
            } else {
#pragma unroll
                for (int k = 0; k < 21; ++k) q[k] = 0.f;
            }
            float Fext[3] = {p.F[0], p.F[1], p.F[2]};
            if (p.force_ncomp >= 1) Fext[0] += __ldg(a.Ffield + n);
            if (p.force_ncomp == 3) {
                Fext[1] += __ldg(a.Ffield + N + n);
                Fext[2] += __ldg(a.Ffield + 2 * N + n);
            }
            lp = node_linearise<MHD>(p, d, q, FLp, Fext);
        }
        float vFL[3] = {0.f, 0.f, 0.f};
        if (MHD) {
            vFL[0] = lk[n];
            vFL[1] = lk[N + n];
            vFL[2] = lk[2 * N + n];
        } else {
#pragma unroll
            for (int k = 0; k < 21; ++k) vg[k] = 0.f;
        }
        float wu[3] = {0.f, 0.f, 0.f};
        if (a.objective) {
            if (a.w) {
                wu[0] = a.w[n];
                wu[1] = a.w[N + n];
                wu[2] = a.w[2 * N + n];
            } else {
                wu[0] = a.w_uniform[0];
                wu[1] = a.w_uniform[1];
                wu[2] = a.w_uniform[2];
            }
        }
        // values this thread reads back are loaded before any store (a load
        // after the stores waits for their completion)
        float acc_in[3] = {0.f, 0.f, 0.f}, snap[3] = {0.f, 0.f, 0.f};
        if (a.accumulate)
            for (int k = 0; k < 3; ++k) acc_in[k] = a.dQdF[(size_t)k * N + n];
        if (RESID && a.have_snap)
            for (int k = 0; k < 3; ++k) snap[k] = a.dsnap[(size_t)k * N + n];
        NodeAdjoint r;
        node_reverse_at<MHD>(p, lp, vf, vg, vFL, wu, r);
#pragma unroll
        for (int k = 0; k < 19; ++k) of[(size_t)k * N + n] = r.d[k];
        if (MHD) {
#pragma unroll
            for (int k = 0; k < 21; ++k) og[(size_t)k * N + n] = r.q[k];
            for (int k = 0; k < 3; ++k) ok[(size_t)k * N + n] = r.FLp[k];
        }
        for (int k = 0; k < 3; ++k) a.dQdF[(size_t)k * N + n] = a.accumulate ? acc_in[k] + r.F[k] : r.F[k];
        if (RESID) {
            if (a.have_snap) {
                const float e0 = r.F[0] - snap[0], e1 = r.F[1] - snap[1], e2 = r.F[2] - snap[2];
                acc[0] = e0 * e0 + e1 * e1 + e2 * e2;
            }
            acc[1] = r.F[0] * r.F[0] + r.F[1] * r.F[1] + r.F[2] * r.F[2];
            acc[6] = vnonfinite(r.F[0] + r.F[1] + r.F[2]);
            a.dsnap[n] = r.F[0];
            a.dsnap[N + n] = r.F[1];
            a.dsnap[2 * N + n] = r.F[2];
        }
    }
    if (RESID) block_partials<ADJ_THREADS>(acc, a.partials);
}

// The linearisation rows of the state at fsrc/gsrc/FL (with the force
// field): NodeLin of every fluid node, 0 on solid nodes.  One launch per
// steady adjoint solve.
template <int ST, bool MHD>
__global__ void __launch_bounds__(ADJ_THREADS) adjoint_lin_kernel(const StepParams p, const AdjArgs a, float* lin)
{
    using S = Store<ST>;
    using T = typename S::T;
    const uint32_t i = blockIdx.x * ADJ_THREADS + threadIdx.x;
    if (i >= p.N) return;
    const size_t N = p.N;
    float d[19], dl[19], q[21], ql[21];
    int wp = 0, wm = 0;
    bool fluid = true;
    if (is_interior(p, i, wp, wm)) {
        load_f_interior<ST>(p, static_cast<const T*>(a.fsrc), i, wp, wm, d, dl);
        if (MHD) load_g_interior<ST>(p, static_cast<const T*>(a.gsrc), i, wp, wm, q, ql);
    } else {
        const Geo g = make_geo(p, i);
        fluid = !g.solid;
        if (fluid) {
            load_f<ST>(p, static_cast<const T*>(a.fsrc), g, d, dl);
            if (MHD) load_g<ST>(p, static_cast<const T*>(a.gsrc), g, q, ql);
        }
    }
    constexpr int R = MHD ? LIN_ROWS_MHD : LIN_ROWS_FLOW;
    if (!fluid) {
#pragma unroll
        for (int k = 0; k < R; ++k) lin[(size_t)k * N + i] = 0.f;
        return;
    }
    if constexpr (S::COMP) {
#pragma unroll
        for (int k = 0; k < 19; ++k) d[k] += dl[k];
        if (MHD) {
#pragma unroll
            for (int k = 0; k < 21; ++k) q[k] += ql[k];
        }
    }
    float FLp[3] = {0.f, 0.f, 0.f};
    if (MHD) {
        FLp[0] = a.FL[i];
        FLp[1] = a.FL[N + i];
        FLp[2] = a.FL[2 * N + i];
    } else {
#pragma unroll
        for (int k = 0; k < 21; ++k) q[k] = 0.f;
    }
    float Fext[3] = {p.F[0], p.F[1], p.F[2]};
    if (p.force_ncomp >= 1) Fext[0] += __ldg(a.Ffield + i);
    if (p.force_ncomp == 3) {
        Fext[1] += __ldg(a.Ffield + N + i);
        Fext[2] += __ldg(a.Ffield + 2 * N + i);
    }
    const NodeLin L = node_linearise<MHD>(p, d, q, FLp, Fext);
    float* __restrict__ o = lin + i;
    o[0] = L.ri;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o[(size_t)(1 + c) * N] = L.j[c];
        o[(size_t)(4 + c) * N] = L.F[c];
        if (MHD) {
            o[(size_t)(7 + c) * N] = L.B[c];
            o[(size_t)(10 + c) * N] = L.u0[c];
            o[(size_t)(13 + c) * N] = L.Jv[c];
        }
    }
}

template <int ST, bool MHD>
cudaError_t launch_adj2(bool resid, const StepParams& p, const AdjArgs& a, cudaStream_t st, unsigned* nblocks)
{
    const unsigned grid = (unsigned)(((size_t)p.N + ADJ_THREADS - 1) / ADJ_THREADS);
    if (a.lin) {
        // no state gather: one instantiation serves both storage forms
        if (resid) adjoint_kernel<ST_F32, MHD, true, true><<<grid, ADJ_THREADS, 0, st>>>(p, a);
        else adjoint_kernel<ST_F32, MHD, false, true><<<grid, ADJ_THREADS, 0, st>>>(p, a);
    } else {
        if (resid) adjoint_kernel<ST, MHD, true, false><<<grid, ADJ_THREADS, 0, st>>>(p, a);
        else adjoint_kernel<ST, MHD, false, false><<<grid, ADJ_THREADS, 0, st>>>(p, a);
    }
    if (nblocks) *nblocks = grid;
    return cudaGetLastError();
}

template <int ST, bool MHD>
cudaError_t launch_lin2(const StepParams& p, const AdjArgs& a, float* lin, cudaStream_t st)
{
    const unsigned grid = (unsigned)(((size_t)p.N + ADJ_THREADS - 1) / ADJ_THREADS);
    adjoint_lin_kernel<ST, MHD><<<grid, ADJ_THREADS, 0, st>>>(p, a, lin);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(int storage, bool mhd, bool resid, const StepParams& p, const AdjArgs& a, cudaStream_t st,
                           unsigned* nblocks)
{
    if (storage == GLBE_F32)
        return mhd ? launch_adj2<ST_F32, true>(resid, p, a, st, nblocks)
                   : launch_adj2<ST_F32, false>(resid, p, a, st, nblocks);
    return mhd ? launch_adj2<ST_F32C, true>(resid, p, a, st, nblocks)
               : launch_adj2<ST_F32C, false>(resid, p, a, st, nblocks);
}

cudaError_t launch_linearise(int storage, bool mhd, const StepParams& p, const AdjArgs& a, float* lin, cudaStream_t st)
{
    if (storage == GLBE_F32) return mhd ? launch_lin2<ST_F32, true>(p, a, lin, st) : launch_lin2<ST_F32, false>(p, a, lin, st);
    return mhd ? launch_lin2<ST_F32C, true>(p, a, lin, st) : launch_lin2<ST_F32C, false>(p, a, lin, st);
}

__global__ void adj_misc_kernel(long long* t_dev, long long t, int* stop, double* tol, double tol_v, double* record,
                                unsigned long long* hist_count)
{
    *t_dev = t;
    *stop = 0;
    *tol = tol_v;
    for (int k = 0; k < RECORD_STRIDE; ++k) record[k] = 0.0;
    record[0] = -1.0;
    *hist_count = 0;
}

// Workspace of the adjoint calls.
struct AdjLayout {
    size_t lam[2];            // cotangent buffers: [19][N] f, [21][N] g, [3][N] F_L (g and F_L unused without induction)
    size_t dsnap, partials, record, hist, misc;
    size_t lin;               // steady form: the linearisation rows [LIN_ROWS][N]
    size_t state_bytes;       // one stored state: f buffer, g buffer, F_L
    size_t state_f, state_g, state_FL;   // offsets inside a stored state
    size_t cp;                // checkpoints
    long ncp;
    size_t seg;               // segment of recomputed states
    long nseg;
    size_t total;
};

AdjLayout adj_layout(const glbe_params* p, long nsteps, long K)
{
    AdjLayout L{};
    const size_t N = (size_t)p->nx * p->ny * p->nz;
    const size_t grid = (N + ADJ_THREADS - 1) / ADJ_THREADS;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
    L.lam[0] = take(43 * N * sizeof(float));
    L.lam[1] = take(43 * N * sizeof(float));
    L.dsnap = take(3 * N * sizeof(float));
    L.partials = take(grid * PARTIAL_STRIDE * sizeof(double));
    L.record = take(RECORD_STRIDE * sizeof(double));
    L.hist = take((size_t)HIST_CAP * RECORD_STRIDE * sizeof(double));
    L.misc = take(64);
    const size_t vb = storage_value_bytes(p->storage);
    L.state_f = 0;
    L.state_g = align_up(19 * N * vb);
    L.state_FL = L.state_g + (p->induction ? align_up(21 * N * vb) : 0);
    L.state_bytes = L.state_FL + (p->induction ? align_up(3 * N * sizeof(float)) : 0);
    if (nsteps == 0) L.lin = take((size_t)(p->induction ? LIN_ROWS_MHD : LIN_ROWS_FLOW) * N * sizeof(float));
    if (nsteps > 0) {
        L.ncp = (nsteps + K - 1) / K;
        L.nseg = K < nsteps ? K : nsteps;
        L.cp = take((size_t)L.ncp * L.state_bytes);
        L.seg = take((size_t)L.nseg * L.state_bytes);
    }
    L.total = off;
    return L;
}

glbe_status check_adjoint_args(const CtxView& v, const void* d_work, size_t bytes, const AdjLayout& L, float* d_dQdF)
{
    if (v.prm.storage != GLBE_F32 && v.prm.storage != GLBE_F32C)
        return fail(GLBE_ERR_ARG, "the adjoint needs F32 or F32C storage (FP32 state)");
    if (v.prm.ghost_lo || v.prm.ghost_hi) return fail(GLBE_ERR_ARG, "the adjoint runs on a whole grid (no ghost planes)");
    if (v.prm.collision) return fail(GLBE_ERR_ARG, "the adjoint differentiates the MRT collision");
    if (v.sp.cavity) return fail(GLBE_ERR_ARG, "the adjoint does not take a fluid box or a moving lid");
    if (!d_work) return fail(GLBE_ERR_ARG, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(d_work) % ALIGN) != 0)
        return fail(GLBE_ERR_ARG, "workspace must be %zu-byte aligned", ALIGN);
    if (bytes < L.total) return fail(GLBE_ERR_ARG, "workspace of %zu bytes is smaller than the %zu needed", bytes, L.total);
    if (!d_dQdF) return fail(GLBE_ERR_ARG, "dQdF is NULL");
    return GLBE_OK;
}

AdjArgs base_args(const CtxView& v, const float* d_w, float* d_dQdF)
{
    AdjArgs a{};
    a.Ffield = v.Ffield;
    a.w = d_w;
    const int Lx = v.prm.nx - v.prm.wall_lo[0] - v.prm.wall_hi[0];
    a.w_uniform[0] = 1.0f / (float)Lx;    // Q = (1/L_x) sum_fluid u_x
    a.w_uniform[1] = a.w_uniform[2] = 0.f;
    a.dQdF = d_dQdF;
    return a;
}

#define ADJ_CUDA(call, what)                                                                         \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return fail(GLBE_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e_), cudaGetErrorString(e_)); \
    } while (0)

// Copies the state (f, g, F_L) the step from level t gathers from into a slot.
glbe_status save_state(const CtxView& v, const AdjLayout& L, char* slot, cudaStream_t st)
{
    ADJ_CUDA(cudaMemcpyAsync(slot + L.state_f, v.fsrc, v.f_bytes, cudaMemcpyDeviceToDevice, st), "checkpoint f");
    if (v.prm.induction) {
        ADJ_CUDA(cudaMemcpyAsync(slot + L.state_g, v.gsrc, v.g_bytes, cudaMemcpyDeviceToDevice, st), "checkpoint g");
        ADJ_CUDA(cudaMemcpyAsync(slot + L.state_FL, v.FL, 3 * v.N * sizeof(float), cudaMemcpyDeviceToDevice, st),
                 "checkpoint F_L");
    }
    return GLBE_OK;
}

cudaError_t forward_step(const CtxView& v, const AdjLayout& L, const char* from, char* to, cudaStream_t st)
{
    StepBuffers b{};
    b.fsrc = from + L.state_f;
    b.fdst = to + L.state_f;
    b.gsrc = v.prm.induction ? from + L.state_g : nullptr;
    b.gdst = v.prm.induction ? to + L.state_g : nullptr;
    b.FL = v.prm.induction ? reinterpret_cast<float*>(to + L.state_FL) : nullptr;
    b.Ffield = v.Ffield;
    const FieldOut fo{nullptr, nullptr, nullptr};
    if (v.prm.induction) {
        // the step updates F_L in place: start the new slot from the old one
        cudaError_t e = cudaMemcpyAsync(to + L.state_FL, from + L.state_FL, 3 * v.N * sizeof(float),
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    if (v.prm.storage == GLBE_F32) return launch_step_t<ST_F32>(v.prm.induction, MODE_STEP, v.sp, b, fo, st, nullptr);
    return launch_step_t<ST_F32C>(v.prm.induction, MODE_STEP, v.sp, b, fo, st, nullptr);
}

void set_forward(AdjArgs& a, const CtxView& v, const AdjLayout& L, const char* slot)
{
    a.fsrc = slot + L.state_f;
    a.gsrc = v.prm.induction ? slot + L.state_g : nullptr;
    a.FL = v.prm.induction ? reinterpret_cast<const float*>(slot + L.state_FL) : nullptr;
}

}  // namespace

extern "C" {

glbe_status glbe_adjoint_workspace_bytes(const glbe_params* p, long nsteps, long K, size_t* bytes)
{
    if (!bytes) return fail(GLBE_ERR_ARG, "bytes is NULL");
    glbe_status s = validate_params(p);
    if (s != GLBE_OK) return s;
    if (nsteps < 0) return fail(GLBE_ERR_ARG, "nsteps must be >= 0");
    if (nsteps > 0 && K < 1) return fail(GLBE_ERR_ARG, "K must be >= 1");
    *bytes = adj_layout(p, nsteps, K).total;
    return GLBE_OK;
}

glbe_status glbe_adjoint_steady(glbe_ctx* ctx, const float* d_w, double tol, long max_iters, void* d_work,
                                size_t bytes, float* d_dQdF, long* iters_out, double* r_out)
{
    NvtxRange range_("glbe_adjoint_steady");
    CtxView v;
    glbe_status s = ctx_view(ctx, &v);
    if (s != GLBE_OK) return s;
    if (!(tol > 0.0)) return fail(GLBE_ERR_ARG, "tol must be > 0");
    if (max_iters < 10) return fail(GLBE_ERR_ARG, "max_iters must be >= 10");
    const AdjLayout L = adj_layout(&v.prm, 0, 1);
    s = check_adjoint_args(v, d_work, bytes, L, d_dQdF);
    if (s != GLBE_OK) return s;
    char* ws = static_cast<char*>(d_work);
    float* lam[2] = {reinterpret_cast<float*>(ws + L.lam[0]), reinterpret_cast<float*>(ws + L.lam[1])};
    double* partials = reinterpret_cast<double*>(ws + L.partials);
    double* record = reinterpret_cast<double*>(ws + L.record);
    double* hist = reinterpret_cast<double*>(ws + L.hist);
    char* misc = ws + L.misc;
    auto* hist_count = reinterpret_cast<unsigned long long*>(misc);
    auto* t_dev = reinterpret_cast<long long*>(misc + 8);
    auto* tol_dev = reinterpret_cast<double*>(misc + 16);
    auto* stop = reinterpret_cast<int*>(misc + 24);
    const cudaStream_t st = v.stream;
    const size_t N = v.N;

    AdjArgs a = base_args(v, d_w, d_dQdF);
    a.fsrc = v.fsrc;
    a.gsrc = v.gsrc;
    a.FL = v.FL;
    a.objective = 1;
    a.accumulate = 0;
    a.dsnap = reinterpret_cast<float*>(ws + L.dsnap);
    a.partials = partials;
    // the state is fixed: its linearisation rows once, then every iteration
    // reads them in place of the state
    float* lin = reinterpret_cast<float*>(ws + L.lin);
    ADJ_CUDA(launch_linearise(v.prm.storage, v.prm.induction, v.sp, a, lin, st), "adjoint linearisation");
    a.lin = lin;
    ADJ_CUDA(cudaMemsetAsync(lam[0], 0, 43 * N * sizeof(float), st), "adjoint init");
    adj_misc_kernel<<<1, 1, 0, st>>>(t_dev, 10, stop, tol_dev, tol, record, hist_count);
    ADJ_CUDA(cudaGetLastError(), "adjoint init");
    const double zero_mass = 0.0;
    // iterations 0..9 directly: the first residual launch only takes the snapshot
    for (int k = 0; k < 10; ++k) {
        a.lam_in = lam[k & 1];
        a.lam_out = lam[(k + 1) & 1];
        a.have_snap = 0;
        ADJ_CUDA(launch_adjoint(v.prm.storage, v.prm.induction, k == 0, v.sp, a, st, nullptr), "adjoint step");
    }
    // chunks of 10 iterations (residual + finalize, nine plain) replayed from a graph
    cudaStream_t cap = nullptr;
    ADJ_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        a.stop = stop;
        for (int k = 0; k < 10 && e == cudaSuccess; ++k) {
            a.lam_in = lam[k & 1];
            a.lam_out = lam[(k + 1) & 1];
            a.have_snap = 1;
            unsigned nb = 0;
            e = launch_adjoint(v.prm.storage, v.prm.induction, k == 0, v.sp, a, cap, &nb);
            if (e == cudaSuccess && k == 0)
                e = launch_finalize(partials, nb, zero_mass, t_dev, record, hist, hist_count, HIST_CAP, stop, tol_dev,
                                    cap);
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        return fail(GLBE_ERR_CUDA, "adjoint chunk graph: %s", cudaGetErrorString(e));
    }
    long it = 10;
    int stopped = 0;
    glbe_status out = GLBE_OK;
    while (it + 10 <= max_iters) {
        long nb = 0;
        for (; nb < 16 && it + 10 * (nb + 1) <= max_iters; ++nb) {
            e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) break;
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaMemcpy(&stopped, stop, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        it += 10 * nb;
        if (stopped) break;
    }
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) return fail(GLBE_ERR_CUDA, "adjoint iteration: %s", cudaGetErrorString(e));
    double rec[RECORD_STRIDE];
    ADJ_CUDA(cudaMemcpy(rec, record, sizeof rec, cudaMemcpyDeviceToHost), "adjoint record");
    if (iters_out) *iters_out = (long)rec[0];
    if (r_out) *r_out = rec[1];
    if (rec[8] > 0.0 || !(rec[1] == rec[1])) return fail(GLBE_ERR_DIVERGED, "non-finite adjoint gradient");
    if (!stopped) {
        out = fail(GLBE_ERR_TIMEOUT, "adjoint residual %g > tol %g after %ld iterations", rec[1], tol, max_iters);
    }
    return out;
}

glbe_status glbe_adjoint_unrolled(glbe_ctx* ctx, const float* d_w, long nsteps, long K, void* d_work, size_t bytes,
                                  float* d_dQdF)
{
    NvtxRange range_("glbe_adjoint_unrolled");
    CtxView v;
    glbe_status s = ctx_view(ctx, &v);
    if (s != GLBE_OK) return s;
    if (nsteps < 1) return fail(GLBE_ERR_ARG, "nsteps must be >= 1");
    if (K < 1) return fail(GLBE_ERR_ARG, "K must be >= 1");
    const AdjLayout L = adj_layout(&v.prm, nsteps, K);
    s = check_adjoint_args(v, d_work, bytes, L, d_dQdF);
    if (s != GLBE_OK) return s;
    char* ws = static_cast<char*>(d_work);
    float* lam[2] = {reinterpret_cast<float*>(ws + L.lam[0]), reinterpret_cast<float*>(ws + L.lam[1])};
    char* cp = ws + L.cp;
    char* seg = ws + L.seg;
    const cudaStream_t st = v.stream;
    const size_t N = v.N;

    // forward march of the context with a checkpoint every K levels
    for (long i = 0; i < L.ncp; ++i) {
        s = ctx_view(ctx, &v);
        if (s != GLBE_OK) return s;
        s = save_state(v, L, cp + (size_t)i * L.state_bytes, st);
        if (s != GLBE_OK) return s;
        const long n = (i + 1) * K <= nsteps ? K : nsteps - i * K;
        s = glbe_step_n(ctx, n);
        if (s != GLBE_OK) return s;
    }
    s = ctx_view(ctx, &v);
    if (s != GLBE_OK) return s;

    // objective on the final level T: lam_T = U_s^t w, dQdF = U_F^t w
    AdjArgs a = base_args(v, d_w, d_dQdF);
    ADJ_CUDA(cudaMemsetAsync(lam[0], 0, 43 * N * sizeof(float), st), "adjoint init");
    ADJ_CUDA(cudaMemsetAsync(d_dQdF, 0, 3 * N * sizeof(float), st), "adjoint init");
    a.fsrc = v.fsrc;
    a.gsrc = v.gsrc;
    a.FL = v.FL;
    a.objective = 1;
    a.accumulate = 1;
    a.lam_in = lam[0];
    a.lam_out = lam[1];
    ADJ_CUDA(launch_adjoint(v.prm.storage, v.prm.induction, false, v.sp, a, st, nullptr), "adjoint objective");
    int cur = 1;
    a.objective = 0;
    // reverse sweep, one segment of up to K levels at a time
    for (long i = L.ncp - 1; i >= 0; --i) {
        const long len = (i + 1) * K <= nsteps ? K : nsteps - i * K;
        ADJ_CUDA(cudaMemcpyAsync(seg, cp + (size_t)i * L.state_bytes, L.state_bytes, cudaMemcpyDeviceToDevice, st),
                 "restore checkpoint");
        for (long j = 0; j + 1 < len; ++j)
            ADJ_CUDA(forward_step(v, L, seg + (size_t)j * L.state_bytes, seg + (size_t)(j + 1) * L.state_bytes, st),
                     "recompute step");
        for (long j = len - 1; j >= 0; --j) {
            set_forward(a, v, L, seg + (size_t)j * L.state_bytes);
            a.lam_in = lam[cur];
            a.lam_out = lam[cur ^ 1];
            ADJ_CUDA(launch_adjoint(v.prm.storage, v.prm.induction, false, v.sp, a, st, nullptr), "adjoint step");
            cur ^= 1;
        }
    }
    return GLBE_OK;
}

}  // extern "C"
