// glbe_cavity.cuh -- the step of grids with a fluid box and / or a moving
// lid: the 3D lid-driven cavity of Sec. 5 and its MHD case on an extended
// magnetic domain.  One node per thread.
//
// Wall planes of the grid (wall_lo / wall_hi) bound both lattices: the flow
// lattice bounces back there and the vector lattice anti-bounces to B0 (a
// zero induced field).  The flow lattice is fluid only inside the box
// [blo, bhi]; a link whose source lies outside it is bounced back half-way,
// and when the source lies above the highest fluid z plane (the lid) it
// returns with the lid's momentum 6 w_a rho0 (e_a . U) added (Ladd's
// moving-wall rule; the preconditioned equilibrium keeps the unscaled linear
// term 3 e.j, so the term is the plain scheme's).  Outside the box, up to the
// wall planes, the vector lattice continues at rest: its collision relaxes
// g to W_a B (u = 0, Eq. mcollision), no Lorentz force is formed there, and
// the magnetic field diffuses out to the zero induced field at the walls.
#pragma once

namespace glbe {

__device__ __forceinline__ bool in_box(const StepParams& p, int x, int y, int z)
{
    return x >= p.blo[0] && x <= p.bhi[0] && y >= p.blo[1] && y <= p.bhi[1] && z >= p.blo[2] && z <= p.bhi[2];
}

// Gather of f for a fluid node of the box: source x - e_a (periodic wrap on
// axes without walls); a source on a wall plane or outside the box is
// bounced back (own slot of the opposite direction), plus the lid term when
// it lies above top_z.
template <int ST>
__device__ __forceinline__ void load_f_box(const StepParams& p, const typename Store<ST>::T* __restrict__ fs,
                                           const Geo& g, float (&d)[19], float (&l)[19])
{
    const size_t N = p.N;
    const __half* __restrict__ fl = Store<ST>::COMP ? reinterpret_cast<const __half*>(fs + 19 * N) : nullptr;
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        const int ex = dir_ex(a), ey = dir_ey(a), ez = dir_ez(a);
        int sx = g.x - ex, sy = g.y - ey, sz = g.z - ez;
        sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
        sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
        sz = sz < 0 ? sz + p.nz : (sz >= p.nz ? sz - p.nz : sz);
        const bool solid = plane_solid(sx, p.nx, p.wlo[0], p.whi[0]) || plane_solid(sy, p.ny, p.wlo[1], p.whi[1]) ||
                           plane_solid(sz, p.nz, p.wlo[2], p.whi[2]) || !in_box(p, sx, sy, sz);
        const int o = dir_opp(a);
        const size_t slot = solid ? (size_t)o * N + g.n
                                  : (size_t)a * N + ((size_t)sz * p.ny + (size_t)sy) * p.nx + (size_t)sx;
        d[a] = unscale<ST>(p, Store<ST>::ld(fs + slot));
        if constexpr (Store<ST>::COMP) l[a] = Store<ST_F32C>::ld_lo(fl + slot);
        if (solid && g.z - ez > p.top_z) {
            const float c = p.lid_corr[a];
            if constexpr (Store<ST>::COMP) {
                // exact: the rounding of high part + lid term goes to the low part, so the
                // compensated form keeps its resolution at the lid (a rounded add there
                // floored the cavity's residual near 1.7e-7)
                const float s = vadd_rn(d[a], c);
                const float bp = vsub_rn(s, d[a]);
                const float e = vadd_rn(vsub_rn(d[a], vsub_rn(s, bp)), vsub_rn(c, bp));
                d[a] = s;
                l[a] = vadd_rn(l[a], e);
            } else {
                d[a] += c;
            }
        }
    }
}

// Vector lattice alone at a node outside the box (u = 0, no Lorentz force).
template <int ST, int MODE>
__device__ __forceinline__ void induction_at_rest(const StepParams& p, const StepBuffers& b, const FieldOut& fo,
                                                  uint32_t n, const float (&q)[21], const float (&ql)[21])
{
    using S = Store<ST>;
    using T = typename S::T;
    constexpr bool PRECISE = (ST == ST_F32 || ST == ST_F32C);
    const size_t N = p.N;
    float og[21];
    NodeMacro<float> mac;
    const float zero = 0.f;
    induction_collide<float, PRECISE, S::COMP>(p, q, ql, og, 1.f, zero, zero, zero, zero, zero, zero, zero, zero,
                                               zero, mac);
    if (MODE == MODE_FIELDS) {
        if (fo.rho) fo.rho[n] = 0.f;
        if (fo.u) { fo.u[n] = 0.f; fo.u[N + n] = 0.f; fo.u[2 * N + n] = 0.f; }
        if (fo.B) { fo.B[n] = mac.Bx; fo.B[N + n] = mac.By; fo.B[2 * N + n] = mac.Bz; }
        return;
    }
    T* __restrict__ gd = static_cast<T*>(b.gdst);
    if constexpr (S::COMP) {
        __half* __restrict__ gdl = reinterpret_cast<__half*>(gd + 21 * N);
#pragma unroll
        for (int a = 0; a < 21; ++a) {
            float nh, nl;
            comp_add(q[a], ql[a], og[a], nh, nl);
            gd[(size_t)a * N + n] = nh;
            gdl[(size_t)a * N + n] = S::cv_lo(nl);
        }
    } else {
#pragma unroll
        for (int a = 0; a < 21; ++a) gd[(size_t)a * N + n] = S::cv(toscale<ST>(p, q[a] + og[a]));
    }
    b.FL[n] = 0.f;
    b.FL[N + n] = 0.f;
    b.FL[2 * N + n] = 0.f;
}

template <int ST, bool MHD, int MODE, int COLL>
__global__ void __launch_bounds__(STEP_THREADS) cavity_kernel(const StepParams p, const StepBuffers b,
                                                              const FieldOut fo)
{
    using T = typename Store<ST>::T;
    if (b.stop != nullptr && *b.stop) return;
    const uint32_t i = blockIdx.x * STEP_THREADS + threadIdx.x;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < p.N) {
        const uint32_t n = i;
        const size_t N = p.N;
        const Geo g = make_geo(p, n);
        if (g.solid) {
            if (MODE == MODE_FIELDS) {
                if (fo.rho) fo.rho[n] = 0.f;
                if (fo.u) { fo.u[n] = 0.f; fo.u[N + n] = 0.f; fo.u[2 * N + n] = 0.f; }
                if (MHD && fo.B) { fo.B[n] = 0.f; fo.B[N + n] = 0.f; fo.B[2 * N + n] = 0.f; }
            }
        } else {
            float q[21], ql[21];
            int wp = 0, wm = 0;
            if (is_interior(p, n, wp, wm)) {
                // inside the box with a margin of one node: every source at a fixed offset
                float d[19], dl[19];
                load_f_interior<ST>(p, static_cast<const T*>(b.fsrc), n, wp, wm, d, dl);
                if (MHD) load_g_interior<ST>(p, static_cast<const T*>(b.gsrc), n, wp, wm, q, ql);
                node_from_sources<ST, MHD, MODE, false, COLL>(p, b, fo, n, d, dl, q, ql, node_inputs<MHD, MODE>(p, b, n),
                                                             acc);
            } else {
            if (MHD) load_g<ST>(p, static_cast<const T*>(b.gsrc), g, q, ql);
            if (in_box(p, g.x, g.y, g.z)) {
                float d[19], dl[19];
                load_f_box<ST>(p, static_cast<const T*>(b.fsrc), g, d, dl);
                node_from_sources<ST, MHD, MODE, false, COLL>(p, b, fo, n, d, dl, q, ql, node_inputs<MHD, MODE>(p, b, n),
                                                             acc);
            } else if (MHD) {
                induction_at_rest<ST, MODE>(p, b, fo, n, q, ql);
            } else if (MODE == MODE_FIELDS) {
                if (fo.rho) fo.rho[n] = 0.f;
                if (fo.u) { fo.u[n] = 0.f; fo.u[N + n] = 0.f; fo.u[2 * N + n] = 0.f; }
            }
            }
        }
    }
    if (MODE == MODE_STEP_RESID) block_partials<STEP_THREADS>(acc, b.partials);
}

// The coupled cavity step in two passes per thread (the FP32 forms; the
// one-pass coupled F32C update needs 172 registers, one block per SM):
// pass 1 gathers f and g of a box node, forms rho and m and runs the
// induction part (g~ and this step's Lorentz force; a node outside the box
// relaxes g at rest); pass 2 gathers f again and runs the flow update with
// F = F_ext + F_L.  The one-pass arithmetic in the same order, bit for bit.
template <int ST, int MODE>
__global__ void __launch_bounds__(STEP_THREADS, 2) cavity_kernel_coupled2(const StepParams p, const StepBuffers b,
                                                                           const FieldOut fo)
{
    using T = typename Store<ST>::T;
    if (b.stop != nullptr && *b.stop) return;
    const uint32_t i = blockIdx.x * STEP_THREADS + threadIdx.x;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    bool box_node = false, interior = false;
    int wp = 0, wm = 0;
    Geo g{};
    if (i < p.N) {
        const uint32_t n = i;
        g = make_geo(p, n);
        if (!g.solid) {
            float q[21], ql[21];
            interior = is_interior(p, n, wp, wm);
            if (interior) load_g_interior<ST>(p, static_cast<const T*>(b.gsrc), n, wp, wm, q, ql);
            else load_g<ST>(p, static_cast<const T*>(b.gsrc), g, q, ql);
            box_node = in_box(p, g.x, g.y, g.z);
            if (box_node) {
                float d[19], dl[19];
                if (interior) load_f_interior<ST>(p, static_cast<const T*>(b.fsrc), n, wp, wm, d, dl);
                else load_f_box<ST>(p, static_cast<const T*>(b.fsrc), g, d, dl);
                induction_from_sources<ST>(p, b, n, d, dl, q, ql);
            } else {
                induction_at_rest<ST, MODE>(p, b, fo, n, q, ql);
            }
        }
    }
    if (box_node) {
        const uint32_t n = i;
        float d[19], dl[19], q[21], ql[21];
        if (interior) load_f_interior<ST>(p, static_cast<const T*>(b.fsrc), n, wp, wm, d, dl);
        else load_f_box<ST>(p, static_cast<const T*>(b.fsrc), g, d, dl);
        node_from_sources<ST, false, MODE, false, 0>(p, b, fo, n, d, dl, q, ql, node_inputs<false, MODE, true>(p, b, n),
                                                     acc);
    }
    if (MODE == MODE_STEP_RESID) block_partials<STEP_THREADS>(acc, b.partials);
}

// Initial state under a moving lid.  A pull gathers from the other buffer as
// from the post-collision values of the previous step, so a link bounced off
// the lid returns with the lid term added.  For the first step to gather the
// rest state, the slot of every such link of buffer fbuf holds -lid_corr of
// the direction it returns as (the slot is read by that bounce only).
template <int ST>
__global__ void lid_init_kernel(const StepParams p, void* fbuf)
{
    using S = Store<ST>;
    using T = typename S::T;
    const uint32_t i = blockIdx.x * STEP_THREADS + threadIdx.x;
    if (i >= p.N) return;
    const Geo g = make_geo(p, i);
    if (g.solid || !in_box(p, g.x, g.y, g.z) || g.z != p.top_z) return;
    T* fs = static_cast<T*>(fbuf);
    const size_t N = p.N;
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        if (dir_ez(a) != -1) continue;     // returns from above the top fluid plane
        const int ex = dir_ex(a), ey = dir_ey(a);
        int sx = g.x - ex, sy = g.y - ey;
        sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
        sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
        const int sz = g.z + 1 >= p.nz ? g.z + 1 - p.nz : g.z + 1;
        const bool solid = plane_solid(sx, p.nx, p.wlo[0], p.whi[0]) || plane_solid(sy, p.ny, p.wlo[1], p.whi[1]) ||
                           plane_solid(sz, p.nz, p.wlo[2], p.whi[2]) || !in_box(p, sx, sy, sz);
        if (!solid) continue;
        const size_t slot = (size_t)dir_opp(a) * N + g.n;
        fs[slot] = S::cv(toscale<ST>(p, -p.lid_corr[a]));
        if constexpr (S::COMP) reinterpret_cast<__half*>(fs + 19 * N)[slot] = __float2half_rn(0.f);
    }
}

template <int ST>
cudaError_t launch_lid_init_t(const StepParams& p, void* fbuf, cudaStream_t st)
{
    const unsigned grid = (unsigned)(((size_t)p.N + STEP_THREADS - 1) / STEP_THREADS);
    lid_init_kernel<ST><<<grid, STEP_THREADS, 0, st>>>(p, fbuf);
    return cudaGetLastError();
}

}  // namespace glbe
