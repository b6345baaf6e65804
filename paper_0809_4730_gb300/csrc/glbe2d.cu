// glbe2d.cu -- the two-dimensional forms of the method: the preconditioned
// GLBE with forcing term on the D2Q9 lattice and the preconditioned vector
// lattice kinetic equation for the magnetic induction on the D2Q5 lattice
// (arXiv:0809.4730 Secs. 2-4, App. A D2Q9 tables), and their C-ABI
// (include/glbe2d.h).
//
// Same scheme as the D3Q19 library: a pull step, one node per thread.  The
// thread gathers the previous step's post-collision deviations from its
// upstream neighbours (half-way bounce-back for f, anti-bounce-back to B0 for
// g where the upstream node is solid), forms rho, j, B, J_z and the Lorentz
// force, collides in moment space and writes the new post-collision values
// into its own slots of the other buffer.  Buffers hold deviations from the
// rest state, df = f - w rho0, dg = g - W B0.
//
// The D2Q9 moment basis of App. A (rows rho, e, e^2, j_x, q_x, j_y, q_y,
// p_xx, p_xy) is applied through partial sums over the axis and diagonal
// groups; its inverse is T^t diag(1/|row_k|^2) with |row_k|^2 = 9, 36, 36,
// 6, 12, 6, 12, 4, 4.  The conserved rows change by 0 (rho) and F/gamma
// (j: the relaxation towards j = m + F/(2 gamma) and the source term add up
// to F/gamma whatever the rate).
//
// Memory traffic per node and step (algorithmic): f 9 values read and 9
// written, with induction g 10 read and 10 written and the lagged Lorentz
// force 2 read and 2 written (FP32), and the force field 2 read when present.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "glbe2d.h"
#include "glbe_internal.h"

using namespace glbe;

namespace {

constexpr int T2D = 256;               // threads per block, one node each
constexpr unsigned HIST_CAP2 = 4096;
constexpr size_t ALIGN2 = 256;
constexpr float LO2_SCALE = 68719476736.0f;        // 2^36: the FP16 low part of the compensated form
constexpr float LO2_INV = 1.4551915228366852e-11f; // 2^-36

size_t align2(size_t x) { return (x + ALIGN2 - 1) / ALIGN2 * ALIGN2; }

// D2Q9 (0 rest; 1 (1,0), 2 (0,1), 3 (-1,0), 4 (0,-1), 5 (1,1), 6 (-1,1),
// 7 (-1,-1), 8 (1,-1)) and D2Q5 (0 rest; 1 +x, 2 -x, 3 +y, 4 -y)
__host__ __device__ constexpr int ex9(int a) { return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0); }
__host__ __device__ constexpr int ey9(int a) { return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0); }
__host__ __device__ constexpr int ex5(int a) { return a == 1 ? 1 : (a == 2 ? -1 : 0); }
__host__ __device__ constexpr int ey5(int a) { return a == 3 ? 1 : (a == 4 ? -1 : 0); }
__host__ __device__ constexpr int opp5(int a) { return a == 0 ? 0 : (a == 1 ? 2 : (a == 2 ? 1 : (a == 3 ? 4 : 3))); }

// opposite directions of D2Q9, tabulated
__host__ __device__ constexpr int opp9t(int a)
{
    return a == 0 ? 0 : a == 1 ? 3 : a == 2 ? 4 : a == 3 ? 1 : a == 4 ? 2 : a == 5 ? 7 : a == 6 ? 8 : a == 7 ? 5 : 6;
}
static_assert(ex9(opp9t(5)) == -ex9(5) && ey9(opp9t(6)) == -ey9(6) && opp9t(opp9t(8)) == 8, "D2Q9 opposites");
static_assert(ex5(opp5(1)) == -1 && ey5(opp5(4)) == 1, "D2Q5 opposites");

// ---------------------------------------------------------------------------
// Storage: FP32, BF16, or FP32 + FP16 remainder (compensated; the low parts
// follow the high parts in the same buffer, scaled by 2^36).
// ---------------------------------------------------------------------------
// Read-only loads asking L2 for the whole 256-byte block (a warp reads 128
// bytes of a population row, the next warp the following 128).
__device__ __forceinline__ float ld256(const float* p)
{
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ unsigned short ld256(const unsigned short* p)
{
    unsigned short v;
    asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

template <int ST> struct Sto2;
template <> struct Sto2<GLBE_F32> {
    using T = float;
    static constexpr bool COMP = false;
    static __device__ __forceinline__ float ld(const T* p) { return ld256(p); }
    static __device__ __forceinline__ T cv(float v) { return v; }
};
template <> struct Sto2<GLBE_BF16> {
    using T = __nv_bfloat16;
    static constexpr bool COMP = false;
    static __device__ __forceinline__ float ld(const T* p)
    {
        return __uint_as_float((unsigned)ld256(reinterpret_cast<const unsigned short*>(p)) << 16);
    }
    static __device__ __forceinline__ T cv(float v) { return __float2bfloat16_rn(v); }
};
template <> struct Sto2<GLBE_F32C> {
    using T = float;
    static constexpr bool COMP = true;
    static __device__ __forceinline__ float ld(const T* p) { return ld256(p); }
    static __device__ __forceinline__ T cv(float v) { return v; }
};

struct P2 {
    int nx, ny, N;
    uint32_t div_m, div_s;    // n / nx = (umulhi(n, div_m) + n) >> div_s
    int wlx, whx, wly, why;
    int ix0, ix1, iy0, iy1;   // interior: every source fluid, no seam crossed
    float rho0;
    // relaxation of row k folded on the host: dm_k / |row_k|^2 = a_k n_k + b_k R_k,
    // n_k the non-equilibrium part, R_k the source polynomial of App. A
    // (rows 1, 2: F.u; 4, 6: F_x, F_y; 7: F_x u_x - F_y u_y; 8: F_x u_y + F_y u_x)
    float a1, a2, a4, a6, a7, a8;
    float b1, b2, b4, b6, b7, b8;
    float c3;                 // 1/(6 gamma): rows 3, 5 change by F/gamma
    float inv_gamma, half_inv_gamma;
    float Fx, Fy;
    // induction
    float inv_tau_m;       // 1/tau_m*
    float ceq;             // chi/(gamma_m theta_m): g^eq carries W_a e_ak ceq (u_k B_j - B_k u_j)
    float cJ;              // 1/(mu chi tau_m theta_m)
    float B0x, B0y;
};

struct B2 {
    const void* fsrc;
    void* fdst;
    const void* gsrc;
    void* gdst;
    float* FL;              // [2][N], read (lagged) and written in place
    const float* Ffield;    // [2][N] or null
    float* usnap;           // [4][N]: u_hi x, y and u_lo x, y of the last residual level
    double* partials;       // [8][blocks]
    int have_snap;
    const int* stop;        // solve: the kernels of a converged march return at once
    int pf_ahead;           // L2 prefetch of the rows block blockIdx.x + pf_ahead gathers (0: none)
};

struct Out2 {
    float* rho;
    float* u;
    float* B;
};

enum { M2_STEP = 0, M2_RESID = 1, M2_FIELDS = 2 };

__device__ __forceinline__ float warp_sum2(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// fl(a + b) with its exact rounding error
__device__ __forceinline__ float two_sum(float a, float b, float& e)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return s;
}

// Double-float running sum (high part plus accumulated rounding errors).
struct DF {
    float h, l;
    __device__ __forceinline__ void add(float x)
    {
        float e;
        h = two_sum(h, x, e);
        l = __fadd_rn(l, e);
    }
};

// Gathers the pre-collision deviations of node (x, y) from the buffer of the
// previous step: src of direction a is (x - e_a); a solid source bounces the
// node's own opposite population back (f) or returns it with the sign
// changed (g: anti-bounce-back to B0, the wall value being the applied field).
struct Nb {
    int xm, xp, ym, yp;        // periodic neighbours
    bool cm, cp, rm, rp;       // the column x-1 / x+1, the row y-1 / y+1 is a wall line
};

__device__ __forceinline__ Nb neighbours(const P2& p, int x, int y)
{
    Nb b;
    b.xm = x == 0 ? p.nx - 1 : x - 1;
    b.xp = x == p.nx - 1 ? 0 : x + 1;
    b.ym = y == 0 ? p.ny - 1 : y - 1;
    b.yp = y == p.ny - 1 ? 0 : y + 1;
    b.cm = (p.wlx && b.xm == 0) || (p.whx && b.xm == p.nx - 1);
    b.cp = (p.wlx && b.xp == 0) || (p.whx && b.xp == p.nx - 1);
    b.rm = (p.wly && b.ym == 0) || (p.why && b.ym == p.ny - 1);
    b.rp = (p.wly && b.yp == 0) || (p.why && b.yp == p.ny - 1);
    return b;
}

__device__ __forceinline__ bool is_solid(const P2& p, int x, int y)
{
    return (p.wlx && x == 0) || (p.whx && x == p.nx - 1) || (p.wly && y == 0) || (p.why && y == p.ny - 1);
}

__device__ __forceinline__ int row_of(const P2& p, int n)
{
    return (int)((__umulhi((uint32_t)n, p.div_m) + (uint32_t)n) >> p.div_s);
}

// source node of a direction (ex, ey) and whether it is solid
__device__ __forceinline__ int source(const P2& p, const Nb& b, int x, int y, int ex, int ey, bool& solid)
{
    const int xs = ex == 1 ? b.xm : (ex == -1 ? b.xp : x);
    const int ys = ey == 1 ? b.ym : (ey == -1 ? b.yp : y);
    solid = (ex == 1 && b.cm) || (ex == -1 && b.cp) || (ey == 1 && b.rm) || (ey == -1 && b.rp);
    return ys * p.nx + xs;
}

template <int ST>
__device__ __forceinline__ void gather_f(const P2& p, const Nb& b, int x, int y, int n, const void* buf, float (&d)[9],
                                         float (&dl)[9])
{
    using S = Sto2<ST>;
    const typename S::T* f = static_cast<const typename S::T*>(buf);
    const __half* fl = S::COMP ? reinterpret_cast<const __half*>(static_cast<const float*>(buf) + 9 * (size_t)p.N)
                               : nullptr;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        bool sol;
        const int s = source(p, b, x, y, ex9(a), ey9(a), sol);
        // row of direction a (or of its opposite, bounced back) and the node in it
        const int row = sol ? opp9t(a) : a;
        const int at = sol ? n : s;
        d[a] = S::ld(f + (size_t)row * p.N + at);
        dl[a] = S::COMP ? __half2float(__ldg(fl + (size_t)row * p.N + at)) * LO2_INV : 0.f;
    }
}

template <int ST>
__device__ __forceinline__ void gather_g(const P2& p, const Nb& b, int x, int y, int n, const void* buf, float (&q)[10],
                                         float (&ql)[10])
{
    using S = Sto2<ST>;
    const typename S::T* g = static_cast<const typename S::T*>(buf);
    const __half* gl = S::COMP ? reinterpret_cast<const __half*>(static_cast<const float*>(buf) + 10 * (size_t)p.N)
                               : nullptr;
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        bool sol;
        const int s = source(p, b, x, y, ex5(a), ey5(a), sol);
        const int at = sol ? n : s;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int row = j * 5 + (sol ? opp5(a) : a);
            const float v = S::ld(g + (size_t)row * p.N + at);
            const float vl = S::COMP ? __half2float(__ldg(gl + (size_t)row * p.N + at)) * LO2_INV : 0.f;
            q[j * 5 + a] = sol ? -v : v;
            ql[j * 5 + a] = sol ? -vl : vl;
        }
    }
}

// Interior nodes (every source fluid and inside the grid): direction a's
// source is n - (e_ax + e_ay nx), read at a fixed offset from its row.
template <int ST>
__device__ __forceinline__ void gather_f_interior(const P2& p, int n, const void* buf, float (&d)[9], float (&dl)[9])
{
    using S = Sto2<ST>;
    const typename S::T* f = static_cast<const typename S::T*>(buf);
    const __half* fl = S::COMP ? reinterpret_cast<const __half*>(static_cast<const float*>(buf) + 9 * (size_t)p.N)
                               : nullptr;
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const ptrdiff_t k = (ptrdiff_t)a * p.N - (ex9(a) + ey9(a) * p.nx) + n;
        d[a] = S::ld(f + k);
        dl[a] = S::COMP ? __half2float(__ldg(fl + k)) * LO2_INV : 0.f;
    }
}

template <int ST>
__device__ __forceinline__ void gather_g_interior(const P2& p, int n, const void* buf, float (&q)[10], float (&ql)[10])
{
    using S = Sto2<ST>;
    const typename S::T* g = static_cast<const typename S::T*>(buf);
    const __half* gl = S::COMP ? reinterpret_cast<const __half*>(static_cast<const float*>(buf) + 10 * (size_t)p.N)
                               : nullptr;
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const int a = i % 5;
        const ptrdiff_t k = (ptrdiff_t)i * p.N - (ex5(a) + ey5(a) * p.nx) + n;
        q[i] = S::ld(g + k);
        ql[i] = S::COMP ? __half2float(__ldg(gl + k)) * LO2_INV : 0.f;
    }
}

// Linear moments of the deviations (App. A basis, D2Q9).
struct Mom9 {
    float drho, e, e2, mx, qx, my, qy, pxx, pxy;
};
__device__ __forceinline__ Mom9 moments9(const float (&d)[9])
{
    Mom9 m;
    const float ax = d[1] + d[3], ay = d[2] + d[4];
    const float dg = d[5] + d[6] + d[7] + d[8];
    const float sx = d[1] - d[3], sy = d[2] - d[4];
    const float gx = d[5] - d[6] - d[7] + d[8];
    const float gy = d[5] + d[6] - d[7] - d[8];
    m.drho = d[0] + ax + ay + dg;
    m.e = -4.f * d[0] - (ax + ay) + 2.f * dg;
    m.e2 = 4.f * d[0] - 2.f * (ax + ay) + dg;
    m.mx = sx + gx;
    m.qx = -2.f * sx + gx;
    m.my = sy + gy;
    m.qy = -2.f * sy + gy;
    m.pxx = ax - ay;
    m.pxy = d[5] - d[6] + d[7] - d[8];
    return m;
}

// Macroscopic quantities of a node.
struct Node2 {
    float rho, jx, jy, ux, uy;     // u = j/rho, j = m + F/(2 gamma) with F including the Lorentz force
    float Bx, By, FLx, FLy;
};

// Exact split of a deviation into a part on the 2^-28 grid (whose sums with
// small integer weights are exact in FP32 while below 2^-4) and a remainder:
// the moments of the parts are then exact up to the remainder's own
// rounding (~1e-16), so that the FP32 time march settles on its fixed point
// instead of wandering at the round-off of the large moment sums.
constexpr float SPLIT2 = 0.046875f;   // 1.5 * 2^-5
__device__ __forceinline__ void split2(float x, float& h, float& l)
{
    h = __fsub_rn(__fadd_rn(x, SPLIT2), SPLIT2);
    l = __fsub_rn(x, h);
}

// Induction part: B, J_z, the Lorentz force (-J_z B_y, J_z B_x) and the
// D2Q5 collision increments og (Sec. 4).  u0 is the velocity g^eq sees: the
// half force of the previous step's Lorentz force and the external force.
// ql: the low parts of the compensated storage (0 otherwise).
template <bool COLLIDE, bool PRECISE>
__device__ __forceinline__ void induction2(const P2& p, const float (&q)[10], const float (&ql)[10], float u0x,
                                           float u0y, Node2& nd, float (&og)[10])
{
    float dBx, dBy;
    if constexpr (PRECISE) {
        float h[10], l[10];
#pragma unroll
        for (int i = 0; i < 10; ++i) {
            split2(q[i], h[i], l[i]);
            l[i] += ql[i];
        }
        dBx = (h[0] + h[1] + h[2] + h[3] + h[4]) + (l[0] + l[1] + l[2] + l[3] + l[4]);
        dBy = (h[5] + h[6] + h[7] + h[8] + h[9]) + (l[5] + l[6] + l[7] + l[8] + l[9]);
    } else {
        dBx = q[0] + q[1] + q[2] + q[3] + q[4];
        dBy = q[5] + q[6] + q[7] + q[8] + q[9];
    }
    nd.Bx = p.B0x + dBx;
    nd.By = p.B0y + dBy;
    // E = u_x B_y - u_y B_x; g^eq deviations (W_0 = 1/3, W_a = 1/6):
    //   x: W dBx on 0, +-x; W (dBx -+ ceq E) on +-y;
    //   y: W (dBy +- ceq E) on +-x; W dBy on 0, +-y
    const float cE = p.ceq * (u0x * nd.By - u0y * nd.Bx);
    constexpr float W0 = 1.f / 3.f, W1 = 1.f / 6.f;
    // non-equilibrium first moments L[k][j] = sum_a e_ak (g - g^eq)_ja; the
    // equilibrium's part of (+x) - (-x) of B_y is 2 W_1 ceq E = ceq E / 3
    const float Lxy = ((q[6] - q[7]) + (ql[6] - ql[7])) - cE * (1.f / 3.f);
    const float Lyx = ((q[3] - q[4]) + (ql[3] - ql[4])) + cE * (1.f / 3.f);
    const float Jz = -p.cJ * (Lxy - Lyx);
    nd.FLx = -Jz * nd.By;
    nd.FLy = Jz * nd.Bx;
    if (COLLIDE) {
        float geq[10];
        geq[0] = W0 * dBx;
        geq[1] = W1 * dBx;
        geq[2] = W1 * dBx;
        geq[3] = W1 * (dBx - cE);
        geq[4] = W1 * (dBx + cE);
        geq[5] = W0 * dBy;
        geq[6] = W1 * (dBy + cE);
        geq[7] = W1 * (dBy - cE);
        geq[8] = W1 * dBy;
        geq[9] = W1 * dBy;
#pragma unroll
        for (int i = 0; i < 10; ++i) og[i] = -((q[i] - geq[i]) + ql[i]) * p.inv_tau_m;
    }
}

// D2Q9 collision increments om (Sec. 3, App. A): dm_k = -s_k (m_k - m_k^eq)
// + (1 - s_k/2) S*_k, back to particle space through T^t diag(1/|row|^2).
// H and L are the moments of the high and low parts of the deviations (L = 0
// without the exact split); the non-equilibrium parts are formed from the
// exact high sums first.
__device__ __forceinline__ void collide9(const P2& p, const Mom9& H, const Mom9& L, const Node2& nd, float Fx,
                                         float Fy, float (&om)[9])
{
    const float rg = p.inv_gamma / nd.rho;              // 1/(gamma rho)
    const float jj3 = 3.f * (nd.jx * nd.jx + nd.jy * nd.jy) * rg;
    const float Fu = Fx * nd.ux + Fy * nd.uy;
    // m_k - m_k^eq: e^eq = -2 drho + 3 j.j/(gamma rho), e2^eq = drho - 3 j.j/(gamma rho),
    // q^eq = -j, p_xx^eq = (jx^2 - jy^2)/(gamma rho), p_xy^eq = jx jy/(gamma rho)
    const float ne = ((H.e + 2.f * H.drho) + (L.e + 2.f * L.drho)) - jj3;
    const float ne2 = ((H.e2 - H.drho) + (L.e2 - L.drho)) + jj3;
    const float nqx = ((H.qx + H.mx) + (L.qx + L.mx)) + p.half_inv_gamma * Fx;
    const float nqy = ((H.qy + H.my) + (L.qy + L.my)) + p.half_inv_gamma * Fy;
    const float npxx = (H.pxx + L.pxx) - (nd.jx * nd.jx - nd.jy * nd.jy) * rg;
    const float npxy = (H.pxy + L.pxy) - nd.jx * nd.jy * rg;
    const float d1 = fmaf(p.a1, ne, p.b1 * Fu);
    const float d2 = fmaf(p.a2, ne2, p.b2 * Fu);
    const float d3 = p.c3 * Fx;
    const float d4 = fmaf(p.a4, nqx, p.b4 * Fx);
    const float d5 = p.c3 * Fy;
    const float d6 = fmaf(p.a6, nqy, p.b6 * Fy);
    const float d7 = fmaf(p.a7, npxx, p.b7 * (Fx * nd.ux - Fy * nd.uy));
    const float d8 = fmaf(p.a8, npxy, p.b8 * (Fx * nd.uy + Fy * nd.ux));
    const float A = -d1 - 2.f * d2;            // axis directions: e = -1, e^2 = -2
    const float Dg = 2.f * d1 + d2;            // diagonals: e = 2, e^2 = 1
    const float X1 = d3 - 2.f * d4, Y1 = d5 - 2.f * d6;
    const float X2 = d3 + d4, Y2 = d5 + d6;
    om[0] = -4.f * d1 + 4.f * d2;
    om[1] = A + X1 + d7;
    om[3] = A - X1 + d7;
    om[2] = A + Y1 - d7;
    om[4] = A - Y1 - d7;
    om[5] = Dg + X2 + Y2 + d8;
    om[6] = Dg - X2 + Y2 - d8;
    om[7] = Dg - X2 - Y2 + d8;
    om[8] = Dg + X2 - Y2 - d8;
}

// new = old + inc into the storage; the compensated form keeps the rounding
// remainder (with the old remainder) in the low part.
template <int ST>
__device__ __forceinline__ void put(void* buf, size_t N, int rows, size_t k, float old, float old_lo, float inc)
{
    using S = Sto2<ST>;
    typename S::T* f = static_cast<typename S::T*>(buf);
    if constexpr (S::COMP) {
        float e;
        const float s = two_sum(old, inc, e);
        const float t = __fadd_rn(e, old_lo);
        const float hi = __fadd_rn(s, t);
        const float lo = __fsub_rn(t, __fsub_rn(hi, s));
        f[k] = hi;
        reinterpret_cast<__half*>(static_cast<float*>(buf) + rows * N)[k] = __float2half_rn(lo * LO2_SCALE);
    } else {
        f[k] = S::cv(old + inc);
    }
}

// The update of one node from its gathered pre-collision deviations (d, dl:
// f and its compensated low parts; q, ql: g), the external force and the
// lagged Lorentz force: the macroscopic fields in nd, the total force F and,
// with COLLIDE, the collision changes om (f) and og (g).
template <int ST, bool MHD, bool COLLIDE>
__device__ __forceinline__ void node_update2(const P2& p, const float (&d)[9], const float (&dl)[9],
                                             const float (&q)[10], const float (&ql)[10], float Fex, float Fey,
                                             float FLpx, float FLpy, Node2& nd, float& Fx, float& Fy, float (&om)[9],
                                             float (&og)[10])
{
    // FP32 storage forms: moments from the exact split (high parts on the
    // 2^-28 grid, low parts with the compensated remainder)
    constexpr bool PRECISE = (ST == GLBE_F32 || ST == GLBE_F32C);
    Mom9 H, L;
    if constexpr (PRECISE) {
        float dh[9], dlo[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            split2(d[a], dh[a], dlo[a]);
            dlo[a] += dl[a];
        }
        H = moments9(dh);
        L = moments9(dlo);
    } else {
        H = moments9(d);
        L = Mom9{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    }
    const float drho = H.drho + L.drho;
    nd.rho = p.rho0 + drho;
    const float rinv = 1.f / nd.rho;
    const float mx = H.mx + L.mx, my = H.my + L.my;
    nd.Bx = nd.By = nd.FLx = nd.FLy = 0.f;
    if (MHD) {
        const float u0x = (mx + p.half_inv_gamma * (Fex + FLpx)) * rinv;
        const float u0y = (my + p.half_inv_gamma * (Fey + FLpy)) * rinv;
        induction2<COLLIDE, PRECISE>(p, q, ql, u0x, u0y, nd, og);
    }
    Fx = Fex + nd.FLx;
    Fy = Fey + nd.FLy;
    if constexpr (PRECISE) {
        // j = m + F/(2 gamma): high sum and half force added exactly, rounded once
        float ex, ey;
        const float sx = two_sum(H.mx, p.half_inv_gamma * Fx, ex);
        const float sy = two_sum(H.my, p.half_inv_gamma * Fy, ey);
        nd.jx = sx + (ex + L.mx);
        nd.jy = sy + (ey + L.my);
    } else {
        nd.jx = mx + p.half_inv_gamma * Fx;
        nd.jy = my + p.half_inv_gamma * Fy;
    }
    nd.ux = nd.jx * rinv;
    nd.uy = nd.jy * rinv;
    if (COLLIDE) collide9(p, H, L, nd, Fx, Fy, om);
}

// ---------------------------------------------------------------------------
// The BF16 node update, written once for one node (V = float) and for two
// x-adjacent nodes at once (V = V2: packed FP32x2 instructions, one
// instruction for both nodes).  Every operation is explicit and rounded on
// its own -- nothing is left to the compiler to contract -- so the two-node
// form gives the one-node form's values bit for bit.  Same moments, fields,
// collision (Sec. 3, App. A) and induction part (Sec. 4) as node_update2
// without the exact split.
// ---------------------------------------------------------------------------
struct V2 {
    float2 v;
    __device__ __forceinline__ V2() {}
    __device__ __forceinline__ V2(float c) : v(make_float2(c, c)) {}
    __device__ __forceinline__ V2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ V2 vadd(V2 a, V2 b)
{
    V2 r;
    r.v = __fadd2_rn(a.v, b.v);
    return r;
}
// a - b = fma(b, -1, a), rounded once like the scalar subtraction
__device__ __forceinline__ V2 vsub(V2 a, V2 b)
{
    V2 r;
    r.v = __ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v);
    return r;
}
__device__ __forceinline__ V2 vmul(V2 a, V2 b)
{
    V2 r;
    r.v = __fmul2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ V2 vfma(V2 a, V2 b, V2 c)
{
    V2 r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
}
__device__ __forceinline__ V2 vdiv(V2 a, V2 b) { return V2(__fdiv_rn(a.v.x, b.v.x), __fdiv_rn(a.v.y, b.v.y)); }
template <class V>
__device__ __forceinline__ V vneg(V a) { return vmul(V(-1.f), a); }

template <class V>
struct Mom9V {
    V drho, e, e2, mx, qx, my, qy, pxx, pxy;
};
template <class V>
__device__ __forceinline__ Mom9V<V> moments9v(const V (&d)[9])
{
    Mom9V<V> m;
    const V ax = vadd(d[1], d[3]), ay = vadd(d[2], d[4]);
    const V dg = vadd(vadd(d[5], d[6]), vadd(d[7], d[8]));
    const V sx = vsub(d[1], d[3]), sy = vsub(d[2], d[4]);
    const V gx = vadd(vsub(d[5], d[6]), vsub(d[8], d[7]));
    const V gy = vsub(vadd(d[5], d[6]), vadd(d[7], d[8]));
    const V axy = vadd(ax, ay);
    m.drho = vadd(vadd(d[0], axy), dg);
    m.e = vfma(V(2.f), dg, vsub(vmul(V(-4.f), d[0]), axy));
    m.e2 = vadd(vfma(V(-2.f), axy, vmul(V(4.f), d[0])), dg);
    m.mx = vadd(sx, gx);
    m.qx = vfma(V(-2.f), sx, gx);
    m.my = vadd(sy, gy);
    m.qy = vfma(V(-2.f), sy, gy);
    m.pxx = vsub(ax, ay);
    m.pxy = vadd(vsub(d[5], d[6]), vsub(d[7], d[8]));
    return m;
}

template <class V>
struct Node2V {
    V rho, jx, jy, ux, uy;
    V Bx, By, FLx, FLy;
};

template <class V, bool COLLIDE>
__device__ __forceinline__ void induction2v(const P2& p, const V (&q)[10], V u0x, V u0y, Node2V<V>& nd, V (&og)[10])
{
    const V dBx = vadd(vadd(vadd(q[0], q[1]), vadd(q[2], q[3])), q[4]);
    const V dBy = vadd(vadd(vadd(q[5], q[6]), vadd(q[7], q[8])), q[9]);
    nd.Bx = vadd(V(p.B0x), dBx);
    nd.By = vadd(V(p.B0y), dBy);
    // E = u_x B_y - u_y B_x; the equilibrium's part of (+x) - (-x) of B_y is ceq E / 3
    const V cE = vmul(V(p.ceq), vsub(vmul(u0x, nd.By), vmul(u0y, nd.Bx)));
    const V cE3 = vmul(cE, V(1.f / 3.f));
    const V Lxy = vsub(vsub(q[6], q[7]), cE3);
    const V Lyx = vadd(vsub(q[3], q[4]), cE3);
    const V nJz = vmul(V(p.cJ), vsub(Lxy, Lyx));      // -J_z
    nd.FLx = vmul(nJz, nd.By);                        // -J_z B_y
    nd.FLy = vneg(vmul(nJz, nd.Bx));                  //  J_z B_x
    if (COLLIDE) {
        constexpr float W0 = 1.f / 3.f, W1 = 1.f / 6.f;
        V geq[10];
        geq[0] = vmul(V(W0), dBx);
        geq[1] = vmul(V(W1), dBx);
        geq[2] = geq[1];
        geq[3] = vmul(V(W1), vsub(dBx, cE));
        geq[4] = vmul(V(W1), vadd(dBx, cE));
        geq[5] = vmul(V(W0), dBy);
        geq[6] = vmul(V(W1), vadd(dBy, cE));
        geq[7] = vmul(V(W1), vsub(dBy, cE));
        geq[8] = vmul(V(W1), dBy);
        geq[9] = geq[8];
#pragma unroll
        for (int i = 0; i < 10; ++i) og[i] = vmul(vsub(geq[i], q[i]), V(p.inv_tau_m));
    }
}

template <class V>
__device__ __forceinline__ void collide9v(const P2& p, const Mom9V<V>& H, const Node2V<V>& nd, V Fx, V Fy,
                                          V (&om)[9])
{
    const V rg = vdiv(V(p.inv_gamma), nd.rho);
    const V jj3 = vmul(vmul(V(3.f), vfma(nd.jx, nd.jx, vmul(nd.jy, nd.jy))), rg);
    const V Fu = vfma(Fx, nd.ux, vmul(Fy, nd.uy));
    const V ne = vsub(vfma(V(2.f), H.drho, H.e), jj3);
    const V ne2 = vadd(vsub(H.e2, H.drho), jj3);
    const V nqx = vfma(V(p.half_inv_gamma), Fx, vadd(H.qx, H.mx));
    const V nqy = vfma(V(p.half_inv_gamma), Fy, vadd(H.qy, H.my));
    const V npxx = vsub(H.pxx, vmul(vfma(nd.jx, nd.jx, vneg(vmul(nd.jy, nd.jy))), rg));
    const V npxy = vsub(H.pxy, vmul(vmul(nd.jx, nd.jy), rg));
    const V d1 = vfma(V(p.a1), ne, vmul(V(p.b1), Fu));
    const V d2 = vfma(V(p.a2), ne2, vmul(V(p.b2), Fu));
    const V d3 = vmul(V(p.c3), Fx);
    const V d4 = vfma(V(p.a4), nqx, vmul(V(p.b4), Fx));
    const V d5 = vmul(V(p.c3), Fy);
    const V d6 = vfma(V(p.a6), nqy, vmul(V(p.b6), Fy));
    const V d7 = vfma(V(p.a7), npxx, vmul(V(p.b7), vfma(Fx, nd.ux, vneg(vmul(Fy, nd.uy)))));
    const V d8 = vfma(V(p.a8), npxy, vmul(V(p.b8), vfma(Fx, nd.uy, vmul(Fy, nd.ux))));
    const V A = vneg(vfma(V(2.f), d2, d1));          // axis directions: e = -1, e^2 = -2
    const V Dg = vfma(V(2.f), d1, d2);               // diagonals: e = 2, e^2 = 1
    const V X1 = vfma(V(-2.f), d4, d3), Y1 = vfma(V(-2.f), d6, d5);
    const V X2 = vadd(d3, d4), Y2 = vadd(d5, d6);
    om[0] = vmul(V(4.f), vsub(d2, d1));
    om[1] = vadd(vadd(A, X1), d7);
    om[3] = vadd(vsub(A, X1), d7);
    om[2] = vsub(vadd(A, Y1), d7);
    om[4] = vsub(vsub(A, Y1), d7);
    om[5] = vadd(vadd(vadd(Dg, X2), Y2), d8);
    om[6] = vsub(vadd(vsub(Dg, X2), Y2), d8);
    om[7] = vadd(vsub(vsub(Dg, X2), Y2), d8);
    om[8] = vsub(vsub(vadd(Dg, X2), Y2), d8);
}

template <class V, bool MHD, bool COLLIDE>
__device__ __forceinline__ void node_update2v(const P2& p, const V (&d)[9], const V (&q)[10], V Fex, V Fey, V FLpx,
                                              V FLpy, Node2V<V>& nd, V& Fx, V& Fy, V (&om)[9], V (&og)[10])
{
    const Mom9V<V> H = moments9v(d);
    nd.rho = vadd(V(p.rho0), H.drho);
    const V rinv = vdiv(V(1.f), nd.rho);
    nd.Bx = nd.By = nd.FLx = nd.FLy = V(0.f);
    if (MHD) {
        const V u0x = vmul(vfma(V(p.half_inv_gamma), vadd(Fex, FLpx), H.mx), rinv);
        const V u0y = vmul(vfma(V(p.half_inv_gamma), vadd(Fey, FLpy), H.my), rinv);
        induction2v<V, COLLIDE>(p, q, u0x, u0y, nd, og);
        Fx = vadd(Fex, nd.FLx);
        Fy = vadd(Fey, nd.FLy);
    } else {
        Fx = Fex;
        Fy = Fey;
    }
    nd.jx = vfma(V(p.half_inv_gamma), Fx, H.mx);
    nd.jy = vfma(V(p.half_inv_gamma), Fy, H.my);
    nd.ux = vmul(nd.jx, rinv);
    nd.uy = vmul(nd.jy, rinv);
    if (COLLIDE) collide9v(p, H, nd, Fx, Fy, om);
}

// u of a residual level as a double-float pair: the sums of the deviations
// (with their low parts) carried with their rounding errors, so that the
// residual resolves changes of u below one unit in the last place of its
// FP32 value.  Adds the node's terms to acc (num, den, sum drho, jx, jy,
// -, nonfinite) against the snapshot (us: u_hi x, y, u_lo x, y) and returns
// the new snapshot in us.
__device__ __forceinline__ void resid_node(const P2& p, const float (&d)[9], const float (&dl)[9], float Fx, float Fy,
                                           bool have_snap, float (&us)[4], float (&acc)[7])
{
    DF r{0.f, 0.f}, sx{0.f, 0.f}, sy{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        r.add(d[a]);
        r.l += dl[a];
        if (ex9(a) != 0) {
            sx.add(ex9(a) > 0 ? d[a] : -d[a]);
            sx.l += ex9(a) > 0 ? dl[a] : -dl[a];
        }
        if (ey9(a) != 0) {
            sy.add(ey9(a) > 0 ? d[a] : -d[a]);
            sy.l += ey9(a) > 0 ? dl[a] : -dl[a];
        }
    }
    float er, ejx, ejy;
    const float rh = two_sum(p.rho0, r.h, er);
    const float rl = __fadd_rn(er, r.l);
    const float jxh = two_sum(sx.h, p.half_inv_gamma * Fx, ejx);
    const float jyh = two_sum(sy.h, p.half_inv_gamma * Fy, ejy);
    const float jxl = ejx + sx.l, jyl = ejy + sy.l;
    const float ri = 1.f / rh;
    const float uxh = jxh * ri, uyh = jyh * ri;
    const float uxl = (fmaf(-uxh, rh, jxh) + jxl - uxh * rl) * ri;
    const float uyl = (fmaf(-uyh, rh, jyh) + jyl - uyh * rl) * ri;
    if (have_snap) {
        const float dx = (uxh - us[0]) + (uxl - us[2]);
        const float dy = (uyh - us[1]) + (uyl - us[3]);
        acc[0] += dx * dx + dy * dy;
    }
    acc[1] += uxh * uxh + uyh * uyh;
    acc[2] += r.h + r.l;
    acc[3] += jxh + jxl;
    acc[4] += jyh + jyl;
    acc[6] += (isfinite(uxh) && isfinite(uyh)) ? 0.f : 1.f;
    us[0] = uxh;
    us[1] = uyh;
    us[2] = uxl;
    us[3] = uyl;
}

// Block sums of the residual terms into partials[k][block] (FP32 within the
// block of at most 512 nodes, FP64 from the partials on).
__device__ __forceinline__ void block_partials2(const float (&acc)[7], double* partials)
{
    __shared__ float sh[T2D / 32][7];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const float v = warp_sum2(acc[k]);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < T2D / 32; ++w) s += sh[w][threadIdx.x];
        partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = (double)s;
    }
}

// L2 prefetch of the rows that block blockIdx.x + b.pf_ahead will gather
// (its T2D nodes shifted by each direction's offset, one node of halo),
// one bulk prefetch per row by the first threads of the block: f (and the
// compensated low rows), g, the lagged Lorentz force, the force field and,
// on residual levels, the snapshot.
template <int ST, bool MHD, bool RESID>
__device__ __forceinline__ void prefetch2d(const P2& p, const B2& b)
{
    using S = Sto2<ST>;
    constexpr int NF = 9, NG = MHD ? 10 : 0, NC = S::COMP ? NF + NG : 0, NL = MHD ? 2 : 0, NS = RESID ? 4 : 0;
    const int t = threadIdx.x;
    if (b.pf_ahead <= 0 || t >= NF + NG + NC + NL + 2 + NS) return;
    const long long N = p.N;
    const long long nb = ((long long)blockIdx.x + b.pf_ahead) * T2D;
    if (nb >= N) return;
    uintptr_t row;
    size_t esz;
    long long shift = 0, halo = 0;
    int r = t;
    if (r < NF + NG) {                       // f then g rows, in the storage type
        const int a = r < NF ? r : (r - NF) % 5;
        const long long off = r < NF ? ex9(a) + (long long)ey9(a) * p.nx : ex5(a) + (long long)ey5(a) * p.nx;
        row = reinterpret_cast<uintptr_t>(r < NF ? b.fsrc : b.gsrc) +
              (uintptr_t)(r < NF ? r : r - NF) * (uintptr_t)N * sizeof(typename S::T);
        esz = sizeof(typename S::T);
        shift = -off;
        halo = 1;
    } else if ((r -= NF + NG) < NC) {        // the compensated low rows
        const int rr = r < NF ? r : r - NF;
        const int a = r < NF ? r : rr % 5;
        const long long off = r < NF ? ex9(a) + (long long)ey9(a) * p.nx : ex5(a) + (long long)ey5(a) * p.nx;
        row = reinterpret_cast<uintptr_t>(r < NF ? b.fsrc : b.gsrc) +
              (uintptr_t)(r < NF ? NF : 10) * (uintptr_t)N * sizeof(float) + (uintptr_t)rr * (uintptr_t)N * sizeof(__half);
        esz = sizeof(__half);
        shift = -off;
        halo = 1;
    } else if ((r -= NC) < NL) {
        row = reinterpret_cast<uintptr_t>(b.FL) + (uintptr_t)r * (uintptr_t)N * sizeof(float);
        esz = sizeof(float);
    } else if ((r -= NL) < 2) {
        if (b.Ffield == nullptr) return;
        row = reinterpret_cast<uintptr_t>(b.Ffield) + (uintptr_t)r * (uintptr_t)N * sizeof(float);
        esz = sizeof(float);
    } else {
        r -= 2;
        row = reinterpret_cast<uintptr_t>(b.usnap) + (uintptr_t)r * (uintptr_t)N * sizeof(float);
        esz = sizeof(float);
    }
    const long long s0 = nb + shift - halo, s1 = nb + T2D + shift + halo;
    uintptr_t lo = row + (uintptr_t)(s0 < 0 ? 0 : s0) * esz;
    uintptr_t hi = row + (uintptr_t)(s1 > N ? N : s1) * esz;
    lo = (lo + 15) & ~(uintptr_t)15;
    hi &= ~(uintptr_t)15;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)(hi - lo)) : "memory");
}

// One node per thread: any geometry.
template <int ST, bool MHD, int MODE>
__device__ __forceinline__ void step2d_body(const P2& p, const B2& b, const Out2& o)
{
    if (b.stop && *b.stop) return;   // the march converged in an earlier launch of this chunk
    if constexpr (MODE != M2_FIELDS) prefetch2d<ST, MHD, MODE == M2_RESID>(p, b);
    const int n = blockIdx.x * T2D + threadIdx.x;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (n < p.N) {
        const int y = row_of(p, n), x = n - y * p.nx;
        if (MODE == M2_FIELDS && is_solid(p, x, y)) {
            // solid nodes: zero in every output
            if (o.rho) o.rho[n] = 0.f;
            if (o.u) o.u[n] = o.u[p.N + n] = 0.f;
            if (MHD && o.B) o.B[n] = o.B[p.N + n] = 0.f;
        } else if (!is_solid(p, x, y)) {
            // the residual snapshot is read before the node's stores: a load
            // after them waits for them (the stores may alias it)
            float us[4] = {0.f, 0.f, 0.f, 0.f};
            if (MODE == M2_RESID && b.have_snap) {
                us[0] = b.usnap[n];
                us[1] = b.usnap[p.N + n];
                us[2] = b.usnap[2 * (size_t)p.N + n];
                us[3] = b.usnap[3 * (size_t)p.N + n];
            }
            float d[9], dl[9], q[10], ql[10];
            if (x >= p.ix0 && x <= p.ix1 && y >= p.iy0 && y <= p.iy1) {
                gather_f_interior<ST>(p, n, b.fsrc, d, dl);
                if (MHD) gather_g_interior<ST>(p, n, b.gsrc, q, ql);
            } else {
                const Nb nb = neighbours(p, x, y);
                gather_f<ST>(p, nb, x, y, n, b.fsrc, d, dl);
                if (MHD) gather_g<ST>(p, nb, x, y, n, b.gsrc, q, ql);
            }
            float Fex = p.Fx, Fey = p.Fy;
            if (b.Ffield) {
                Fex += __ldg(b.Ffield + n);
                Fey += __ldg(b.Ffield + p.N + n);
            }
            const float FLpx = MHD ? b.FL[n] : 0.f, FLpy = MHD ? b.FL[p.N + n] : 0.f;
            Node2 nd;
            float Fx, Fy, om[9], og[10];
            if constexpr (ST == GLBE_BF16) {
                Node2V<float> v;
                node_update2v<float, MHD, MODE != M2_FIELDS>(p, d, q, Fex, Fey, FLpx, FLpy, v, Fx, Fy, om, og);
                nd = Node2{v.rho, v.jx, v.jy, v.ux, v.uy, v.Bx, v.By, v.FLx, v.FLy};
            } else {
                node_update2<ST, MHD, MODE != M2_FIELDS>(p, d, dl, q, ql, Fex, Fey, FLpx, FLpy, nd, Fx, Fy, om, og);
            }
            if constexpr (MODE == M2_FIELDS) {
                if (o.rho) o.rho[n] = nd.rho;
                if (o.u) {
                    o.u[n] = nd.ux;
                    o.u[p.N + n] = nd.uy;
                }
                if (MHD && o.B) {
                    o.B[n] = nd.Bx;
                    o.B[p.N + n] = nd.By;
                }
            } else {
                const size_t N = p.N;
#pragma unroll
                for (int a = 0; a < 9; ++a) put<ST>(b.fdst, N, 9, (size_t)a * N + n, d[a], dl[a], om[a]);
                if (MHD) {
#pragma unroll
                    for (int i = 0; i < 10; ++i) put<ST>(b.gdst, N, 10, (size_t)i * N + n, q[i], ql[i], og[i]);
                    b.FL[n] = nd.FLx;
                    b.FL[N + n] = nd.FLy;
                }
                if constexpr (MODE == M2_RESID) {
                    resid_node(p, d, dl, Fx, Fy, b.have_snap, us, acc);
                    b.usnap[n] = us[0];
                    b.usnap[N + n] = us[1];
                    b.usnap[2 * N + n] = us[2];
                    b.usnap[3 * N + n] = us[3];
                }
            }
        }
    }
    if constexpr (MODE == M2_RESID) block_partials2(acc, b.partials);
}

template <int ST, bool MHD, int MODE>
__global__ void __launch_bounds__(T2D) step2d_kernel(const P2 p, const B2 b, const Out2 o)
{
    step2d_body<ST, MHD, MODE>(p, b, o);
}

// The plain step held to MINB resident blocks of 256 per SM (measured on the
// 4096^2 channel against the free allocation): F32 coupled 4 (64 registers,
// 36 B spilled; 0.86 against 0.78 of HBM), F32 flow 6 (40 registers, 20 B;
// 0.80 against 0.78), F32C coupled 3 (80 registers, 64 B; 0.80 against
// 0.70), F32C flow 5 (48 registers, 24 B; 0.77 against 0.76), BF16 flow 8
// (32 registers, 16 B; 0.55 against 0.52).  BF16 coupled stays free (held to
// 5 blocks it measured the same).  A kernel of its own: stating a minimum
// changes the register allocation of the forms left free.
template <int ST, bool MHD, int MINB>
__global__ void __launch_bounds__(T2D, MINB) step2d_kernel_dense(const P2 p, const B2 b, const Out2 o)
{
    step2d_body<ST, MHD, M2_STEP>(p, b, o);
}
// The coupled F32 residual step held likewise (4 blocks: 64 registers, 52 B
// spilled).
template <int ST, int MINB>
__global__ void __launch_bounds__(T2D, MINB) step2d_kernel_dense_resid(const P2 p, const B2 b, const Out2 o)
{
    step2d_body<ST, true, M2_RESID>(p, b, o);
}
template <int ST, bool MHD>
constexpr int dense2d_blocks()
{
    return ST == GLBE_F32 ? (MHD ? 4 : 6) : (ST == GLBE_BF16 ? (MHD ? 0 : 8) : (MHD ? 3 : 5));
}

// Two x-adjacent nodes per thread (x periodic, even nx; FP32 or BF16
// storage): the thread of pair (x0, x0 + 1) loads direction a's source row
// as the aligned pair at x0 (a vector load) and forms the x-shifted sources
// with one lane shuffle of the neighbouring pair; the lanes at a warp edge or
// at the x seam load the missing value themselves.  A wall row bounces both
// nodes back from their own pair of the opposite direction.  Every step is
// the one-node kernel's arithmetic, node by node, bit for bit.
template <int ST> struct Pair2;
template <> struct Pair2<GLBE_F32> {
    static __device__ __forceinline__ float2 ld(const void* base, size_t k)
    {
        return __ldg(reinterpret_cast<const float2*>(static_cast<const float*>(base) + k));
    }
    static __device__ __forceinline__ float ld1(const void* base, size_t k)
    {
        return ld256(static_cast<const float*>(base) + k);
    }
    static __device__ __forceinline__ void st(void* base, size_t k, float a, float b)
    {
        *reinterpret_cast<float2*>(static_cast<float*>(base) + k) = make_float2(a, b);
    }
};
template <> struct Pair2<GLBE_BF16> {
    // a BF16 value is the high half of the FP32 with the same bits: the pair
    // is widened from one 32-bit load by a shift and a mask (exact)
    static __device__ __forceinline__ float2 ld(const void* base, size_t k)
    {
        uint32_t u;
        asm("ld.global.nc.L2::256B.b32 %0, [%1];"
            : "=r"(u)
            : "l"(static_cast<const __nv_bfloat16*>(base) + k));
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
    static __device__ __forceinline__ float ld1(const void* base, size_t k)
    {
        return __uint_as_float((unsigned)ld256(reinterpret_cast<const unsigned short*>(
                                   static_cast<const __nv_bfloat16*>(base) + k)) << 16);
    }
    static __device__ __forceinline__ void st(void* base, size_t k, float a, float b)
    {
        *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(base) + k) = __floats2bfloat162_rn(a, b);
    }
};

// Gathers the pair's values of the populations rows[0..R) (direction a_r of
// the lattice EXR/EYR; bounced from row opp_r; sign of the bounce +1 for f,
// -1 for g) in two phases, so that every load of a step -- f and g -- is
// issued before the first lane shuffle waits for one: pair_loads issues the
// aligned pairs and, at a warp edge or the x seam, the lane's own value;
// pair_shuffles forms the x-shifted sources.
template <int R>
struct PairGather {
    float2 P[R];
    float E[R];
    bool bounce[R];
};
template <int ST, int R, class DIR>
__device__ __forceinline__ void pair_loads(const P2& p, const void* buf, bool live, int y, int x0, int n0, int lane,
                                           PairGather<R>& G)
{
    const size_t N = p.N;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ex = DIR::ex(r), ey = DIR::ey(r);
        int ys = y - ey;
        if (ey != 0) ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
        G.bounce[r] = ey != 0 && ((p.wly && ys == 0) || (p.why && ys == p.ny - 1));
        const size_t rb = (size_t)DIR::row(r) * N + (size_t)ys * p.nx;
        const bool edge = ex == 1 ? (lane == 0 || x0 == 0) : (ex == -1 ? (lane == 31 || x0 + 2 == p.nx) : false);
        const int xe = ex == 1 ? (x0 == 0 ? p.nx - 1 : x0 - 1) : (x0 + 2 == p.nx ? 0 : x0 + 2);
        G.P[r] = make_float2(0.f, 0.f);
        G.E[r] = 0.f;
        if (live) {
            G.P[r] = Pair2<ST>::ld(buf, G.bounce[r] ? (size_t)DIR::opp(r) * N + n0 : rb + x0);
            if (ex != 0 && edge && !G.bounce[r]) G.E[r] = Pair2<ST>::ld1(buf, rb + xe);
        }
    }
}
template <int R, class DIR>
__device__ __forceinline__ void pair_shuffles(const P2& p, int x0, int lane, float sign, const PairGather<R>& G,
                                              float (&v0)[R], float (&v1)[R])
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int ex = DIR::ex(r);
        // every lane takes part in the shuffles (uniform control flow)
        float sh = 0.f;
        if (ex == 1) sh = __shfl_up_sync(0xffffffffu, G.P[r].y, 1);
        if (ex == -1) sh = __shfl_down_sync(0xffffffffu, G.P[r].x, 1);
        const bool edge = ex == 1 ? (lane == 0 || x0 == 0) : (ex == -1 ? (lane == 31 || x0 + 2 == p.nx) : false);
        if (edge) sh = G.E[r];
        if (ex == 0 || G.bounce[r]) {
            v0[r] = G.bounce[r] ? sign * G.P[r].x : G.P[r].x;
            v1[r] = G.bounce[r] ? sign * G.P[r].y : G.P[r].y;
        } else if (ex == 1) {                // sources x0 - 1 and x0
            v0[r] = sh;
            v1[r] = G.P[r].x;
        } else {                             // sources x0 + 1 and x0 + 2
            v0[r] = G.P[r].y;
            v1[r] = sh;
        }
    }
}

struct DirF {    // the 9 rows of f
    static __device__ __forceinline__ constexpr int ex(int r) { return ex9(r); }
    static __device__ __forceinline__ constexpr int ey(int r) { return ey9(r); }
    static __device__ __forceinline__ constexpr int row(int r) { return r; }
    static __device__ __forceinline__ constexpr int opp(int r) { return opp9t(r); }
};
struct DirG {    // the 10 rows of g: component j = r / 5, direction r % 5
    static __device__ __forceinline__ constexpr int ex(int r) { return ex5(r % 5); }
    static __device__ __forceinline__ constexpr int ey(int r) { return ey5(r % 5); }
    static __device__ __forceinline__ constexpr int row(int r) { return r; }
    static __device__ __forceinline__ constexpr int opp(int r) { return (r / 5) * 5 + opp5(r % 5); }
};

template <int ST, bool MHD, int MODE>
__global__ void __launch_bounds__(T2D) step2d_pair_kernel(const P2 p, const B2 b)
{
    if (b.stop && *b.stop) return;
    const int lane = threadIdx.x & 31;
    const int n0 = 2 * (blockIdx.x * T2D + threadIdx.x);
    const size_t N = p.N;
    int y = 0, x0 = 0;
    if (n0 < p.N) {
        y = row_of(p, n0);
        x0 = n0 - y * p.nx;
    }
    // a wall row, or past the last pair: no loads, no update (but the lanes
    // take part in the shuffles)
    const bool live = n0 < p.N && !((p.wly && y == 0) || (p.why && y == p.ny - 1));
    float d0[9], d1[9], q0[10], q1[10];
    PairGather<9> gf;
    PairGather<10> gg;
    pair_loads<ST, 9, DirF>(p, b.fsrc, live, y, x0, n0, lane, gf);
    if (MHD) pair_loads<ST, 10, DirG>(p, b.gsrc, live, y, x0, n0, lane, gg);
    pair_shuffles<9, DirF>(p, x0, lane, 1.f, gf, d0, d1);
    if (MHD) pair_shuffles<10, DirG>(p, x0, lane, -1.f, gg, q0, q1);
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float us0[4] = {0.f, 0.f, 0.f, 0.f}, us1[4] = {0.f, 0.f, 0.f, 0.f};
    if (MODE == M2_RESID && live && b.have_snap) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 v = *reinterpret_cast<const float2*>(b.usnap + k * N + n0);
            us0[k] = v.x;
            us1[k] = v.y;
        }
    }
    if (live) {
        float2 Fe = make_float2(p.Fx, p.Fy), Fe1 = Fe;
        if (b.Ffield) {
            const float2 fx = *reinterpret_cast<const float2*>(b.Ffield + n0);
            const float2 fy = *reinterpret_cast<const float2*>(b.Ffield + N + n0);
            Fe = make_float2(p.Fx + fx.x, p.Fy + fy.x);
            Fe1 = make_float2(p.Fx + fx.y, p.Fy + fy.y);
        }
        float2 FLx = make_float2(0.f, 0.f), FLy = FLx;
        if (MHD) {
            FLx = *reinterpret_cast<const float2*>(b.FL + n0);
            FLy = *reinterpret_cast<const float2*>(b.FL + N + n0);
        }
        const float z9[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const float z10[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float F0x, F0y, F1x, F1y;
        if constexpr (ST == GLBE_BF16) {
            // both nodes in packed FP32x2 instructions
            V2 dv[9], qv[10], om[9], og[10], Fx, Fy;
#pragma unroll
            for (int a = 0; a < 9; ++a) dv[a] = V2(d0[a], d1[a]);
            if (MHD) {
#pragma unroll
                for (int i = 0; i < 10; ++i) qv[i] = V2(q0[i], q1[i]);
            }
            Node2V<V2> nd;
            node_update2v<V2, MHD, true>(p, dv, qv, V2(Fe.x, Fe1.x), V2(Fe.y, Fe1.y), V2(FLx.x, FLx.y),
                                         V2(FLy.x, FLy.y), nd, Fx, Fy, om, og);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                const V2 v = vadd(dv[a], om[a]);
                Pair2<ST>::st(b.fdst, (size_t)a * N + n0, v.v.x, v.v.y);
            }
            if (MHD) {
#pragma unroll
                for (int i = 0; i < 10; ++i) {
                    const V2 v = vadd(qv[i], og[i]);
                    Pair2<ST>::st(b.gdst, (size_t)i * N + n0, v.v.x, v.v.y);
                }
                *reinterpret_cast<float2*>(b.FL + n0) = nd.FLx.v;
                *reinterpret_cast<float2*>(b.FL + N + n0) = nd.FLy.v;
            }
            F0x = Fx.v.x;
            F1x = Fx.v.y;
            F0y = Fy.v.x;
            F1y = Fy.v.y;
        } else {
            Node2 nd0, nd1;
            float om0[9], og0[10], om1[9], og1[10];
            node_update2<ST, MHD, true>(p, d0, z9, q0, z10, Fe.x, Fe.y, FLx.x, FLy.x, nd0, F0x, F0y, om0, og0);
            node_update2<ST, MHD, true>(p, d1, z9, q1, z10, Fe1.x, Fe1.y, FLx.y, FLy.y, nd1, F1x, F1y, om1, og1);
#pragma unroll
            for (int a = 0; a < 9; ++a) Pair2<ST>::st(b.fdst, (size_t)a * N + n0, d0[a] + om0[a], d1[a] + om1[a]);
            if (MHD) {
#pragma unroll
                for (int i = 0; i < 10; ++i) Pair2<ST>::st(b.gdst, (size_t)i * N + n0, q0[i] + og0[i], q1[i] + og1[i]);
                *reinterpret_cast<float2*>(b.FL + n0) = make_float2(nd0.FLx, nd1.FLx);
                *reinterpret_cast<float2*>(b.FL + N + n0) = make_float2(nd0.FLy, nd1.FLy);
            }
        }
        if constexpr (MODE == M2_RESID) {
            resid_node(p, d0, z9, F0x, F0y, b.have_snap, us0, acc);
            resid_node(p, d1, z9, F1x, F1y, b.have_snap, us1, acc);
#pragma unroll
            for (int k = 0; k < 4; ++k) *reinterpret_cast<float2*>(b.usnap + k * N + n0) = make_float2(us0[k], us1[k]);
        }
    }
    if constexpr (MODE == M2_RESID) block_partials2(acc, b.partials);
}

// Pre-collision deviations of the current state (the gather of a step).
template <int ST, bool MHD>
__global__ void __launch_bounds__(T2D) get_state2d_kernel(const P2 p, const void* fsrc, const void* gsrc,
                                                           const float* FL, float* df, float* dg, float* dFL)
{
    const int n = blockIdx.x * T2D + threadIdx.x;
    if (n >= p.N) return;
    const int y = n / p.nx, x = n - y * p.nx;
    const size_t N = p.N;
    if (is_solid(p, x, y)) {
        if (df)
            for (int a = 0; a < 9; ++a) df[a * N + n] = 0.f;
        if (MHD && dg)
            for (int i = 0; i < 10; ++i) dg[i * N + n] = 0.f;
        if (MHD && dFL) dFL[n] = dFL[N + n] = 0.f;
        return;
    }
    const Nb nb = neighbours(p, x, y);
    if (df) {
        float d[9], dl[9];
        gather_f<ST>(p, nb, x, y, n, fsrc, d, dl);
        for (int a = 0; a < 9; ++a) df[a * N + n] = d[a] + dl[a];
    }
    if (MHD && dg) {
        float q[10], ql[10];
        gather_g<ST>(p, nb, x, y, n, gsrc, q, ql);
        for (int i = 0; i < 10; ++i) dg[i * N + n] = q[i] + ql[i];
    }
    if (MHD && dFL) {
        dFL[n] = FL[n];
        dFL[N + n] = FL[N + n];
    }
}

// Inverse of the gather: writes the given pre-collision deviations into the
// slots the next step reads (every slot of a fluid node is read exactly once:
// from downstream, or bounced back into the node itself).
template <int ST>
__device__ __forceinline__ void put_raw(void* buf, size_t N, int rows, size_t k, float v)
{
    using S = Sto2<ST>;
    static_cast<typename S::T*>(buf)[k] = S::cv(v);
    if constexpr (S::COMP) reinterpret_cast<__half*>(static_cast<float*>(buf) + rows * N)[k] = __float2half_rn(0.f);
}

template <int ST, bool MHD>
__global__ void __launch_bounds__(T2D) set_state2d_kernel(const P2 p, void* fsrc, void* gsrc, float* FL,
                                                           const float* df, const float* dg, const float* dFL)
{
    const int n = blockIdx.x * T2D + threadIdx.x;
    if (n >= p.N) return;
    const int y = n / p.nx, x = n - y * p.nx;
    if (is_solid(p, x, y)) return;
    const size_t N = p.N;
    const Nb nb = neighbours(p, x, y);
    for (int a = 0; a < 9; ++a) {
        bool sol;
        const int s = source(p, nb, x, y, ex9(a), ey9(a), sol);
        const size_t k = sol ? (size_t)opp9t(a) * N + n : (size_t)a * N + s;
        put_raw<ST>(fsrc, N, 9, k, df[a * N + n]);
    }
    if (MHD && dg) {
        for (int a = 0; a < 5; ++a) {
            bool sol;
            const int s = source(p, nb, x, y, ex5(a), ey5(a), sol);
            for (int j = 0; j < 2; ++j) {
                const float v = dg[(j * 5 + a) * N + n];
                const size_t k = sol ? (size_t)(j * 5 + opp5(a)) * N + n : (size_t)(j * 5 + a) * N + s;
                put_raw<ST>(gsrc, N, 10, k, sol ? -v : v);
            }
        }
    }
    if (MHD && dFL) {
        FL[n] = dFL[n];
        FL[N + n] = dFL[N + n];
    }
}

__global__ void ctl2d_kernel(long long* t_dev, long long t, int* stop, int stop_v, double* tol, double tol_v,
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

glbe_status cuda_fail2(cudaError_t e, const char* what)
{
    return fail(GLBE_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define GLBE2D_CUDA(call, what)                              \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail2(e_, what);  \
    } while (0)

size_t value_bytes(int st) { return st == GLBE_F32 ? 4 : (st == GLBE_F32C ? 6 : 2); }

struct Layout2 {
    size_t f[2], g[2], FL, Ffield, usnap, partials, record, hist, misc, total;
};

unsigned blocks_of(size_t N) { return (unsigned)((N + T2D - 1) / T2D); }

Layout2 layout2(const glbe2d_params* p)
{
    const size_t N = (size_t)p->nx * p->ny;
    const size_t vb = value_bytes(p->storage);
    Layout2 L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align2(bytes);
        return at;
    };
    L.f[0] = take(9 * N * vb);
    L.f[1] = take(9 * N * vb);
    if (p->induction) {
        L.g[0] = take(10 * N * vb);
        L.g[1] = take(10 * N * vb);
        L.FL = take(2 * N * sizeof(float));
    }
    if (p->force_field) L.Ffield = take(2 * N * sizeof(float));
    L.usnap = take(4 * N * sizeof(float));
    L.partials = take((size_t)PARTIAL_STRIDE * blocks_of(N) * sizeof(double));
    L.record = take(RECORD_STRIDE * sizeof(double));
    L.hist = take((size_t)HIST_CAP2 * RECORD_STRIDE * sizeof(double));
    L.misc = take(64);   // t_dev, hist_count, tol, stop
    L.total = o;
    return L;
}

glbe_status validate2(const glbe2d_params* p)
{
    if (!p) return fail(GLBE_ERR_ARG, "params is NULL");
    if (p->nx < 1 || p->ny < 1) return fail(GLBE_ERR_ARG, "grid must be at least 1 x 1");
    if ((long long)p->nx * p->ny >= (1LL << 31)) return fail(GLBE_ERR_ARG, "grid too large (N >= 2^31)");
    const int n[2] = {p->nx, p->ny};
    for (int d = 0; d < 2; ++d) {
        if ((p->wall_lo[d] != 0 && p->wall_lo[d] != 1) || (p->wall_hi[d] != 0 && p->wall_hi[d] != 1))
            return fail(GLBE_ERR_ARG, "wall flags must be 0 or 1");
        if (n[d] - p->wall_lo[d] - p->wall_hi[d] < 1) return fail(GLBE_ERR_ARG, "walls leave no fluid line");
    }
    if (!(p->gamma > 0.0 && p->gamma <= 1.0)) return fail(GLBE_ERR_ARG, "gamma must be in (0, 1]");
    if (!(p->nu > 0.0)) return fail(GLBE_ERR_ARG, "nu must be > 0");
    if (!(p->rho0 > 0.0)) return fail(GLBE_ERR_ARG, "rho0 must be > 0");
    for (int k = 0; k < 9; ++k)
        if (!(p->s[k] > 0.0 && p->s[k] < 2.0)) return fail(GLBE_ERR_ARG, "rate s[%d] must be in (0, 2)", k);
    if (p->storage != GLBE_F32 && p->storage != GLBE_BF16 && p->storage != GLBE_F32C)
        return fail(GLBE_ERR_ARG, "storage must be GLBE_F32, GLBE_BF16 or GLBE_F32C");
    if (p->force_field != 0 && p->force_field != 2) return fail(GLBE_ERR_ARG, "force_field must be 0 or 2");
    if (p->induction != 0 && p->induction != 1) return fail(GLBE_ERR_ARG, "induction must be 0 or 1");
    if (p->variant < 0 || p->variant > 2) return fail(GLBE_ERR_ARG, "variant must be 0, 1 or 2");
    if (p->induction) {
        if (!(p->gamma_m > 0.0 && p->gamma_m <= 1.0)) return fail(GLBE_ERR_ARG, "gamma_m must be in (0, 1]");
        if (!(p->eta > 0.0) || !(p->chi > 0.0) || !(p->mu > 0.0))
            return fail(GLBE_ERR_ARG, "eta, chi and mu must be > 0");
    }
    return GLBE_OK;
}

P2 make_p2(const glbe2d_params* p)
{
    P2 q{};
    q.nx = p->nx;
    q.ny = p->ny;
    q.N = p->nx * p->ny;
    q.wlx = p->wall_lo[0];
    q.whx = p->wall_hi[0];
    q.wly = p->wall_lo[1];
    q.why = p->wall_hi[1];
    const FastDiv fd = make_fastdiv((uint32_t)p->nx);
    q.div_m = fd.m;
    q.div_s = fd.s;
    q.ix0 = 1 + p->wall_lo[0];
    q.ix1 = p->nx - 2 - p->wall_hi[0];
    q.iy0 = 1 + p->wall_lo[1];
    q.iy1 = p->ny - 2 - p->wall_hi[1];
    q.rho0 = (float)p->rho0;
    // s_7 = s_8 = s_nu*, 1/s_nu* = 3 nu/gamma + 1/2 (Sec. 3); source rows
    // S*_k = P_S,k R_k c_k (App. A table, Eq. precondsourceterm)
    const double g = p->gamma, ig = 1.0 / g, ig2 = ig * ig;
    const double snu = 1.0 / (3.0 * p->nu / g + 0.5);
    const double sk[9] = {0.0, p->s[1], p->s[2], 0.0, p->s[4], 0.0, p->s[6], snu, snu};
    auto fold = [&](int k, double norm, double src, float& a, float& b) {
        a = (float)(-sk[k] / norm);
        b = (float)((1.0 - 0.5 * sk[k]) * src / norm);
    };
    fold(1, 36.0, 6.0 * ig2, q.a1, q.b1);
    fold(2, 36.0, -6.0 * ig2, q.a2, q.b2);
    fold(4, 12.0, -ig, q.a4, q.b4);
    fold(6, 12.0, -ig, q.a6, q.b6);
    fold(7, 4.0, 2.0 * ig2, q.a7, q.b7);
    fold(8, 4.0, ig2, q.a8, q.b8);
    q.c3 = (float)(ig / 6.0);
    q.inv_gamma = (float)ig;
    q.half_inv_gamma = (float)(0.5 * ig);
    q.Fx = (float)p->F[0];
    q.Fy = (float)p->F[1];
    if (p->induction) {
        const double theta = 1.0 / 3.0;   // theta_m = 1/N_m, N_m = 3 (Sec. 4)
        const double tau = p->eta / (p->gamma_m * theta) + 0.5;
        q.inv_tau_m = (float)(1.0 / tau);
        q.ceq = (float)(p->chi / (p->gamma_m * theta));
        q.cJ = (float)(1.0 / (p->mu * p->chi * tau * theta));
        q.B0x = (float)p->B0[0];
        q.B0y = (float)p->B0[1];
    }
    return q;
}

}  // namespace

struct glbe2d_ctx {
    glbe2d_params prm;
    P2 p;
    Layout2 L;
    size_t N;
    unsigned blocks;
    int pair;              // the two-node kernel takes the plain and residual steps
    unsigned pair_blocks;  // its grid (the residual partials use the larger one-node grid's rows)
    char* ws;
    void* f[2];
    void* g[2];
    float* FL;
    float* Ffield;
    float* usnap;
    double* partials;
    double* record;
    double* hist;
    long long* t_dev;
    unsigned long long* hist_count;
    double* tol_dev;
    int* stop_dev;
    double mass0;
    long t;
    long t_snap;
    cudaStream_t stream;
    cudaStream_t cap_stream;
    cudaGraphExec_t chunk;
};

namespace {

// Blocks of a kernel resident on the whole GPU at once (one wave).
template <class K>
long long wave2d(K kernel)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, T2D, 0);
    return (long long)sms * per;
}

// The launch's L2 prefetch distance: half a wave ahead on grids of several
// waves, none on small grids.  Taken by the coupled F32 step only: measured
// on the 4096^2 channel it took that plain step from 0.4829 to 0.4337 ms
// (0.86 -> 0.96 of HBM) but slowed every other form (F32C coupled 0.753 ->
// 0.792 ms, BF16 coupled 0.336 -> 0.356, F32C flow 0.346 -> 0.353, BF16
// flow 0.162 -> 0.174; F32 flow unchanged).
template <int ST, bool MHD, class K>
int prefetch_distance(K kernel, unsigned grid)
{
    if constexpr (ST != GLBE_F32 || !MHD) return 0;
    static const long long w = wave2d(kernel);
    return (long long)grid > 4 * w ? (int)(w / 2) : 0;
}

template <int ST>
cudaError_t launch2_t(glbe2d_ctx* c, int mode, const B2& b_in, const Out2& o, cudaStream_t st)
{
    const bool mhd = c->prm.induction;
    const unsigned nb = c->blocks;
    B2 b = b_in;
    if constexpr (ST == GLBE_F32 || ST == GLBE_BF16) {
        if (c->pair && mode != M2_FIELDS) {
            const unsigned pb = c->pair_blocks;
            if (mode == M2_STEP) {
                if (mhd) step2d_pair_kernel<ST, true, M2_STEP><<<pb, T2D, 0, st>>>(c->p, b);
                else step2d_pair_kernel<ST, false, M2_STEP><<<pb, T2D, 0, st>>>(c->p, b);
            } else {
                if (mhd) step2d_pair_kernel<ST, true, M2_RESID><<<pb, T2D, 0, st>>>(c->p, b);
                else step2d_pair_kernel<ST, false, M2_RESID><<<pb, T2D, 0, st>>>(c->p, b);
            }
            return cudaGetLastError();
        }
    }
    if (mode == M2_STEP) {
        constexpr int MBM = dense2d_blocks<ST, true>(), MBF = dense2d_blocks<ST, false>();
        if (mhd) {
            if constexpr (MBM > 0) {
                if (c->prm.variant == 0) {
                    b.pf_ahead = prefetch_distance<ST, true>(step2d_kernel_dense<ST, true, MBM>, nb);
                    step2d_kernel_dense<ST, true, MBM><<<nb, T2D, 0, st>>>(c->p, b, o);
                    return cudaGetLastError();
                }
            }
            b.pf_ahead = prefetch_distance<ST, true>(step2d_kernel<ST, true, M2_STEP>, nb);
            step2d_kernel<ST, true, M2_STEP><<<nb, T2D, 0, st>>>(c->p, b, o);
        } else {
            if constexpr (MBF > 0) {
                if (c->prm.variant == 0) {
                    b.pf_ahead = prefetch_distance<ST, false>(step2d_kernel_dense<ST, false, MBF>, nb);
                    step2d_kernel_dense<ST, false, MBF><<<nb, T2D, 0, st>>>(c->p, b, o);
                    return cudaGetLastError();
                }
            }
            b.pf_ahead = prefetch_distance<ST, false>(step2d_kernel<ST, false, M2_STEP>, nb);
            step2d_kernel<ST, false, M2_STEP><<<nb, T2D, 0, st>>>(c->p, b, o);
        }
    } else if (mode == M2_RESID) {
        if (mhd) {
            if constexpr (ST == GLBE_F32) {
                if (c->prm.variant == 0) {
                    b.pf_ahead = prefetch_distance<ST, true>(step2d_kernel_dense_resid<ST, 4>, nb);
                    step2d_kernel_dense_resid<ST, 4><<<nb, T2D, 0, st>>>(c->p, b, o);
                    return cudaGetLastError();
                }
            }
            b.pf_ahead = prefetch_distance<ST, true>(step2d_kernel<ST, true, M2_RESID>, nb);
            step2d_kernel<ST, true, M2_RESID><<<nb, T2D, 0, st>>>(c->p, b, o);
        } else {
            b.pf_ahead = prefetch_distance<ST, false>(step2d_kernel<ST, false, M2_RESID>, nb);
            step2d_kernel<ST, false, M2_RESID><<<nb, T2D, 0, st>>>(c->p, b, o);
        }
    } else {
        if (mhd) step2d_kernel<ST, true, M2_FIELDS><<<nb, T2D, 0, st>>>(c->p, b, o);
        else step2d_kernel<ST, false, M2_FIELDS><<<nb, T2D, 0, st>>>(c->p, b, o);
    }
    return cudaGetLastError();
}

cudaError_t launch2(glbe2d_ctx* c, int mode, const B2& b, const Out2& o, cudaStream_t st)
{
    switch (c->prm.storage) {
    case GLBE_F32: return launch2_t<GLBE_F32>(c, mode, b, o, st);
    case GLBE_BF16: return launch2_t<GLBE_BF16>(c, mode, b, o, st);
    default: return launch2_t<GLBE_F32C>(c, mode, b, o, st);
    }
}

B2 buffers2(glbe2d_ctx* c, long t)
{
    B2 b{};
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
    return b;
}

glbe_status enqueue2(glbe2d_ctx* c, cudaStream_t st, const int* stop)
{
    B2 b = buffers2(c, c->t);
    b.stop = stop;
    const Out2 o{nullptr, nullptr, nullptr};
    if (c->t % 10 == 0) {
        b.have_snap = (c->t_snap >= 0 && c->t_snap == c->t - 10) ? 1 : 0;
        GLBE2D_CUDA(launch2(c, M2_RESID, b, o, st), "2D step kernel (residual)");
        if (b.have_snap) {
            GLBE2D_CUDA(launch_finalize(c->partials, c->pair ? c->pair_blocks : c->blocks, c->mass0, c->t_dev,
                                        c->record, c->hist, c->hist_count, HIST_CAP2, c->stop_dev, c->tol_dev, st),
                        "2D residual finalize");
        } else {
            ctl2d_kernel<<<1, 1, 0, st>>>(c->t_dev, (long long)c->t + 10, nullptr, 0, nullptr, 0.0, nullptr, nullptr, 0);
            GLBE2D_CUDA(cudaGetLastError(), "2D residual level");
        }
        c->t_snap = c->t;
    } else {
        GLBE2D_CUDA(launch2(c, M2_STEP, b, o, st), "2D step kernel");
    }
    c->t += 1;
    return GLBE_OK;
}

glbe_status read_record2(glbe2d_ctx* c, glbe_residual_info* out)
{
    double rec[RECORD_STRIDE];
    GLBE2D_CUDA(cudaStreamSynchronize(c->stream), "2D residual sync");
    GLBE2D_CUDA(cudaMemcpy(rec, c->record, sizeof rec, cudaMemcpyDeviceToHost), "2D residual read");
    out->t = (long)rec[0];
    out->r = rec[1];
    out->num = rec[2];
    out->den = rec[3];
    out->mass = rec[4];
    out->momentum[0] = rec[5];
    out->momentum[1] = rec[6];
    out->momentum[2] = 0.0;
    out->nonfinite = (int)rec[8];
    if (out->t >= 0 && (out->nonfinite > 0 || !std::isfinite(out->r)))
        return fail(GLBE_ERR_DIVERGED, "non-finite velocity at time level %ld", out->t);
    return GLBE_OK;
}

glbe_status build_chunk2(glbe2d_ctx* c)
{
    if (c->chunk) return GLBE_OK;
    if (!c->cap_stream) GLBE2D_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
    const long t_save = c->t, snap_save = c->t_snap;
    c->t = 10;
    c->t_snap = 0;
    GLBE2D_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    glbe_status s = GLBE_OK;
    for (int k = 0; k < 10 && s == GLBE_OK; ++k) s = enqueue2(c, c->cap_stream, c->stop_dev);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    c->t = t_save;
    c->t_snap = snap_save;
    if (s != GLBE_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail2(e, "end capture");
    const cudaError_t ei = cudaGraphInstantiate(&c->chunk, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        c->chunk = nullptr;
        return cuda_fail2(ei, "graph instantiate");
    }
    return GLBE_OK;
}

long long fluid2(const glbe2d_params* p)
{
    return (long long)(p->nx - p->wall_lo[0] - p->wall_hi[0]) * (p->ny - p->wall_lo[1] - p->wall_hi[1]);
}

}  // namespace

extern "C" {

void glbe2d_params_default(glbe2d_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->rho0 = 1.0;
    p->gamma = 1.0;
    for (int k = 0; k < 9; ++k) p->s[k] = 1.0;
    // kinetic rates of the D2Q9 model quoted in Sec. 3 (Lallemand and Luo)
    p->s[1] = 1.63;
    p->s[2] = 1.14;
    p->s[4] = p->s[6] = 1.92;
    p->gamma_m = 1.0;
    p->eta = 0.1;
    p->chi = 1.0;
    p->mu = 1.0;
    p->storage = GLBE_F32;
}

glbe_status glbe2d_workspace_bytes(const glbe2d_params* p, size_t* bytes)
{
    if (!bytes) return fail(GLBE_ERR_ARG, "bytes is NULL");
    const glbe_status s = validate2(p);
    if (s != GLBE_OK) return s;
    *bytes = layout2(p).total;
    return GLBE_OK;
}

glbe_status glbe2d_init(const glbe2d_params* p, void* d_workspace, size_t bytes, glbe2d_ctx** out)
{
    if (!out) return fail(GLBE_ERR_ARG, "out is NULL");
    *out = nullptr;
    glbe_status s = validate2(p);
    if (s != GLBE_OK) return s;
    if (!d_workspace) return fail(GLBE_ERR_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(d_workspace) % ALIGN2) return fail(GLBE_ERR_ARG, "workspace not 256-byte aligned");
    const Layout2 L = layout2(p);
    if (bytes < L.total) return fail(GLBE_ERR_ARG, "workspace too small: %zu < %zu", bytes, L.total);
    glbe2d_ctx* c = new glbe2d_ctx{};
    c->prm = *p;
    c->p = make_p2(p);
    c->L = L;
    c->N = (size_t)p->nx * p->ny;
    c->blocks = blocks_of(c->N);
    // the two-node form needs x periodic and an even nx, and F32 or BF16
    // storage; it is taken on request only (it measures no faster, and the
    // BF16 steps slower: more index arithmetic per node in an issue-bound step)
    c->pair = (p->variant == 2) && p->wall_lo[0] == 0 && p->wall_hi[0] == 0 && p->nx % 2 == 0 &&
              (p->storage == GLBE_F32 || p->storage == GLBE_BF16);
    c->pair_blocks = blocks_of(c->N / 2);
    c->ws = static_cast<char*>(d_workspace);
    c->f[0] = c->ws + L.f[0];
    c->f[1] = c->ws + L.f[1];
    c->g[0] = p->induction ? c->ws + L.g[0] : nullptr;
    c->g[1] = p->induction ? c->ws + L.g[1] : nullptr;
    c->FL = p->induction ? reinterpret_cast<float*>(c->ws + L.FL) : nullptr;
    c->Ffield = p->force_field ? reinterpret_cast<float*>(c->ws + L.Ffield) : nullptr;
    c->usnap = reinterpret_cast<float*>(c->ws + L.usnap);
    c->partials = reinterpret_cast<double*>(c->ws + L.partials);
    c->record = reinterpret_cast<double*>(c->ws + L.record);
    c->hist = reinterpret_cast<double*>(c->ws + L.hist);
    char* misc = c->ws + L.misc;
    c->t_dev = reinterpret_cast<long long*>(misc);
    c->hist_count = reinterpret_cast<unsigned long long*>(misc + 8);
    c->tol_dev = reinterpret_cast<double*>(misc + 16);
    c->stop_dev = reinterpret_cast<int*>(misc + 24);
    c->mass0 = p->rho0 * (double)fluid2(p);
    c->t = 0;
    c->t_snap = -1;
    c->stream = static_cast<cudaStream_t>(p->stream);
    // the rest state: every deviation, the Lorentz force and the field zero
    cudaError_t e = cudaMemsetAsync(d_workspace, 0, L.record, c->stream);
    if (e == cudaSuccess) {
        ctl2d_kernel<<<1, 1, 0, c->stream>>>(c->t_dev, 10, c->stop_dev, 0, c->tol_dev, 0.0, c->record, c->hist_count, 1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail2(e, "2D init");
    }
    *out = c;
    return GLBE_OK;
}

glbe_status glbe2d_set_force(glbe2d_ctx* c, const float* d_F)
{
    if (!c || !d_F) return fail(GLBE_ERR_ARG, "ctx or field is NULL");
    if (!c->Ffield) return fail(GLBE_ERR_STATE, "the context has no force field (force_field = 0)");
    GLBE2D_CUDA(cudaMemcpyAsync(c->Ffield, d_F, 2 * c->N * sizeof(float), cudaMemcpyDeviceToDevice, c->stream),
                "2D force copy");
    return GLBE_OK;
}

glbe_status glbe2d_step_n(glbe2d_ctx* c, long n)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    if (n < 0) return fail(GLBE_ERR_ARG, "n must be >= 0");
    for (long k = 0; k < n; ++k) {
        const glbe_status s = enqueue2(c, c->stream, nullptr);
        if (s != GLBE_OK) return s;
    }
    return GLBE_OK;
}

glbe_status glbe2d_residual(glbe2d_ctx* c, glbe_residual_info* out)
{
    if (!c || !out) return fail(GLBE_ERR_ARG, "ctx or out is NULL");
    return read_record2(c, out);
}

glbe_status glbe2d_history(glbe2d_ctx* c, glbe_residual_info* out, long cap, long* n)
{
    if (!c || !n || (cap > 0 && !out)) return fail(GLBE_ERR_ARG, "ctx, out or n is NULL");
    *n = 0;
    if (cap <= 0) return GLBE_OK;
    unsigned long long count = 0;
    GLBE2D_CUDA(cudaStreamSynchronize(c->stream), "2D history sync");
    GLBE2D_CUDA(cudaMemcpy(&count, c->hist_count, sizeof count, cudaMemcpyDeviceToHost), "2D history count");
    const unsigned long long kept = count < HIST_CAP2 ? count : HIST_CAP2;
    const unsigned long long take = kept < (unsigned long long)cap ? kept : (unsigned long long)cap;
    double rec[RECORD_STRIDE];
    for (unsigned long long i = 0; i < take; ++i) {
        const unsigned long long idx = (count - take + i) % HIST_CAP2;
        GLBE2D_CUDA(cudaMemcpy(rec, c->hist + idx * RECORD_STRIDE, sizeof rec, cudaMemcpyDeviceToHost),
                    "2D history read");
        glbe_residual_info& o = out[i];
        o.t = (long)rec[0];
        o.r = rec[1];
        o.num = rec[2];
        o.den = rec[3];
        o.mass = rec[4];
        o.momentum[0] = rec[5];
        o.momentum[1] = rec[6];
        o.momentum[2] = 0.0;
        o.nonfinite = (int)rec[8];
    }
    *n = (long)take;
    return GLBE_OK;
}

glbe_status glbe2d_solve(glbe2d_ctx* c, double tol, long max_steps, long* steps_out, double* r_out)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    if (!(tol > 0.0)) return fail(GLBE_ERR_ARG, "tol must be > 0");
    if (max_steps < 0) return fail(GLBE_ERR_ARG, "max_steps must be >= 0");
    const long t_end = c->t + max_steps;
    while (!(c->t % 10 == 0 && c->t_snap >= 0 && c->t_snap == c->t - 10) && c->t < t_end) {
        const glbe_status s = enqueue2(c, c->stream, nullptr);
        if (s != GLBE_OK) return s;
    }
    glbe_status s = build_chunk2(c);
    if (s != GLBE_OK) return s;
    ctl2d_kernel<<<1, 1, 0, c->stream>>>(nullptr, 0, c->stop_dev, 0, c->tol_dev, tol, nullptr, nullptr, 0);
    GLBE2D_CUDA(cudaGetLastError(), "2D solve setup");
    // chunks between host checks: about a millisecond of device work each
    long batch = (long)(4000000 / (c->N + 1));
    batch = batch < 4 ? 4 : (batch > 256 ? 256 : batch);
    int stop = 0;
    while (c->t + 10 <= t_end) {
        long nb = 0;
        for (; nb < batch && c->t + 10 * (nb + 1) <= t_end; ++nb)
            GLBE2D_CUDA(cudaGraphLaunch(c->chunk, c->stream), "2D graph launch");
        GLBE2D_CUDA(cudaStreamSynchronize(c->stream), "2D solve sync");
        GLBE2D_CUDA(cudaMemcpy(&stop, c->stop_dev, sizeof(int), cudaMemcpyDeviceToHost), "2D solve read");
        if (stop) {
            glbe_residual_info info;
            const glbe_status rs = read_record2(c, &info);
            c->t = info.t + 1;
            c->t_snap = info.t;
            if (steps_out) *steps_out = info.t;
            if (r_out) *r_out = info.r;
            ctl2d_kernel<<<1, 1, 0, c->stream>>>(nullptr, 0, c->stop_dev, 0, c->tol_dev, 0.0, nullptr, nullptr, 0);
            GLBE2D_CUDA(cudaGetLastError(), "2D solve reset");
            return rs;
        }
        c->t += 10 * nb;
        c->t_snap = c->t - 10;
    }
    while (c->t < t_end) {
        s = enqueue2(c, c->stream, nullptr);
        if (s != GLBE_OK) return s;
    }
    glbe_residual_info info;
    s = read_record2(c, &info);
    if (steps_out) *steps_out = c->t;
    if (r_out) *r_out = info.t >= 0 ? info.r : NAN;
    if (s != GLBE_OK) return s;
    if (info.t >= 0 && info.r <= tol) return GLBE_OK;
    return fail(GLBE_ERR_TIMEOUT, "residual %g > tol %g after %ld steps", info.r, tol, max_steps);
}

glbe_status glbe2d_fields(glbe2d_ctx* c, float* d_rho, float* d_u, float* d_B)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    const B2 b = buffers2(c, c->t);
    const Out2 o{d_rho, d_u, c->prm.induction ? d_B : nullptr};
    GLBE2D_CUDA(launch2(c, M2_FIELDS, b, o, c->stream), "2D fields kernel");
    return GLBE_OK;
}

glbe_status glbe2d_get_state(glbe2d_ctx* c, float* d_df, float* d_dg, float* d_FL)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    const int s = (int)(c->t & 1);
    const bool mhd = c->prm.induction;
    const unsigned nb = c->blocks;
    switch (c->prm.storage) {
    case GLBE_F32:
        if (mhd) get_state2d_kernel<GLBE_F32, true><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL);
        else get_state2d_kernel<GLBE_F32, false><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], nullptr, nullptr, d_df, nullptr, nullptr);
        break;
    case GLBE_BF16:
        if (mhd) get_state2d_kernel<GLBE_BF16, true><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL);
        else get_state2d_kernel<GLBE_BF16, false><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], nullptr, nullptr, d_df, nullptr, nullptr);
        break;
    default:
        if (mhd) get_state2d_kernel<GLBE_F32C, true><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL);
        else get_state2d_kernel<GLBE_F32C, false><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], nullptr, nullptr, d_df, nullptr, nullptr);
        break;
    }
    GLBE2D_CUDA(cudaGetLastError(), "2D get_state kernel");
    return GLBE_OK;
}

glbe_status glbe2d_set_state(glbe2d_ctx* c, const float* d_df, const float* d_dg, const float* d_FL, long t)
{
    if (!c || !d_df) return fail(GLBE_ERR_ARG, "ctx or df is NULL");
    if (t < 0) return fail(GLBE_ERR_ARG, "t must be >= 0");
    c->t = t;
    c->t_snap = -1;
    const int s = (int)(c->t & 1);
    const bool mhd = c->prm.induction;
    const unsigned nb = c->blocks;
    switch (c->prm.storage) {
    case GLBE_F32:
        if (mhd) set_state2d_kernel<GLBE_F32, true><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL);
        else set_state2d_kernel<GLBE_F32, false><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], nullptr, nullptr, d_df, nullptr, nullptr);
        break;
    case GLBE_BF16:
        if (mhd) set_state2d_kernel<GLBE_BF16, true><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL);
        else set_state2d_kernel<GLBE_BF16, false><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], nullptr, nullptr, d_df, nullptr, nullptr);
        break;
    default:
        if (mhd) set_state2d_kernel<GLBE_F32C, true><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], c->g[s], c->FL, d_df, d_dg, d_FL);
        else set_state2d_kernel<GLBE_F32C, false><<<nb, T2D, 0, c->stream>>>(c->p, c->f[s], nullptr, nullptr, d_df, nullptr, nullptr);
        break;
    }
    GLBE2D_CUDA(cudaGetLastError(), "2D set_state kernel");
    ctl2d_kernel<<<1, 1, 0, c->stream>>>(c->t_dev, ((long long)t + 9) / 10 * 10, c->stop_dev, 0, c->tol_dev, 0.0,
                                         c->record, c->hist_count, 1);
    GLBE2D_CUDA(cudaGetLastError(), "2D set_state reset");
    return GLBE_OK;
}

glbe_status glbe2d_time(const glbe2d_ctx* c, long* t)
{
    if (!c || !t) return fail(GLBE_ERR_ARG, "ctx or t is NULL");
    *t = c->t;
    return GLBE_OK;
}

glbe_status glbe2d_sync(glbe2d_ctx* c)
{
    if (!c) return fail(GLBE_ERR_ARG, "ctx is NULL");
    GLBE2D_CUDA(cudaStreamSynchronize(c->stream), "2D sync");
    GLBE2D_CUDA(cudaGetLastError(), "2D async error");
    return GLBE_OK;
}

void glbe2d_destroy(glbe2d_ctx* c)
{
    if (!c) return;
    if (c->chunk) cudaGraphExecDestroy(c->chunk);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

}  // extern "C"
