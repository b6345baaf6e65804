// glbe_kernels.cuh -- fused time step of the preconditioned GLBE (D3Q19 MRT
// with forcing) and the preconditioned D3Q7 vector kinetic equation for the
// magnetic induction, arXiv:0809.4730 Secs. 2-4 and App. A.
//
// One thread updates one node (pull scheme): it gathers the post-collision
// populations of the previous step from its upstream neighbours (half-way
// bounce-back for f, anti-bounce-back for g where the upstream node is solid),
// forms the macroscopic fields, collides in moment space and writes the new
// post-collision populations to its own slot of the other buffer.  Buffers
// hold deviations from the rest state (df = f - w rho0, dg = g - W B0) so that
// FP32, BF16 and FP16 storage keep the small part that changes.
//
// The moment transform is the integer Gram-Schmidt basis of App. A (rows
// rho, e, e^2, j, q, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz, m) applied
// through partial sums over the velocity groups; the inverse uses the
// orthogonality of the rows, T^-1 = T^t diag(1/|row_k|^2), with
// |row_k|^2 = 19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4,
// 8, 8, 8.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "glbe_internal.h"

namespace glbe {

// Storage of the population deviations.  COMP marks the compensated form:
// an FP32 high part plus an FP16 low part holding the rounding remainder
// (scaled by 2^36), updated with an exact two-sum so that corrections far
// below one FP32 ulp of the stored deviation accumulate instead of being
// dropped.  The low parts follow the high parts in the same buffer.
constexpr float LO_SCALE = 68719476736.0f;        // 2^36
constexpr float LO_INV = 1.4551915228366852e-11f; // 2^-36

template <int ST> struct Store;
template <> struct Store<ST_F32> {
    using T = float;
    static constexpr bool COMP = false;
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float cv(float v) { return v; }
};
template <> struct Store<ST_BF16> {
    using T = __nv_bfloat16;
    static constexpr bool COMP = false;
    static __device__ __forceinline__ float ld(const T* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ T cv(float v) { return __float2bfloat16_rn(v); }
};
template <> struct Store<ST_F16> {
    using T = __half;
    static constexpr bool COMP = false;
    static __device__ __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ T cv(float v) { return __float2half_rn(v); }
};
template <> struct Store<ST_F32C> {
    using T = float;
    static constexpr bool COMP = true;
    static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float cv(float v) { return v; }
    static __device__ __forceinline__ float ld_lo(const __half* p) { return __half2float(__ldg(p)) * LO_INV; }
    static __device__ __forceinline__ __half cv_lo(float v) { return __float2half_rn(v * LO_SCALE); }
};

// fl(a + b + c) for |c| small: the exact two-sum of a and b, its remainder
// plus c, rounded once.
__device__ __forceinline__ float two_sum_round(float a, float b, float c)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return __fadd_rn(s, __fadd_rn(e, c));
}

// h + o + l as a new (high, low) pair: exact two-sum of h and o, the
// remainder plus the old low part renormalised into the new low part.
__device__ __forceinline__ void comp_add(float h, float l, float o, float& nh, float& nl)
{
    const float s = __fadd_rn(h, o);
    const float bp = __fsub_rn(s, h);
    const float ap = __fsub_rn(s, bp);
    float e = __fadd_rn(__fsub_rn(h, ap), __fsub_rn(o, bp));
    e = __fadd_rn(e, l);
    nh = __fadd_rn(s, e);
    nl = __fsub_rn(e, __fsub_rn(nh, s));
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f)
{
    return (__umulhi(n, f.m) + n) >> f.s;
}

__device__ __forceinline__ bool plane_solid(int c, int n, int lo, int hi)
{
    return (lo && c == 0) || (hi && c == n - 1);
}

// Node geometry: coordinates, periodic neighbours, solid flags of the
// neighbouring planes and the row offsets of the nine (y, z) rows D3Q19 uses.
struct Geo {
    uint32_t n;
    int x, y, z, xm, xp;
    bool solid;
    bool sxm, sxp, sym, syp, szm, szp;
    uint32_t r00, rm0, rp0, r0m, r0p, rmm, rpm, rmp, rpp;   // r<y-shift><z-shift>, m: -1, p: +1
};

__device__ __forceinline__ Geo make_geo(const StepParams& p, uint32_t n)
{
    Geo g;
    g.n = n;
    const uint32_t zy = fdiv(n, p.div_nx);
    const uint32_t z = fdiv(n, p.div_nxy);
    g.x = (int)(n - zy * (uint32_t)p.nx);
    g.y = (int)(zy - z * (uint32_t)p.ny);
    g.z = (int)z;
    const int ym = g.y == 0 ? p.ny - 1 : g.y - 1, yp = g.y == p.ny - 1 ? 0 : g.y + 1;
    const int zm = g.z == 0 ? p.nz - 1 : g.z - 1, zp = g.z == p.nz - 1 ? 0 : g.z + 1;
    g.xm = g.x == 0 ? p.nx - 1 : g.x - 1;
    g.xp = g.x == p.nx - 1 ? 0 : g.x + 1;
    g.solid = plane_solid(g.x, p.nx, p.wlo[0], p.whi[0]) || plane_solid(g.y, p.ny, p.wlo[1], p.whi[1]) ||
              plane_solid(g.z, p.nz, p.wlo[2], p.whi[2]);
    g.sxm = plane_solid(g.xm, p.nx, p.wlo[0], p.whi[0]);
    g.sxp = plane_solid(g.xp, p.nx, p.wlo[0], p.whi[0]);
    g.sym = plane_solid(ym, p.ny, p.wlo[1], p.whi[1]);
    g.syp = plane_solid(yp, p.ny, p.wlo[1], p.whi[1]);
    g.szm = plane_solid(zm, p.nz, p.wlo[2], p.whi[2]);
    g.szp = plane_solid(zp, p.nz, p.wlo[2], p.whi[2]);
    const uint32_t nx = (uint32_t)p.nx, ny = (uint32_t)p.ny;
    g.r00 = (z * ny + (uint32_t)g.y) * nx;
    g.rm0 = (z * ny + (uint32_t)ym) * nx;
    g.rp0 = (z * ny + (uint32_t)yp) * nx;
    g.r0m = ((uint32_t)zm * ny + (uint32_t)g.y) * nx;
    g.r0p = ((uint32_t)zp * ny + (uint32_t)g.y) * nx;
    g.rmm = ((uint32_t)zm * ny + (uint32_t)ym) * nx;
    g.rpm = ((uint32_t)zm * ny + (uint32_t)yp) * nx;
    g.rmp = ((uint32_t)zp * ny + (uint32_t)ym) * nx;
    g.rpp = ((uint32_t)zp * ny + (uint32_t)yp) * nx;
    return g;
}

// Upstream index and solidity of the source of direction a (source = x - e_a).
// Pull: f_a(x, t+1) = f~_a(x - e_a, t); if x - e_a is solid the link is
// bounced: f_a(x, t+1) = f~_abar(x, t).
#define GLBE_DIRS(X)                                              \
    X(1, 2, g.r00 + g.xm, g.sxm)                                  \
    X(2, 1, g.r00 + g.xp, g.sxp)                                  \
    X(3, 4, g.rm0 + g.x, g.sym)                                   \
    X(4, 3, g.rp0 + g.x, g.syp)                                   \
    X(5, 6, g.r0m + g.x, g.szm)                                   \
    X(6, 5, g.r0p + g.x, g.szp)                                   \
    X(7, 10, g.rm0 + g.xm, g.sxm || g.sym)                        \
    X(8, 9, g.rm0 + g.xp, g.sxp || g.sym)                         \
    X(9, 8, g.rp0 + g.xm, g.sxm || g.syp)                         \
    X(10, 7, g.rp0 + g.xp, g.sxp || g.syp)                        \
    X(11, 14, g.r0m + g.xm, g.sxm || g.szm)                       \
    X(12, 13, g.r0m + g.xp, g.sxp || g.szm)                       \
    X(13, 12, g.r0p + g.xm, g.sxm || g.szp)                       \
    X(14, 11, g.r0p + g.xp, g.sxp || g.szp)                       \
    X(15, 18, g.rmm + g.x, g.sym || g.szm)                        \
    X(16, 17, g.rpm + g.x, g.syp || g.szm)                        \
    X(17, 16, g.rmp + g.x, g.sym || g.szp)                        \
    X(18, 15, g.rpp + g.x, g.syp || g.szp)

#define GLBE_DIRS7(X)                      \
    X(1, 2, g.r00 + g.xm, g.sxm)           \
    X(2, 1, g.r00 + g.xp, g.sxp)           \
    X(3, 4, g.rm0 + g.x, g.sym)            \
    X(4, 3, g.rp0 + g.x, g.syp)            \
    X(5, 6, g.r0m + g.x, g.szm)            \
    X(6, 5, g.r0p + g.x, g.szp)

template <int ST>
__device__ __forceinline__ void load_f(const StepParams& p, const typename Store<ST>::T* __restrict__ fs,
                                       const Geo& g, float (&d)[19], float (&l)[19])
{
    const size_t N = p.N;
#define GLBE_SRCF(a, o, src, sol) ((sol) ? (size_t)(o) * N + g.n : (size_t)(a) * N + (src))
#define GLBE_LOADF(a, o, src, sol) d[a] = Store<ST>::ld(fs + GLBE_SRCF(a, o, src, sol)) * p.inv_scale;
    d[0] = Store<ST>::ld(fs + g.n) * p.inv_scale;
    GLBE_DIRS(GLBE_LOADF)
#undef GLBE_LOADF
    if constexpr (Store<ST>::COMP) {
        const __half* __restrict__ fl = reinterpret_cast<const __half*>(fs + 19 * N);
#define GLBE_LOADL(a, o, src, sol) l[a] = Store<ST>::ld_lo(fl + GLBE_SRCF(a, o, src, sol));
        l[0] = Store<ST>::ld_lo(fl + g.n);
        GLBE_DIRS(GLBE_LOADL)
#undef GLBE_LOADL
    }
#undef GLBE_SRCF
}

// g is [j*7 + a][N]; anti-bounce-back: g_a(x, t+1) = -g~_abar(x, t) + 2 W_a B_wall,
// i.e. for deviations dg_a = -dg~_abar + 2 W_a (B_wall - B0).  In the
// compensated form the low part is negated with the high part (exact when
// B_wall = B0, the only case the C-ABI exposes).
template <int ST>
__device__ __forceinline__ void load_g(const StepParams& p, const typename Store<ST>::T* __restrict__ gs,
                                       const Geo& g, float (&q)[21], float (&ql)[21])
{
    const size_t N = p.N;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const typename Store<ST>::T* __restrict__ b = gs + (size_t)(j * 7) * N;
        const float wall = 0.25f * p.bwall_dev[j];   // 2 W_a (B_wall - B0), W_a = 1/8
        q[j * 7 + 0] = Store<ST>::ld(b + g.n) * p.inv_scale;
#define GLBE_LOADG(a, o, src, sol)                                                      \
    q[j * 7 + a] = (sol) ? (wall - Store<ST>::ld(b + (size_t)(o) * N + g.n) * p.inv_scale) \
                         : Store<ST>::ld(b + (size_t)(a) * N + (src)) * p.inv_scale;
        GLBE_DIRS7(GLBE_LOADG)
#undef GLBE_LOADG
        if constexpr (Store<ST>::COMP) {
            const __half* __restrict__ bl = reinterpret_cast<const __half*>(gs + 21 * N) + (size_t)(j * 7) * N;
            ql[j * 7 + 0] = Store<ST>::ld_lo(bl + g.n);
#define GLBE_LOADGL(a, o, src, sol)                                             \
    ql[j * 7 + a] = (sol) ? -Store<ST>::ld_lo(bl + (size_t)(o) * N + g.n)       \
                          : Store<ST>::ld_lo(bl + (size_t)(a) * N + (src));
            GLBE_DIRS7(GLBE_LOADGL)
#undef GLBE_LOADGL
        }
    }
}

// Grid constant of the error-free split x = xh + xl, xh = (x + C) - C: for
// |x| <= 2^-5 the high parts are multiples of 2^-28.
constexpr float SPLIT_C = 0.046875f;   // 1.5 * 2^-5

// Everything a node's collision produces besides the new populations.
struct NodeMacro {
    float rho, ux, uy, uz;
    float Bx, By, Bz;
    float FLx, FLy, FLz;
};

// Induction part: B, Lorentz force from the previous step's half-force
// velocity, and the D3Q7 collision change og = (g^eq - g)/tau_m (Eq. mcollision).
// PRECISE: B_j is formed from the exact split of the populations (qh on the
// 2^-28 grid, ql the remainder) and g^eq - g as (W_a Bh_j - qh_a) +
// (W_a Bl_j - ql_a) +- the convective term: W_a is a power of two, so the
// first bracket is exact and the rounding of the 7-term sum B no longer
// biases every population's relaxation (a bias the slow magnetic diffusion
// mode would otherwise integrate into a 3e-5 error of the steady flow).
template <bool PRECISE, bool COMP>
__device__ __forceinline__ void induction_collide(const StepParams& p, const float (&q)[21], const float (&qlo)[21],
                                                  float (&og)[21], float rho_inv, float mx, float my, float mz,
                                                  float Fx, float Fy, float Fz, float FLpx, float FLpy, float FLpz,
                                                  NodeMacro& mac)
{
    float qh[21], ql[21];
    if constexpr (PRECISE) {
#pragma unroll
        for (int i = 0; i < 21; ++i) {
            qh[i] = __fsub_rn(__fadd_rn(q[i], SPLIT_C), SPLIT_C);
            ql[i] = __fsub_rn(q[i], qh[i]);
            if constexpr (COMP) ql[i] += qlo[i];   // low part of the compensated storage
        }
    }
    // B_j = B0_j + sum_a dg_ja (sum_a W_a = 1), Eq. magneticinduction
    float bxh, byh, bzh, bxl = 0.f, byl = 0.f, bzl = 0.f;
    if constexpr (PRECISE) {
        bxh = qh[0] + qh[1] + qh[2] + qh[3] + qh[4] + qh[5] + qh[6];
        byh = qh[7] + qh[8] + qh[9] + qh[10] + qh[11] + qh[12] + qh[13];
        bzh = qh[14] + qh[15] + qh[16] + qh[17] + qh[18] + qh[19] + qh[20];
        bxl = ql[0] + ql[1] + ql[2] + ql[3] + ql[4] + ql[5] + ql[6];
        byl = ql[7] + ql[8] + ql[9] + ql[10] + ql[11] + ql[12] + ql[13];
        bzl = ql[14] + ql[15] + ql[16] + ql[17] + ql[18] + ql[19] + ql[20];
    } else {
        bxh = q[0] + q[1] + q[2] + q[3] + q[4] + q[5] + q[6];
        byh = q[7] + q[8] + q[9] + q[10] + q[11] + q[12] + q[13];
        bzh = q[14] + q[15] + q[16] + q[17] + q[18] + q[19] + q[20];
    }
    const float bx = bxh + bxl, by = byh + byl, bz = bzh + bzl;
    const float Bx = p.B0[0] + bx, By = p.B0[1] + by, Bz = p.B0[2] + bz;
    // velocity with the previous step's Lorentz force in the half-force
    const float hg = 0.5f * p.inv_gamma;
    const float u0x = (mx + hg * (Fx + FLpx)) * rho_inv;
    const float u0y = (my + hg * (Fy + FLpy)) * rho_inv;
    const float u0z = (mz + hg * (Fz + FLpz)) * rho_inv;
    // equilibrium first moment Lambda^eq_kj = (chi/gamma_m)(u_k B_j - B_k u_j)
    const float c = p.conv_coef;
    const float Lxy = c * (u0x * By - Bx * u0y);
    const float Lxz = c * (u0x * Bz - Bx * u0z);
    const float Lyz = c * (u0y * Bz - By * u0z);
    // first moments of g: M_kj = g_{+k,j} - g_{-k,j}; non-equilibrium parts
    const float Nxy = (q[7 + 1] - q[7 + 2]) - Lxy;     // k = x, j = y
    const float Nyx = (q[0 + 3] - q[0 + 4]) + Lxy;     // k = y, j = x (Lambda^eq_yx = -Lxy)
    const float Nxz = (q[14 + 1] - q[14 + 2]) - Lxz;
    const float Nzx = (q[0 + 5] - q[0 + 6]) + Lxz;
    const float Nyz = (q[14 + 3] - q[14 + 4]) - Lyz;
    const float Nzy = (q[7 + 5] - q[7 + 6]) + Lyz;
    // J_i = -(1/(mu chi tau_m theta_m)) eps_ijk Lneq_jk = (1/(mu chi)) (curl B)_i
    const float Jx = p.J_coef * (Nyz - Nzy);
    const float Jy = p.J_coef * (Nzx - Nxz);
    const float Jz = p.J_coef * (Nxy - Nyx);
    mac.FLx = Jy * Bz - Jz * By;
    mac.FLy = Jz * Bx - Jx * Bz;
    mac.FLz = Jx * By - Jy * Bx;
    mac.Bx = Bx; mac.By = By; mac.Bz = Bz;
    // g^eq,* deviations: W_0 b_j (rest), W_1 (b_j +- Lambda^eq_kj / theta_m), 1/theta_m = 4,
    // so the convective part is +-W_1 * 4 * L = +-L/2
    const float w = p.omega_m;
    const float Axy = 0.5f * Lxy, Axz = 0.5f * Lxz, Ayz = 0.5f * Lyz;
    // sign of the convective term of each (j, a): a = 0 rest, 1..6 = +x,-x,+y,-y,+z,-z
    const float conv[21] = {
        0.f, 0.f, 0.f, -Axy, Axy, -Axz, Axz,          // j = x: Lambda^eq_yx = -Lxy, Lambda^eq_zx = -Lxz
        0.f, Axy, -Axy, 0.f, 0.f, -Ayz, Ayz,          // j = y: Lambda^eq_xy = Lxy, Lambda^eq_zy = -Lyz
        0.f, Axz, -Axz, Ayz, -Ayz, 0.f, 0.f};         // j = z: Lambda^eq_xz = Lxz, Lambda^eq_yz = Lyz
#pragma unroll
    for (int i = 0; i < 21; ++i) {
        const int j = i / 7, a = i % 7;
        const float W = a == 0 ? 0.25f : 0.125f;
        const float bh = j == 0 ? bxh : (j == 1 ? byh : bzh);
        const float bl = j == 0 ? bxl : (j == 1 ? byl : bzl);
        float neq;
        if constexpr (PRECISE) neq = (W * bh - qh[i]) + ((W * bl - ql[i]) + conv[i]);
        else neq = (W * bh + conv[i]) - q[i];
        og[i] = w * neq;
    }
}

// Moments of a set of 19 deviations that are linear in them: group sums over
// the rest, axis and the three diagonal planes, then the rows of T (App. A).
struct Lin {
    float drho, mx, my, mz;          // rows 0, 3, 5, 7
    float M1, M2;                    // e, e^2 (rows 1, 2)
    float Qx, Qy, Qz;                // q (rows 4, 6, 8)
    float P9, P10, P11, P12, P13, P14, P15, P16, P17, P18;
};

__device__ __forceinline__ Lin linear_moments(const float (&d)[19])
{
    Lin L;
    const float Ax = d[1] + d[2], Ay = d[3] + d[4], Az = d[5] + d[6];
    const float Sax = Ax + Ay + Az;
    const float Gxy = d[7] + d[8] + d[9] + d[10];
    const float Gxz = d[11] + d[12] + d[13] + d[14];
    const float Gyz = d[15] + d[16] + d[17] + d[18];
    const float Sdg = Gxy + Gxz + Gyz;
    const float Xax = d[1] - d[2], Xxy = d[7] - d[8] + d[9] - d[10], Xxz = d[11] - d[12] + d[13] - d[14];
    const float Yax = d[3] - d[4], Yxy = d[7] + d[8] - d[9] - d[10], Yyz = d[15] - d[16] + d[17] - d[18];
    const float Zax = d[5] - d[6], Zxz = d[11] + d[12] - d[13] - d[14], Zyz = d[15] + d[16] - d[17] - d[18];
    L.drho = d[0] + Sax + Sdg;
    L.mx = Xax + Xxy + Xxz;
    L.my = Yax + Yxy + Yyz;
    L.mz = Zax + Zxz + Zyz;
    L.M1 = -30.f * d[0] - 11.f * Sax + 8.f * Sdg;
    L.M2 = 12.f * d[0] - 4.f * Sax + Sdg;
    L.Qx = -4.f * Xax + Xxy + Xxz;
    L.Qy = -4.f * Yax + Yxy + Yyz;
    L.Qz = -4.f * Zax + Zxz + Zyz;
    L.P9 = 2.f * Ax - Ay - Az + Gxy + Gxz - 2.f * Gyz;
    L.P10 = -4.f * Ax + 2.f * Ay + 2.f * Az + Gxy + Gxz - 2.f * Gyz;
    L.P11 = Ay - Az + Gxy - Gxz;
    L.P12 = -2.f * Ay + 2.f * Az + Gxy - Gxz;
    L.P13 = d[7] - d[8] - d[9] + d[10];
    L.P14 = d[15] - d[16] - d[17] + d[18];
    L.P15 = d[11] - d[12] - d[13] + d[14];
    L.P16 = Xxy - Xxz;
    L.P17 = Yyz - Yxy;
    L.P18 = Zxz - Zyz;
    return L;
}

// Error-free split d = dh + dl with dh on the grid of multiples of 2^-28
// (|d| <= 2^-5): integer-weighted sums of the dh are then exact in FP32 while
// they stay below 2^-4, and the dl (|dl| <= 2^-29) carry the rest.  Moments
// formed as (exact high sum - equilibrium) + low sum keep the small
// non-equilibrium parts free of the round-off of the large sums, which
// otherwise leaves the FP32 time march wandering at r ~ 1e-7 instead of
// settling on its fixed point.

__device__ __forceinline__ void split_exact(const float (&d)[19], float (&dh)[19], float (&dl)[19])
{
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        dh[a] = __fsub_rn(__fadd_rn(d[a], SPLIT_C), SPLIT_C);
        dl[a] = __fsub_rn(d[a], dh[a]);
    }
}

// Non-equilibrium moments and conserved sums of a node.  H holds the linear
// moments of the populations (or of their exact high parts) and L those of the
// low parts (PRECISE) -- L is not read otherwise.
template <bool PRECISE>
struct NodeMoments {
    Lin H, L;
    __device__ __forceinline__ float drho() const { return PRECISE ? H.drho + L.drho : H.drho; }
};

// D3Q19 moment-space collision change om = T^-1 [-Lambda* (f^ - f^eq,*) +
// (I - Lambda*/2) S*] (Eqs. ppostcollision, prelax_term).  F is the total
// force; (jx, jy, jz) = m + F/(2 gamma) rounded to FP32.
template <bool PRECISE>
__device__ __forceinline__ void flow_collide(const StepParams& p, const NodeMoments<PRECISE>& mm, float (&om)[19],
                                             float rho_inv, float jx, float jy, float jz, float Fx, float Fy,
                                             float Fz)
{
    const float ig = p.inv_gamma, ig2 = p.inv_gamma2;
    const float gri = ig * rho_inv;                   // 1/(gamma rho)
    const float ux = jx * rho_inv, uy = jy * rho_inv, uz = jz * rho_inv;
    const float jxx = jx * jx, jyy = jy * jy, jzz = jz * jz, jj = jxx + jyy + jzz;
    const Lin& H = mm.H;
    const Lin& L = mm.L;
#define GLBE_LO(expr) (PRECISE ? (expr) : 0.f)
#define GLBE_NK(hi, lo) (PRECISE ? (hi) + (lo) : (hi))
    // n_k = f^_k - f^eq,*_k; the rest state contributes -11 rho0 to row 1 and
    // 3 rho0 to row 2 only, so the deviations' moments enter directly
    const float n1 = GLBE_NK((H.M1 + 11.f * H.drho) - 19.f * jj * gri, GLBE_LO(L.M1 + 11.f * L.drho));
    const float n2 = GLBE_NK((H.M2 - 3.f * H.drho) + 5.5f * jj * gri, GLBE_LO(L.M2 - 3.f * L.drho));
    const float n4 = GLBE_NK(H.Qx, GLBE_LO(L.Qx)) + (2.f / 3.f) * jx;
    const float n6 = GLBE_NK(H.Qy, GLBE_LO(L.Qy)) + (2.f / 3.f) * jy;
    const float n8 = GLBE_NK(H.Qz, GLBE_LO(L.Qz)) + (2.f / 3.f) * jz;
    const float e9 = (3.f * jxx - jj) * gri;
    const float e11 = (jyy - jzz) * gri;
    const float n9 = GLBE_NK(H.P9 - e9, GLBE_LO(L.P9));
    const float n10 = GLBE_NK(H.P10 + 0.5f * e9, GLBE_LO(L.P10));
    const float n11 = GLBE_NK(H.P11 - e11, GLBE_LO(L.P11));
    const float n12 = GLBE_NK(H.P12 + 0.5f * e11, GLBE_LO(L.P12));
    const float n13 = GLBE_NK(H.P13 - jx * jy * gri, GLBE_LO(L.P13));
    const float n14 = GLBE_NK(H.P14 - jy * jz * gri, GLBE_LO(L.P14));
    const float n15 = GLBE_NK(H.P15 - jx * jz * gri, GLBE_LO(L.P15));
    const float n16 = GLBE_NK(H.P16, GLBE_LO(L.P16));
    const float n17 = GLBE_NK(H.P17, GLBE_LO(L.P17));
    const float n18 = GLBE_NK(H.P18, GLBE_LO(L.P18));
#undef GLBE_LO
#undef GLBE_NK

    // preconditioned source moments S* = P_S S (App. A, Eq. precondsourceterm)
    const float Fux = Fx * ux, Fuy = Fy * uy, Fuz = Fz * uz, Fu = Fux + Fuy + Fuz;
    const float S1 = 38.f * Fu * ig2, S2 = -11.f * Fu * ig2;
    const float S4 = (-2.f / 3.f) * Fx * ig, S6 = (-2.f / 3.f) * Fy * ig, S8 = (-2.f / 3.f) * Fz * ig;
    const float S9 = 2.f * (2.f * Fux - Fuy - Fuz) * ig2, S10 = -0.5f * S9;
    const float S11 = 2.f * (Fuy - Fuz) * ig2, S12 = -0.5f * S11;
    const float S13 = (Fx * uy + Fy * ux) * ig2;
    const float S14 = (Fy * uz + Fz * uy) * ig2;
    const float S15 = (Fx * uz + Fz * ux) * ig2;

    // delta_k = [-s_k n_k + (1 - s_k/2) S*_k] / |row_k|^2; conserved rows:
    // delta_3,5,7 = (F/gamma)/10 whatever the rate; delta_0 = 0.
#define GLBE_DK(k, nk, Sk, inv) (((-p.s[k]) * (nk) + (1.f - 0.5f * p.s[k]) * (Sk)) * (inv))
    const float q1 = GLBE_DK(1, n1, S1, 1.f / 2394.f);
    const float q2 = GLBE_DK(2, n2, S2, 1.f / 252.f);
    const float q3 = Fx * ig * 0.1f, q5 = Fy * ig * 0.1f, q7 = Fz * ig * 0.1f;
    const float q4 = GLBE_DK(4, n4, S4, 1.f / 40.f);
    const float q6 = GLBE_DK(6, n6, S6, 1.f / 40.f);
    const float q8 = GLBE_DK(8, n8, S8, 1.f / 40.f);
    const float q9 = GLBE_DK(9, n9, S9, 1.f / 36.f);
    const float q10 = GLBE_DK(10, n10, S10, 1.f / 72.f);
    const float q11 = GLBE_DK(11, n11, S11, 1.f / 12.f);
    const float q12 = GLBE_DK(12, n12, S12, 1.f / 24.f);
    const float q13 = GLBE_DK(13, n13, S13, 0.25f);
    const float q14 = GLBE_DK(14, n14, S14, 0.25f);
    const float q15 = GLBE_DK(15, n15, S15, 0.25f);
    const float q16 = -p.s[16] * n16 * 0.125f;
    const float q17 = -p.s[17] * n17 * 0.125f;
    const float q18 = -p.s[18] * n18 * 0.125f;
#undef GLBE_DK

    // om = T^t delta  (columns of T read from the basis polynomials); f~ = f + om
    om[0] = -30.f * q1 + 12.f * q2;
    const float A = -11.f * q1 - 4.f * q2;          // axis directions, c^2 = 1
    const float X9 = 2.f * q9 - 4.f * q10;           // 3c_x^2 - c^2 = 2 on +-x
    const float Y9 = -q9 + 2.f * q10;                // ... = -1 on +-y, +-z
    const float W11 = q11 - 2.f * q12;
    float t = q3 - 4.f * q4;
    om[1] = A + X9 + t;
    om[2] = A + X9 - t;
    t = q5 - 4.f * q6;
    om[3] = A + Y9 + W11 + t;
    om[4] = A + Y9 + W11 - t;
    t = q7 - 4.f * q8;
    om[5] = A + Y9 - W11 + t;
    om[6] = A + Y9 - W11 - t;
    const float Dg = 8.f * q1 + q2;                  // diagonal directions, c^2 = 2
    const float P = q9 + q10, Q = q11 + q12;
    {   // (+-1, +-1, 0)
        const float b = Dg + P + Q, ax = q3 + q4 + q16, by = q5 + q6 - q17;
        om[7] = b + ax + by + q13;
        om[8] = b - ax + by - q13;
        om[9] = b + ax - by - q13;
        om[10] = b - ax - by + q13;
    }
    {   // (+-1, 0, +-1)
        const float b = Dg + P - Q, ax = q3 + q4 - q16, bz = q7 + q8 + q18;
        om[11] = b + ax + bz + q15;
        om[12] = b - ax + bz - q15;
        om[13] = b + ax - bz - q15;
        om[14] = b - ax - bz + q15;
    }
    {   // (0, +-1, +-1)
        const float b = Dg - 2.f * P, ay = q5 + q6 + q17, bz = q7 + q8 - q18;
        om[15] = b + ay + bz + q14;
        om[16] = b - ay + bz - q14;
        om[17] = b + ay - bz - q14;
        om[18] = b - ay - bz + q14;
    }
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int ST, bool MHD, int MODE>
__global__ void __launch_bounds__(STEP_THREADS) step_kernel(const StepParams p, const StepBuffers b, const FieldOut fo)
{
    using S = Store<ST>;
    using T = typename S::T;
    if (b.stop != nullptr && *b.stop) return;   // converged solve: remaining steps of the chunk are skipped
    const uint32_t i = blockIdx.x * STEP_THREADS + threadIdx.x;
    const bool inb = i < p.N;
    const uint32_t n = inb ? i : 0u;
    const Geo g = make_geo(p, n);
    const bool fluid = inb && !g.solid;
    const size_t N = p.N;

    if (MODE == MODE_STEP && !fluid) return;
    if (MODE == MODE_FIELDS && !inb) return;

    // residual sums: FP32 per node and per warp (each term is one node's
    // FP32 quantity), FP64 from the block level on -- GB300's FP64 pipe is
    // kept off the per-node path
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (fluid) {
        float d[19], dl[19];
        load_f<ST>(p, static_cast<const T*>(b.fsrc), g, d, dl);
        float q[21], ql[21];
        float FLpx = 0.f, FLpy = 0.f, FLpz = 0.f;
        if (MHD) {
            load_g<ST>(p, static_cast<const T*>(b.gsrc), g, q, ql);
            FLpx = b.FL[n];
            FLpy = b.FL[N + n];
            FLpz = b.FL[2 * N + n];
        }
        // moments linear in the populations; density and bare first moment
        // (Eq. precondhydrofields)
        constexpr bool PRECISE = (ST == ST_F32 || ST == ST_F32C);
        NodeMoments<PRECISE> mm;
        if constexpr (PRECISE) {
            float dh[19], dlo[19];
            split_exact(d, dh, dlo);
            if constexpr (S::COMP) {
#pragma unroll
                for (int a = 0; a < 19; ++a) dlo[a] += dl[a];
            }
            mm.H = linear_moments(dh);
            mm.L = linear_moments(dlo);
        } else {
            mm.H = linear_moments(d);
        }
        const float drho = mm.drho();
        const float rho = p.rho0 + drho;
        const float rho_inv = 1.0f / rho;
        const float mxh = mm.H.mx, myh = mm.H.my, mzh = mm.H.mz;
        const float mxl = PRECISE ? mm.L.mx : 0.f, myl = PRECISE ? mm.L.my : 0.f, mzl = PRECISE ? mm.L.mz : 0.f;
        // external force
        float Fx = p.F[0], Fy = p.F[1], Fz = p.F[2];
        if (p.force_ncomp >= 1) Fx += __ldg(b.Ffield + n);
        if (p.force_ncomp == 3) {
            Fy += __ldg(b.Ffield + N + n);
            Fz += __ldg(b.Ffield + 2 * N + n);
        }
        NodeMacro mac;
        mac.Bx = mac.By = mac.Bz = 0.f;
        mac.FLx = mac.FLy = mac.FLz = 0.f;
        float og[21];
        if (MHD) {
            induction_collide<PRECISE, S::COMP>(p, q, ql, og, rho_inv, mxh + mxl, myh + myl, mzh + mzl, Fx, Fy, Fz,
                                                FLpx, FLpy, FLpz, mac);
            Fx += mac.FLx;
            Fy += mac.FLy;
            Fz += mac.FLz;
        }
        // j = m + F/(2 gamma): in the precise path the high parts and the
        // half-force are added by an exact two-sum before rounding once
        const float hg = 0.5f * p.inv_gamma;
        float jx, jy, jz;
        if constexpr (PRECISE) {
            jx = two_sum_round(mxh, hg * Fx, mxl);
            jy = two_sum_round(myh, hg * Fy, myl);
            jz = two_sum_round(mzh, hg * Fz, mzl);
        } else {
            jx = mxh + hg * Fx;
            jy = myh + hg * Fy;
            jz = mzh + hg * Fz;
        }
        const float ux = jx * rho_inv, uy = jy * rho_inv, uz = jz * rho_inv;

        if (MODE == MODE_FIELDS) {
            if (fo.rho) fo.rho[n] = rho;
            if (fo.u) { fo.u[n] = ux; fo.u[N + n] = uy; fo.u[2 * N + n] = uz; }
            if (MHD && fo.B) { fo.B[n] = mac.Bx; fo.B[N + n] = mac.By; fo.B[2 * N + n] = mac.Bz; }
            return;
        }

        float om[19];
        flow_collide<PRECISE>(p, mm, om, rho_inv, jx, jy, jz, Fx, Fy, Fz);
        // f~ = f + om, written to the node's own slot of the other buffer
        T* __restrict__ fd = static_cast<T*>(b.fdst);
        if constexpr (S::COMP) {
            __half* __restrict__ fdl = reinterpret_cast<__half*>(fd + 19 * N);
#pragma unroll
            for (int a = 0; a < 19; ++a) {
                float nh, nl;
                comp_add(d[a], dl[a], om[a], nh, nl);
                fd[(size_t)a * N + n] = nh;
                fdl[(size_t)a * N + n] = S::cv_lo(nl);
            }
        } else {
#pragma unroll
            for (int a = 0; a < 19; ++a) fd[(size_t)a * N + n] = S::cv((d[a] + om[a]) * p.scale);
        }
        if (MHD) {
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
                for (int a = 0; a < 21; ++a) gd[(size_t)a * N + n] = S::cv((q[a] + og[a]) * p.scale);
            }
            b.FL[n] = mac.FLx;
            b.FL[N + n] = mac.FLy;
            b.FL[2 * N + n] = mac.FLz;
        }
        if (MODE == MODE_STEP_RESID) {
            if (b.have_snap) {
                const float dx = ux - b.usnap[n], dy = uy - b.usnap[N + n], dz = uz - b.usnap[2 * N + n];
                acc[0] = dx * dx + dy * dy + dz * dz;
            }
            acc[1] = ux * ux + uy * uy + uz * uz;
            acc[2] = drho;                 // the mass is rho0 * (fluid nodes) + sum drho
            acc[3] = jx;
            acc[4] = jy;
            acc[5] = jz;
            acc[6] = isfinite(ux + uy + uz) ? 0.f : 1.f;
            b.usnap[n] = ux;
            b.usnap[N + n] = uy;
            b.usnap[2 * N + n] = uz;
        }
    } else if (MODE == MODE_FIELDS) {
        if (fo.rho) fo.rho[n] = 0.f;
        if (fo.u) { fo.u[n] = 0.f; fo.u[N + n] = 0.f; fo.u[2 * N + n] = 0.f; }
        if (MHD && fo.B) { fo.B[n] = 0.f; fo.B[N + n] = 0.f; fo.B[2 * N + n] = 0.f; }
        return;
    }

    if (MODE == MODE_STEP_RESID) {
        __shared__ double sh[STEP_THREADS / 32][7];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const float v = warp_sum(acc[k]);
            if (lane == 0) sh[warp][k] = (double)v;
        }
        __syncthreads();
        if (threadIdx.x < 7) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < STEP_THREADS / 32; ++w) s += sh[w][threadIdx.x];
            // structure of arrays: partials[k][block] (coalesced in the finalize)
            b.partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
        }
    }
}

// Pre-collision state (deviations, FP32, C-ABI layout) of every fluid node.
// The compensated form returns high + low rounded to FP32.
template <int ST, bool MHD>
__global__ void __launch_bounds__(STEP_THREADS) get_state_kernel(const StepParams p, const void* fsrc,
                                                                 const void* gsrc, const float* FL, float* df,
                                                                 float* dg, float* dFL)
{
    using T = typename Store<ST>::T;
    const uint32_t i = blockIdx.x * STEP_THREADS + threadIdx.x;
    if (i >= p.N) return;
    const Geo g = make_geo(p, i);
    const size_t N = p.N;
    if (g.solid) {
        if (df) for (int a = 0; a < 19; ++a) df[(size_t)a * N + i] = 0.f;
        if (MHD && dg) for (int a = 0; a < 21; ++a) dg[(size_t)a * N + i] = 0.f;
        if (MHD && dFL) for (int k = 0; k < 3; ++k) dFL[(size_t)k * N + i] = 0.f;
        return;
    }
    if (df) {
        float d[19], l[19];
        load_f<ST>(p, static_cast<const T*>(fsrc), g, d, l);
        for (int a = 0; a < 19; ++a) df[(size_t)a * N + i] = Store<ST>::COMP ? d[a] + l[a] : d[a];
    }
    if (MHD && dg) {
        float q[21], ql[21];
        load_g<ST>(p, static_cast<const T*>(gsrc), g, q, ql);
        for (int a = 0; a < 21; ++a) dg[(size_t)a * N + i] = Store<ST>::COMP ? q[a] + ql[a] : q[a];
    }
    if (MHD && dFL)
        for (int k = 0; k < 3; ++k) dFL[(size_t)k * N + i] = FL[(size_t)k * N + i];
}

// Inverse of get_state: each pre-collision value is written into the slot the
// next pull reads it from (the upstream node's slot, or the own node's
// opposite slot across a wall).  Every slot of a fluid node is written once.
// The compensated form starts with a zero low part.
template <int ST, bool MHD>
__global__ void __launch_bounds__(STEP_THREADS) set_state_kernel(const StepParams p, void* fsrc, void* gsrc,
                                                                 float* FL, const float* df, const float* dg,
                                                                 const float* dFL)
{
    using T = typename Store<ST>::T;
    const uint32_t i = blockIdx.x * STEP_THREADS + threadIdx.x;
    if (i >= p.N) return;
    const Geo g = make_geo(p, i);
    if (g.solid) return;
    const size_t N = p.N;
    if (df) {
        T* fs = static_cast<T*>(fsrc);
        __half* fl = Store<ST>::COMP ? reinterpret_cast<__half*>(fs + 19 * N) : nullptr;
#define GLBE_SLOTF(a, o, src, sol) ((sol) ? (size_t)(o) * N + i : (size_t)(a) * N + (src))
#define GLBE_STOREF(a, o, src, sol)                                                         \
    {                                                                                       \
        const size_t s_ = GLBE_SLOTF(a, o, src, sol);                                       \
        fs[s_] = Store<ST>::cv(df[(size_t)(a) * N + i] * p.scale);                          \
        if (Store<ST>::COMP) fl[s_] = __float2half_rn(0.f);                                 \
    }
        GLBE_STOREF(0, 0, i, false)
        GLBE_DIRS(GLBE_STOREF)
#undef GLBE_STOREF
#undef GLBE_SLOTF
    }
    if (MHD && dg) {
        T* gs = static_cast<T*>(gsrc);
        __half* gl = Store<ST>::COMP ? reinterpret_cast<__half*>(gs + 21 * N) : nullptr;
        for (int j = 0; j < 3; ++j) {
            T* bj = gs + (size_t)(j * 7) * N;
            __half* blj = Store<ST>::COMP ? gl + (size_t)(j * 7) * N : nullptr;
            const float* vj = dg + (size_t)(j * 7) * N;
            const float wall = 0.25f * p.bwall_dev[j];
#define GLBE_STOREG(a, o, src, sol)                                                                  \
    {                                                                                                \
        const size_t s_ = (sol) ? (size_t)(o) * N + i : (size_t)(a) * N + (src);                     \
        const float v_ = (sol) ? wall - vj[(size_t)(a) * N + i] : vj[(size_t)(a) * N + i];          \
        bj[s_] = Store<ST>::cv(v_ * p.scale);                                                        \
        if (Store<ST>::COMP) blj[s_] = __float2half_rn(0.f);                                         \
    }
            GLBE_STOREG(0, 0, i, false)
            GLBE_DIRS7(GLBE_STOREG)
#undef GLBE_STOREG
        }
    }
    if (MHD && dFL)
        for (int k = 0; k < 3; ++k) FL[(size_t)k * N + i] = dFL[(size_t)k * N + i];
}

template <int ST>
cudaError_t launch_step_t(bool mhd, int mode, const StepParams& p, const StepBuffers& b, const FieldOut& fo,
                          unsigned grid, cudaStream_t st)
{
    const dim3 blk(STEP_THREADS);
    if (mhd) {
        if (mode == MODE_STEP) step_kernel<ST, true, MODE_STEP><<<grid, blk, 0, st>>>(p, b, fo);
        else if (mode == MODE_STEP_RESID) step_kernel<ST, true, MODE_STEP_RESID><<<grid, blk, 0, st>>>(p, b, fo);
        else step_kernel<ST, true, MODE_FIELDS><<<grid, blk, 0, st>>>(p, b, fo);
    } else {
        if (mode == MODE_STEP) step_kernel<ST, false, MODE_STEP><<<grid, blk, 0, st>>>(p, b, fo);
        else if (mode == MODE_STEP_RESID) step_kernel<ST, false, MODE_STEP_RESID><<<grid, blk, 0, st>>>(p, b, fo);
        else step_kernel<ST, false, MODE_FIELDS><<<grid, blk, 0, st>>>(p, b, fo);
    }
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_get_state_t(bool mhd, const StepParams& p, const void* fsrc, const void* gsrc, const float* FL,
                               float* df, float* dg, float* dFL, cudaStream_t st)
{
    const unsigned grid = (p.N + STEP_THREADS - 1) / STEP_THREADS;
    if (mhd) get_state_kernel<ST, true><<<grid, STEP_THREADS, 0, st>>>(p, fsrc, gsrc, FL, df, dg, dFL);
    else get_state_kernel<ST, false><<<grid, STEP_THREADS, 0, st>>>(p, fsrc, gsrc, FL, df, dg, dFL);
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_set_state_t(bool mhd, const StepParams& p, void* fsrc, void* gsrc, float* FL, const float* df,
                               const float* dg, const float* dFL, cudaStream_t st)
{
    const unsigned grid = (p.N + STEP_THREADS - 1) / STEP_THREADS;
    if (mhd) set_state_kernel<ST, true><<<grid, STEP_THREADS, 0, st>>>(p, fsrc, gsrc, FL, df, dg, dFL);
    else set_state_kernel<ST, false><<<grid, STEP_THREADS, 0, st>>>(p, fsrc, gsrc, FL, df, dg, dFL);
    return cudaGetLastError();
}

}  // namespace glbe
