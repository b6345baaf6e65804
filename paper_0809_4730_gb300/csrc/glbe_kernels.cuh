// glbe_kernels.cuh -- fused time step of the preconditioned GLBE (D3Q19 MRT
// with forcing) and the preconditioned D3Q7 vector kinetic equation for the
// magnetic induction, arXiv:0809.4730 Secs. 2-4 and App. A.
//
// Pull scheme: a thread gathers the post-collision populations of the
// previous step from the upstream neighbours of its node (half-way
// bounce-back for f, anti-bounce-back for g where the upstream node is solid),
// forms the macroscopic fields, collides in moment space and writes the new
// post-collision populations into its own slots of the other buffer.  Buffers
// hold deviations from the rest state (df = f - w rho0, dg = g - W B0).
//
// Two kernels share one statement of the arithmetic, written over a value type
// V: the scalar kernel (V = float, one node per thread, any geometry) and the
// paired kernel (V = F2, two x-adjacent nodes per thread, x periodic with an
// even nx).  F2 maps onto Blackwell's packed FP32x2 add/mul/fma, so the paired
// kernel issues one arithmetic instruction for two nodes; its populations move
// as aligned 2-element vectors, and the two x-shifted sources per thread come
// from one aligned pair plus a lane shuffle.
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

// ---------------------------------------------------------------------------
// Value types: float, and F2 = two lanes of packed FP32 (sm_100+ FFMA2/FADD2/
// FMUL2).  Every operation rounds each lane to nearest exactly as the scalar
// one does.
// ---------------------------------------------------------------------------
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float c) : v(make_float2(c, c)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(float2 w) : v(w) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { a = a + b; return a; }

__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ F2 vfma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
// additions/subtractions that must not be contracted or reassociated
__device__ __forceinline__ float vadd_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ F2 vadd_rn(F2 a, F2 b) { return a + b; }
__device__ __forceinline__ F2 vsub_rn(F2 a, F2 b) { return a - b; }
__device__ __forceinline__ float vrcp(float a) { return 1.0f / a; }
__device__ __forceinline__ F2 vrcp(F2 a) { return F2(1.0f / a.v.x, 1.0f / a.v.y); }
__device__ __forceinline__ float lane_sum(float a) { return a; }
__device__ __forceinline__ float lane_sum(F2 a) { return a.v.x + a.v.y; }
__device__ __forceinline__ float vnonfinite(float a) { return isfinite(a) ? 0.f : 1.f; }
__device__ __forceinline__ float vnonfinite(F2 a) { return (isfinite(a.v.x) ? 0.f : 1.f) + (isfinite(a.v.y) ? 0.f : 1.f); }

// fl(a + b + c) for |c| small: the exact two-sum of a and b, its remainder
// plus c, rounded once.
template <class V>
__device__ __forceinline__ V two_sum_round(V a, V b, V c)
{
    const V s = vadd_rn(a, b);
    const V bp = vsub_rn(s, a);
    const V e = vadd_rn(vsub_rn(a, vsub_rn(s, bp)), vsub_rn(b, bp));
    return vadd_rn(s, vadd_rn(e, c));
}

// The same rounded sum, and in lo its remainder: hi + lo = fl(a + b) exactly
// + fl(e + c) (the double-float value the rounding of hi dropped).
template <class V>
__device__ __forceinline__ V two_sum_round_lo(V a, V b, V c, V& lo)
{
    const V s = vadd_rn(a, b);
    const V bp = vsub_rn(s, a);
    const V e = vadd_rn(vsub_rn(a, vsub_rn(s, bp)), vsub_rn(b, bp));
    const V t = vadd_rn(e, c);
    const V hi = vadd_rn(s, t);
    lo = vsub_rn(t, vsub_rn(hi, s));
    return hi;
}

// h + o + l as a new (high, low) pair: exact two-sum of h and o, the
// remainder plus the old low part renormalised into the new low part.
template <class V>
__device__ __forceinline__ void comp_add(V h, V l, V o, V& nh, V& nl)
{
    const V s = vadd_rn(h, o);
    const V bp = vsub_rn(s, h);
    const V ap = vsub_rn(s, bp);
    V e = vadd_rn(vsub_rn(h, ap), vsub_rn(o, bp));
    e = vadd_rn(e, l);
    nh = vadd_rn(s, e);
    nl = vsub_rn(e, vsub_rn(nh, s));
}

// ---------------------------------------------------------------------------
// Storage of the population deviations.  Only FP16 is stored scaled (by
// p.scale).  COMP marks the compensated form: an FP32 high part plus an FP16
// low part holding the rounding remainder (scaled by 2^36), updated with an
// exact two-sum; the low parts follow the high parts in the same buffer.
// ---------------------------------------------------------------------------
constexpr float LO_SCALE = 68719476736.0f;        // 2^36
constexpr float LO_INV = 1.4551915228366852e-11f; // 2^-36

template <int ST> struct Store;
// Read-only load asking L2 for the whole 256-byte block: a warp reads 128
// bytes of a population row and the next warp the following 128 (measured:
// F32 step 0.888 against 0.893 ms, F16 paired step 0.509 against 0.517 ms,
// BF16 paired step 0.485 against 0.489 ms, steady adjoint iteration 0.2455
// against 0.2462 ms)
__device__ __forceinline__ float ldg_l2_256(const float* p)
{
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ldg_l2_256(const uint32_t* p)
{
    uint32_t v;
    asm("ld.global.nc.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

template <> struct Store<ST_F32> {
    using T = float;
    static constexpr bool COMP = false, SCALED = false, SR = false;
    static __device__ __forceinline__ float ld(const T* p) { return ldg_l2_256(p); }
    static __device__ __forceinline__ T cv(float v) { return v; }
    static __device__ __forceinline__ F2 ld2(const T* p) { return F2(__ldg(reinterpret_cast<const float2*>(p))); }
    static __device__ __forceinline__ void st2(T* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }
};
template <> struct Store<ST_BF16> {
    using T = __nv_bfloat16;
    static constexpr bool COMP = false, SCALED = false, SR = false;
    static __device__ __forceinline__ float ld(const T* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ T cv(float v) { return __float2bfloat16_rn(v); }
    // a BF16 value is the high half of the FP32 with the same bits: the pair
    // is widened from one 32-bit load by a shift and a mask (exact; measured
    // 0.584 against 0.620 ms per paired step with __bfloat1622float2)
    static __device__ __forceinline__ F2 ld2(const T* p)
    {
        const uint32_t u = ldg_l2_256(reinterpret_cast<const uint32_t*>(p));
        return F2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
    static __device__ __forceinline__ void st2(T* p, F2 v)
    {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v.v);
    }
};
template <> struct Store<ST_F16> {
    using T = __half;
    static constexpr bool COMP = false, SCALED = true, SR = false;
    static __device__ __forceinline__ float ld(const T* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ T cv(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ F2 ld2(const T* p)
    {
        const uint32_t u = ldg_l2_256(reinterpret_cast<const uint32_t*>(p));
        __half2 h;
        memcpy(&h, &u, 4);
        return F2(__half22float2(h));
    }
    static __device__ __forceinline__ void st2(T* p, F2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v); }
};
template <> struct Store<ST_F32C> {
    using T = float;
    static constexpr bool COMP = true, SCALED = false, SR = false;
    static __device__ __forceinline__ float ld(const T* p) { return ldg_l2_256(p); }
    static __device__ __forceinline__ T cv(float v) { return v; }
    static __device__ __forceinline__ F2 ld2(const T* p) { return F2(__ldg(reinterpret_cast<const float2*>(p))); }
    static __device__ __forceinline__ void st2(T* p, F2 v) { *reinterpret_cast<float2*>(p) = v.v; }
    static __device__ __forceinline__ float ld_lo(const __half* p) { return __half2float(__ldg(p)) * LO_INV; }
    static __device__ __forceinline__ __half cv_lo(float v) { return __float2half_rn(v * LO_SCALE); }
    static __device__ __forceinline__ F2 ld2_lo(const __half* p)
    {
        const float2 w = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
        return F2(w.x * LO_INV, w.y * LO_INV);
    }
    static __device__ __forceinline__ void st2_lo(__half* p, F2 v)
    {
        *reinterpret_cast<__half2*>(p) = __float22half2_rn(make_float2(v.v.x * LO_SCALE, v.v.y * LO_SCALE));
    }
};

// Stochastically rounded 16-bit forms.  A value is stored as the 16-bit
// number next to it towards zero or away from zero, the latter with
// probability equal to the fraction of a unit in the last place by which it
// exceeds the former, so the stored value is unbiased.  Round-to-nearest
// drops every correction smaller than half a unit in the last place, which
// freezes the slow modes of a steady march at a false fixed point (the
// stagnation error ~ ulp / decay rate); rounded stochastically they keep
// moving to the right state on average.  Blackwell converts with explicit
// random bits (cvt.rs): the conversion of the pair (a, b) packs a into the
// upper and b into the lower 16 bits.
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float a, float b, uint32_t rbits)
{
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
    return d;
}
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float a, float b, uint32_t rbits)
{
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(a), "f"(b), "r"(rbits));
    return d;
}

template <> struct Store<ST_BF16_SR> : Store<ST_BF16> {
    static constexpr bool SR = true;
    static __device__ __forceinline__ T cv_sr(float v, uint32_t r)
    {
        return __ushort_as_bfloat16((unsigned short)(cvt_rs_bf16x2(v, 0.f, r) >> 16));
    }
    static __device__ __forceinline__ void st2_sr(T* p, F2 v, uint32_t r)
    {
        *reinterpret_cast<uint32_t*>(p) = cvt_rs_bf16x2(v.v.y, v.v.x, r);   // element 0 in the low half
    }
};
template <> struct Store<ST_F16_SR> : Store<ST_F16> {
    static constexpr bool SR = true;
    static __device__ __forceinline__ T cv_sr(float v, uint32_t r)
    {
        return __ushort_as_half((unsigned short)(cvt_rs_f16x2(v, 0.f, r) >> 16));
    }
    static __device__ __forceinline__ void st2_sr(T* p, F2 v, uint32_t r)
    {
        *reinterpret_cast<uint32_t*>(p) = cvt_rs_f16x2(v.v.y, v.v.x, r);
    }
};

// Random bits of the stochastic rounding: counter-based, so that a march is
// reproducible.  A node's (or pair's) generator starts from the MurmurHash3
// 32-bit finalizer (Appleby) of its index mixed with the hashed step seed,
// then steps a linear congruential generator (Numerical Recipes constants)
// once per stored population, its output whitened by a xor-shift.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
struct SrBits {
    uint32_t s;
    __device__ __forceinline__ SrBits(uint32_t node, uint32_t seed) : s(fmix32(node * 0x9e3779b9u + fmix32(seed))) {}
    __device__ __forceinline__ uint32_t next()
    {
        s = s * 1664525u + 1013904223u;
        return s ^ (s >> 16);
    }
};
// The step's seed (see StepBuffers::sr_ctr); 0 for the other forms.
template <int ST>
__device__ __forceinline__ uint32_t step_seed(const StepBuffers& b)
{
    if constexpr (Store<ST>::SR) return b.sr_ctr ? __ldg(b.sr_ctr + b.sr_par) : b.sr_seed;
    else return 0u;
}
// One thread of the step writes the next step's seed; no block of this step
// reads that slot.
template <int ST>
__device__ __forceinline__ void advance_seed(const StepBuffers& b)
{
    if constexpr (Store<ST>::SR) {
        if (b.sr_ctr && blockIdx.x == 0 && threadIdx.x == 0) b.sr_ctr[b.sr_par ^ 1] = step_seed<ST>(b) + 1u;
    }
}
// Stores of one value / one x-adjacent pair in the storage type.
template <int ST>
__device__ __forceinline__ typename Store<ST>::T store_cv(float v, SrBits& rb)
{
    if constexpr (Store<ST>::SR) return Store<ST>::cv_sr(v, rb.next());
    else return Store<ST>::cv(v);
}
template <int ST>
__device__ __forceinline__ void store_pair(typename Store<ST>::T* p, F2 v, SrBits& rb)
{
    if constexpr (Store<ST>::SR) Store<ST>::st2_sr(p, v, rb.next());
    else Store<ST>::st2(p, v);
}

// Loads of populations written earlier in the same launch (the persistent
// batch kernel) must not use the non-coherent read-only path.  CG = true
// gathers with coherent loads that are still cached in L1 (ld.global.ca):
// the gpu-scope fences of the grid barrier between levels order them after
// the previous level's stores, and no buffer is written in the level that
// reads it.  The second gather of a coupled node's two-pass update then hits
// L1 (64-duct F32C batch: 9.05 ms per level, 9.11 with ld.global.cg).
template <int ST, bool CG>
__device__ __forceinline__ float ldp(const typename Store<ST>::T* p)
{
    if constexpr (CG) {
        if constexpr (base_storage(ST) == ST_BF16) return __bfloat162float(__ldca(p));
        else if constexpr (base_storage(ST) == ST_F16) return __half2float(__ldca(p));
        else return __ldca(p);
    } else {
        return Store<ST>::ld(p);
    }
}
template <bool CG>
__device__ __forceinline__ float ldlo(const __half* p)
{
    if constexpr (CG) return __half2float(__ldca(p)) * LO_INV;
    else return Store<ST_F32C>::ld_lo(p);
}

template <int ST>
__device__ __forceinline__ float unscale(const StepParams& p, float v) { return Store<ST>::SCALED ? v * p.inv_scale : v; }
template <int ST>
__device__ __forceinline__ F2 unscale(const StepParams& p, F2 v) { return Store<ST>::SCALED ? v * F2(p.inv_scale) : v; }
template <int ST>
__device__ __forceinline__ float toscale(const StepParams& p, float v) { return Store<ST>::SCALED ? v * p.scale : v; }
template <int ST>
__device__ __forceinline__ F2 toscale(const StepParams& p, F2 v) { return Store<ST>::SCALED ? v * F2(p.scale) : v; }

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
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

__device__ __forceinline__ void row_geometry(const StepParams& p, int y, int z, Geo& g)
{
    const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
    g.sym = plane_solid(ym, p.ny, p.wlo[1], p.whi[1]);
    g.syp = plane_solid(yp, p.ny, p.wlo[1], p.whi[1]);
    g.szm = plane_solid(zm, p.nz, p.wlo[2], p.whi[2]);
    g.szp = plane_solid(zp, p.nz, p.wlo[2], p.whi[2]);
    const uint32_t nx = (uint32_t)p.nx, ny = (uint32_t)p.ny;
    g.r00 = ((uint32_t)z * ny + (uint32_t)y) * nx;
    g.rm0 = ((uint32_t)z * ny + (uint32_t)ym) * nx;
    g.rp0 = ((uint32_t)z * ny + (uint32_t)yp) * nx;
    g.r0m = ((uint32_t)zm * ny + (uint32_t)y) * nx;
    g.r0p = ((uint32_t)zp * ny + (uint32_t)y) * nx;
    g.rmm = ((uint32_t)zm * ny + (uint32_t)ym) * nx;
    g.rpm = ((uint32_t)zm * ny + (uint32_t)yp) * nx;
    g.rmp = ((uint32_t)zp * ny + (uint32_t)ym) * nx;
    g.rpp = ((uint32_t)zp * ny + (uint32_t)yp) * nx;
}

__device__ __forceinline__ Geo make_geo(const StepParams& p, uint32_t n)
{
    Geo g;
    g.n = n;
    const uint32_t zy = fdiv(n, p.div_nx);
    const uint32_t z = fdiv(n, p.div_nxy);
    g.x = (int)(n - zy * (uint32_t)p.nx);
    g.y = (int)(zy - z * (uint32_t)p.ny);
    g.z = (int)z;
    g.xm = g.x == 0 ? p.nx - 1 : g.x - 1;
    g.xp = g.x == p.nx - 1 ? 0 : g.x + 1;
    // a ghost plane is skipped like a solid one, but its neighbours gather from it as fluid
    g.solid = plane_solid(g.x, p.nx, p.wlo[0], p.whi[0]) || plane_solid(g.y, p.ny, p.wlo[1], p.whi[1]) ||
              plane_solid(g.z, p.nz, p.wlo[2], p.whi[2]) || plane_solid(g.z, p.nz, p.glo_z, p.ghi_z);
    g.sxm = plane_solid(g.xm, p.nx, p.wlo[0], p.whi[0]);
    g.sxp = plane_solid(g.xp, p.nx, p.wlo[0], p.whi[0]);
    row_geometry(p, g.y, g.z, g);
    return g;
}

// Pair geometry: nodes x0, x0 + 1 (x0 even) of one row of an x-periodic grid.
struct GeoP {
    Geo g;             // row data; g.x = x0, g.n = linear index of node x0
    int xl, xr;        // x0 - 1 and x0 + 2, wrapped
    bool left_own;     // the value at x0 - 1 is not in the left lane (warp or row start)
    bool right_own;    // the value at x0 + 2 is not in the right lane (warp or row end)
};

__device__ __forceinline__ GeoP make_geo_pair(const StepParams& p, uint32_t n0)
{
    GeoP q;
    Geo& g = q.g;
    g.n = n0;
    const uint32_t zy = fdiv(n0, p.div_nx);
    const uint32_t z = fdiv(n0, p.div_nxy);
    g.x = (int)(n0 - zy * (uint32_t)p.nx);
    g.y = (int)(zy - z * (uint32_t)p.ny);
    g.z = (int)z;
    g.xm = g.xp = 0;
    g.solid = plane_solid(g.y, p.ny, p.wlo[1], p.whi[1]) || plane_solid(g.z, p.nz, p.wlo[2], p.whi[2]) ||
              plane_solid(g.z, p.nz, p.glo_z, p.ghi_z);
    g.sxm = g.sxp = false;
    row_geometry(p, g.y, g.z, g);
    q.xl = g.x == 0 ? p.nx - 1 : g.x - 1;
    q.xr = g.x + 2 == p.nx ? 0 : g.x + 2;
    const int lane = threadIdx.x & 31;
    q.left_own = lane == 0 || g.x == 0;
    q.right_own = lane == 31 || g.x + 2 == p.nx;
    return q;
}

// Upstream row and solidity of the source of direction a (source = x - e_a),
// with the opposite direction o.  Pull: f_a(x, t+1) = f~_a(x - e_a, t); if
// x - e_a is solid the link is bounced: f_a(x, t+1) = f~_o(x, t).
// Scalar form: (a, o, source index, solid).
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

// Pair form: (a, o, source row, solid, x-shift e_x of the direction).
#define GLBE_PDIRS(X)                      \
    X(1, 2, g.r00, false, 1)               \
    X(2, 1, g.r00, false, -1)              \
    X(3, 4, g.rm0, g.sym, 0)               \
    X(4, 3, g.rp0, g.syp, 0)               \
    X(5, 6, g.r0m, g.szm, 0)               \
    X(6, 5, g.r0p, g.szp, 0)               \
    X(7, 10, g.rm0, g.sym, 1)              \
    X(8, 9, g.rm0, g.sym, -1)              \
    X(9, 8, g.rp0, g.syp, 1)               \
    X(10, 7, g.rp0, g.syp, -1)             \
    X(11, 14, g.r0m, g.szm, 1)             \
    X(12, 13, g.r0m, g.szm, -1)            \
    X(13, 12, g.r0p, g.szp, 1)             \
    X(14, 11, g.r0p, g.szp, -1)            \
    X(15, 18, g.rmm, g.sym || g.szm, 0)    \
    X(16, 17, g.rpm, g.syp || g.szm, 0)    \
    X(17, 16, g.rmp, g.sym || g.szp, 0)    \
    X(18, 15, g.rpp, g.syp || g.szp, 0)

#define GLBE_PDIRS7(X)                     \
    X(1, 2, g.r00, false, 1)               \
    X(2, 1, g.r00, false, -1)              \
    X(3, 4, g.rm0, g.sym, 0)               \
    X(4, 3, g.rp0, g.syp, 0)               \
    X(5, 6, g.r0m, g.szm, 0)               \
    X(6, 5, g.r0p, g.szp, 0)

// ---------------------------------------------------------------------------
// Gathers
// ---------------------------------------------------------------------------
template <int ST, bool CG = false>
__device__ __forceinline__ void load_f(const StepParams& p, const typename Store<ST>::T* __restrict__ fs,
                                       const Geo& g, float (&d)[19], float (&l)[19])
{
    const size_t N = p.N;
#define GLBE_SRCF(a, o, src, sol) ((sol) ? (size_t)(o) * N + g.n : (size_t)(a) * N + (src))
#define GLBE_LOADF(a, o, src, sol) d[a] = unscale<ST>(p, ldp<ST, CG>(fs + GLBE_SRCF(a, o, src, sol)));
    d[0] = unscale<ST>(p, ldp<ST, CG>(fs + g.n));
    GLBE_DIRS(GLBE_LOADF)
#undef GLBE_LOADF
    if constexpr (Store<ST>::COMP) {
        const __half* __restrict__ fl = reinterpret_cast<const __half*>(fs + 19 * N);
#define GLBE_LOADL(a, o, src, sol) l[a] = ldlo<CG>(fl + GLBE_SRCF(a, o, src, sol));
        l[0] = ldlo<CG>(fl + g.n);
        GLBE_DIRS(GLBE_LOADL)
#undef GLBE_LOADL
    }
#undef GLBE_SRCF
}

// g is [j*7 + a][N]; anti-bounce-back: g_a(x, t+1) = -g~_abar(x, t) + 2 W_a B_wall,
// i.e. for deviations dg_a = -dg~_abar + 2 W_a (B_wall - B0).  In the
// compensated form the low part is negated with the high part (exact when
// B_wall = B0, the only case the C-ABI exposes).
template <int ST, bool CG = false>
__device__ __forceinline__ void load_g(const StepParams& p, const typename Store<ST>::T* __restrict__ gs,
                                       const Geo& g, float (&q)[21], float (&ql)[21])
{
    const size_t N = p.N;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const typename Store<ST>::T* __restrict__ b = gs + (size_t)(j * 7) * N;
        const float wall = 0.25f * p.bwall_dev[j];   // 2 W_a (B_wall - B0), W_a = 1/8
        q[j * 7 + 0] = unscale<ST>(p, ldp<ST, CG>(b + g.n));
#define GLBE_LOADG(a, o, src, sol)                                                               \
    q[j * 7 + a] = (sol) ? (wall - unscale<ST>(p, ldp<ST, CG>(b + (size_t)(o) * N + g.n)))      \
                         : unscale<ST>(p, ldp<ST, CG>(b + (size_t)(a) * N + (src)));
        GLBE_DIRS7(GLBE_LOADG)
#undef GLBE_LOADG
        if constexpr (Store<ST>::COMP) {
            const __half* __restrict__ bl = reinterpret_cast<const __half*>(gs + 21 * N) + (size_t)(j * 7) * N;
            ql[j * 7 + 0] = ldlo<CG>(bl + g.n);
#define GLBE_LOADGL(a, o, src, sol)                                             \
    ql[j * 7 + a] = (sol) ? -ldlo<CG>(bl + (size_t)(o) * N + g.n)              \
                          : ldlo<CG>(bl + (size_t)(a) * N + (src));
            GLBE_DIRS7(GLBE_LOADGL)
#undef GLBE_LOADGL
        }
    }
}

// Interior nodes: the node and its 18 neighbours are fluid and no neighbour
// wraps around a periodic y or z axis, so the source of direction a is the
// fixed offset p.doff[a] = a N - (e_ax + e_ay nx + e_az nx ny) from the node,
// the same for every such node (no geometry, no bounce-back choice).  On an x
// axis without walls the x-seam nodes are interior too: the source x - 1 of
// x = 0 (directions with e_x = +1) lies nx further on (wp = nx), the source
// x + 1 of x = nx - 1 (e_x = -1) nx back (wm = -nx); elsewhere wp = wm = 0.
// (With walls on x no interior node lies on x = 0 or nx - 1.)
__device__ __forceinline__ bool is_interior(const StepParams& p, uint32_t n, int& wp, int& wm)
{
    if (!p.interior_ok) return false;
    const uint32_t zy = fdiv(n, p.div_nx);
    const uint32_t z = fdiv(n, p.div_nxy);
    const uint32_t x = n - zy * (uint32_t)p.nx;
    const uint32_t y = zy - z * (uint32_t)p.ny;
    wp = x == 0u ? p.nx : 0;
    wm = x == (uint32_t)p.nx - 1u ? -p.nx : 0;
    return (x - p.ilo[0]) <= p.ispan[0] && (y - p.ilo[1]) <= p.ispan[1] && (z - p.ilo[2]) <= p.ispan[2];
}

// x component of D3Q19 direction a (the order of include/glbe.h; its first
// seven are the D3Q7 directions)
__host__ __device__ constexpr int dir_ex(int a)
{
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
           : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}

// direction opposite to D3Q19 direction a (the order of include/glbe.h)
__host__ __device__ constexpr int dir_opp(int a)
{
    return a == 0 ? 0 : a <= 6 ? (a % 2 ? a + 1 : a - 1) : 7 + 4 * ((a - 7) / 4) + 3 - (a - 7) % 4;
}

static_assert(dir_opp(1) == 2 && dir_opp(4) == 3 && dir_opp(7) == 10 && dir_opp(8) == 9 && dir_opp(12) == 13 &&
                  dir_opp(14) == 11 && dir_opp(16) == 17 && dir_opp(18) == 15,
              "D3Q19 opposite directions");
static_assert(dir_ex(dir_opp(9)) == -dir_ex(9) && dir_ex(dir_opp(13)) == -dir_ex(13) && dir_ex(15) == 0,
              "D3Q19 x components");

// Source of direction a of an interior node from the node's own position
// base0 and its x-seam corrected positions: fixed per a after unrolling.
template <class P>
__device__ __forceinline__ P seam_src(int a, P base0, P basep, P basem)
{
    return dir_ex(a) > 0 ? basep : dir_ex(a) < 0 ? basem : base0;
}

template <int ST, bool CG = false>
__device__ __forceinline__ void load_f_interior(const StepParams& p, const typename Store<ST>::T* __restrict__ fs,
                                                uint32_t n, int wp, int wm, float (&d)[19], float (&l)[19])
{
    using T = typename Store<ST>::T;
    const T* __restrict__ f0 = fs + n;
    const T* __restrict__ fp = f0 + wp;
    const T* __restrict__ fm = f0 + wm;
#pragma unroll
    for (int a = 0; a < 19; ++a) d[a] = unscale<ST>(p, ldp<ST, CG>(seam_src(a, f0, fp, fm) + p.doff[a]));
    if constexpr (Store<ST>::COMP) {
        const __half* __restrict__ l0 = reinterpret_cast<const __half*>(fs + 19 * (size_t)p.N) + n;
        const __half* __restrict__ lp = l0 + wp;
        const __half* __restrict__ lm = l0 + wm;
#pragma unroll
        for (int a = 0; a < 19; ++a) l[a] = ldlo<CG>(seam_src(a, l0, lp, lm) + p.doff[a]);
    }
}

template <int ST, bool CG = false>
__device__ __forceinline__ void load_g_interior(const StepParams& p, const typename Store<ST>::T* __restrict__ gs,
                                                uint32_t n, int wp, int wm, float (&q)[21], float (&ql)[21])
{
    using T = typename Store<ST>::T;
    const size_t N = p.N;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const T* __restrict__ b0 = gs + (size_t)(j * 7) * N + n;
        const T* __restrict__ bp = b0 + wp;
        const T* __restrict__ bm = b0 + wm;
#pragma unroll
        for (int a = 0; a < 7; ++a) q[j * 7 + a] = unscale<ST>(p, ldp<ST, CG>(seam_src(a, b0, bp, bm) + p.doff[a]));
        if constexpr (Store<ST>::COMP) {
            const __half* __restrict__ l0 = reinterpret_cast<const __half*>(gs + 21 * N) + (size_t)(j * 7) * N + n;
            const __half* __restrict__ lp = l0 + wp;
            const __half* __restrict__ lm = l0 + wm;
#pragma unroll
            for (int a = 0; a < 7; ++a) ql[j * 7 + a] = ldlo<CG>(seam_src(a, l0, lp, lm) + p.doff[a]);
        }
    }
}

// One population of a pair: the two sources of direction a with x-shift ex
// from row `row` (solid: bounce-back from the own row's opposite slot o).
// ex = 0: one aligned pair.  ex = +1: node x0 needs x0 - 1 (the left lane's
// pair, or an own load at a warp or row start), node x0 + 1 needs x0.
// ex = -1: node x0 needs x0 + 1, node x0 + 1 needs x0 + 2 (the right lane's
// pair, or an own load at a warp or row end).  Every lane executes the
// shuffles; bounced rows never use them.
template <class LD2, class LD1>
__device__ __forceinline__ F2 pair_gather(const GeoP& q, size_t base_a, size_t base_o, uint32_t row, bool sol,
                                          int ex, LD2 ld2, LD1 ld1)
{
    const Geo& g = q.g;
    const F2 v = sol ? ld2(base_o + g.r00 + (uint32_t)g.x) : ld2(base_a + row + (uint32_t)g.x);
    if (ex > 0) {
        const float t = __shfl_up_sync(0xffffffffu, v.v.y, 1);
        if (sol) return v;
        const float left = q.left_own ? ld1(base_a + row + (uint32_t)q.xl) : t;
        return F2(left, v.v.x);
    }
    if (ex < 0) {
        const float t = __shfl_down_sync(0xffffffffu, v.v.x, 1);
        if (sol) return v;
        const float right = q.right_own ? ld1(base_a + row + (uint32_t)q.xr) : t;
        return F2(v.v.y, right);
    }
    return v;
}

template <int ST>
__device__ __forceinline__ void load_f_pair(const StepParams& p, const typename Store<ST>::T* __restrict__ fs,
                                            const GeoP& q, F2 (&d)[19], F2 (&l)[19])
{
    using S = Store<ST>;
    const size_t N = p.N;
    const Geo& g = q.g;
    auto ld2 = [&](size_t i) { return unscale<ST>(p, S::ld2(fs + i)); };
    auto ld1 = [&](size_t i) { return unscale<ST>(p, S::ld(fs + i)); };
    d[0] = ld2((size_t)g.r00 + (uint32_t)g.x);
#define GLBE_PLOADF(a, o, row, sol, ex) d[a] = pair_gather(q, (size_t)(a) * N, (size_t)(o) * N, row, sol, ex, ld2, ld1);
    GLBE_PDIRS(GLBE_PLOADF)
#undef GLBE_PLOADF
    if constexpr (S::COMP) {
        const __half* __restrict__ fl = reinterpret_cast<const __half*>(fs + 19 * N);
        auto lo2 = [&](size_t i) { return S::ld2_lo(fl + i); };
        auto lo1 = [&](size_t i) { return S::ld_lo(fl + i); };
        l[0] = lo2((size_t)g.r00 + (uint32_t)g.x);
#define GLBE_PLOADL(a, o, row, sol, ex) l[a] = pair_gather(q, (size_t)(a) * N, (size_t)(o) * N, row, sol, ex, lo2, lo1);
        GLBE_PDIRS(GLBE_PLOADL)
#undef GLBE_PLOADL
    }
}

template <int ST>
__device__ __forceinline__ void load_g_pair(const StepParams& p, const typename Store<ST>::T* __restrict__ gs,
                                            const GeoP& q, F2 (&v)[21], F2 (&vl)[21])
{
    using S = Store<ST>;
    const size_t N = p.N;
    const Geo& g = q.g;
    auto ld2 = [&](size_t i) { return unscale<ST>(p, S::ld2(gs + i)); };
    auto ld1 = [&](size_t i) { return unscale<ST>(p, S::ld(gs + i)); };
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const size_t jb = (size_t)(j * 7) * N;
        const F2 wall(0.25f * p.bwall_dev[j]);
        v[j * 7] = ld2(jb + g.r00 + (uint32_t)g.x);
#define GLBE_PLOADG(a, o, row, sol, ex)                                                              \
    {                                                                                                \
        const F2 t_ = pair_gather(q, jb + (size_t)(a) * N, jb + (size_t)(o) * N, row, sol, ex, ld2, ld1); \
        v[j * 7 + a] = (sol) ? wall - t_ : t_;                                                       \
    }
        GLBE_PDIRS7(GLBE_PLOADG)
#undef GLBE_PLOADG
        if constexpr (S::COMP) {
            const __half* __restrict__ gl = reinterpret_cast<const __half*>(gs + 21 * N);
            auto lo2 = [&](size_t i) { return S::ld2_lo(gl + i); };
            auto lo1 = [&](size_t i) { return S::ld_lo(gl + i); };
            vl[j * 7] = lo2(jb + g.r00 + (uint32_t)g.x);
#define GLBE_PLOADGL(a, o, row, sol, ex)                                                              \
    {                                                                                                 \
        const F2 t_ = pair_gather(q, jb + (size_t)(a) * N, jb + (size_t)(o) * N, row, sol, ex, lo2, lo1); \
        vl[j * 7 + a] = (sol) ? -t_ : t_;                                                             \
    }
            GLBE_PDIRS7(GLBE_PLOADGL)
#undef GLBE_PLOADGL
        }
    }
}

// ---------------------------------------------------------------------------
// Arithmetic of one node (V = float) or one pair of nodes (V = F2)
// ---------------------------------------------------------------------------

// Grid constant of the error-free split x = xh + xl, xh = (x + C) - C: for
// |x| <= 2^-5 the high parts are multiples of 2^-28, so integer-weighted sums
// of them are exact in FP32 while they stay below 2^-4, and the xl
// (|xl| <= 2^-29) carry the rest.  Moments formed as (exact high sum -
// equilibrium) + low sum keep the small non-equilibrium parts free of the
// round-off of the large sums, which otherwise leaves the FP32 time march
// wandering at r ~ 1e-7 instead of settling on its fixed point.
constexpr float SPLIT_C = 0.046875f;   // 1.5 * 2^-5

template <class V>
__device__ __forceinline__ void split_exact(const V& x, V& xh, V& xl)
{
    xh = vsub_rn(vadd_rn(x, V(SPLIT_C)), V(SPLIT_C));
    xl = vsub_rn(x, xh);
}

// Everything the induction part produces besides the new populations.
template <class V>
struct NodeMacro {
    V Bx, By, Bz;
    V FLx, FLy, FLz;
};

// Induction part: B, Lorentz force from the previous step's half-force
// velocity, and the D3Q7 collision change og = (g^eq - g)/tau_m (Eq. mcollision).
// PRECISE: B_j is formed from the exact split of the populations (qh on the
// 2^-28 grid, ql the remainder) and g^eq - g as (W_a Bh_j - qh_a) +
// (W_a Bl_j - ql_a) +- the convective term: W_a is a power of two, so the
// first bracket is exact and the rounding of the 7-term sum B no longer
// biases every population's relaxation (a bias the slow magnetic diffusion
// mode would otherwise integrate into a 3e-5 error of the steady flow).
template <class V, bool PRECISE, bool COMP>
__device__ __forceinline__ void induction_collide(const StepParams& p, const V (&q)[21], const V (&qlo)[21],
                                                  V (&og)[21], V rho_inv, V mx, V my, V mz, V Fx, V Fy, V Fz,
                                                  V FLpx, V FLpy, V FLpz, NodeMacro<V>& mac)
{
    V qh[21], ql[21];
    if constexpr (PRECISE) {
#pragma unroll
        for (int i = 0; i < 21; ++i) {
            split_exact(q[i], qh[i], ql[i]);
            if constexpr (COMP) ql[i] += qlo[i];   // low part of the compensated storage
        }
    }
    // B_j = B0_j + sum_a dg_ja (sum_a W_a = 1), Eq. magneticinduction
    V bxh, byh, bzh, bxl(0.f), byl(0.f), bzl(0.f);
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
    const V bx = PRECISE ? bxh + bxl : bxh, by = PRECISE ? byh + byl : byh, bz = PRECISE ? bzh + bzl : bzh;
    const V Bx = V(p.B0[0]) + bx, By = V(p.B0[1]) + by, Bz = V(p.B0[2]) + bz;
    // velocity with the previous step's Lorentz force in the half-force
    const V hg(0.5f * p.inv_gamma);
    const V u0x = (mx + hg * (Fx + FLpx)) * rho_inv;
    const V u0y = (my + hg * (Fy + FLpy)) * rho_inv;
    const V u0z = (mz + hg * (Fz + FLpz)) * rho_inv;
    // equilibrium first moment Lambda^eq_kj = (chi/gamma_m)(u_k B_j - B_k u_j)
    const V c(p.conv_coef);
    const V Lxy = c * (u0x * By - Bx * u0y);
    const V Lxz = c * (u0x * Bz - Bx * u0z);
    const V Lyz = c * (u0y * Bz - By * u0z);
    // first moments of g: M_kj = g_{+k,j} - g_{-k,j}; non-equilibrium parts
    const V Nxy = (q[7 + 1] - q[7 + 2]) - Lxy;     // k = x, j = y
    const V Nyx = (q[0 + 3] - q[0 + 4]) + Lxy;     // k = y, j = x (Lambda^eq_yx = -Lxy)
    const V Nxz = (q[14 + 1] - q[14 + 2]) - Lxz;
    const V Nzx = (q[0 + 5] - q[0 + 6]) + Lxz;
    const V Nyz = (q[14 + 3] - q[14 + 4]) - Lyz;
    const V Nzy = (q[7 + 5] - q[7 + 6]) + Lyz;
    // J_i = -(1/(mu chi tau_m theta_m)) eps_ijk Lneq_jk = (1/(mu chi)) (curl B)_i
    const V Jc(p.J_coef);
    const V Jx = Jc * (Nyz - Nzy);
    const V Jy = Jc * (Nzx - Nxz);
    const V Jz = Jc * (Nxy - Nyx);
    mac.FLx = Jy * Bz - Jz * By;
    mac.FLy = Jz * Bx - Jx * Bz;
    mac.FLz = Jx * By - Jy * Bx;
    mac.Bx = Bx;
    mac.By = By;
    mac.Bz = Bz;
    // g^eq,* deviations: W_0 b_j (rest), W_1 (b_j +- Lambda^eq_kj / theta_m), 1/theta_m = 4,
    // so the convective part is +-W_1 * 4 * L = +-L/2
    const V w(p.omega_m);
    const V Axy = V(0.5f) * Lxy, Axz = V(0.5f) * Lxz, Ayz = V(0.5f) * Lyz;
    const V zero(0.f);
    // convective term of each (j, a): a = 0 rest, 1..6 = +x,-x,+y,-y,+z,-z
    const V conv[21] = {
        zero, zero, zero, -Axy, Axy, -Axz, Axz,       // j = x: Lambda^eq_yx = -Lxy, Lambda^eq_zx = -Lxz
        zero, Axy, -Axy, zero, zero, -Ayz, Ayz,       // j = y: Lambda^eq_xy = Lxy, Lambda^eq_zy = -Lyz
        zero, Axz, -Axz, Ayz, -Ayz, zero, zero};      // j = z: Lambda^eq_xz = Lxz, Lambda^eq_yz = Lyz
#pragma unroll
    for (int i = 0; i < 21; ++i) {
        const int j = i / 7, a = i % 7;
        const V W(a == 0 ? 0.25f : 0.125f);
        const V bh = j == 0 ? bxh : (j == 1 ? byh : bzh);
        V neq;
        if constexpr (PRECISE) {
            const V bl = j == 0 ? bxl : (j == 1 ? byl : bzl);
            neq = (W * bh - qh[i]) + ((W * bl - ql[i]) + conv[i]);
        } else {
            neq = (W * bh + conv[i]) - q[i];
        }
        og[i] = w * neq;
    }
}

// Moments of a set of 19 deviations that are linear in them: group sums over
// the rest, axis and the three diagonal planes, then the rows of T (App. A).
template <class V>
struct Lin {
    V drho, mx, my, mz;          // rows 0, 3, 5, 7
    V M1, M2;                    // e, e^2 (rows 1, 2)
    V E1, E2;                    // M1 + 11 drho and M2 - 3 drho (the parts of n_1, n_2 linear in f)
    V Qx, Qy, Qz;                // q (rows 4, 6, 8)
    V Kx, Ky, Kz;                // (3 q + 2 m) / 5: the part of the heat-flux non-equilibrium linear in f
    V P9, P10, P11, P12, P13, P14, P15, P16, P17, P18;
};

template <class V>
__device__ __forceinline__ Lin<V> linear_moments(const V (&d)[19])
{
    Lin<V> L;
    const V Ax = d[1] + d[2], Ay = d[3] + d[4], Az = d[5] + d[6];
    const V Sax = Ax + Ay + Az;
    const V Gxy = d[7] + d[8] + d[9] + d[10];
    const V Gxz = d[11] + d[12] + d[13] + d[14];
    const V Gyz = d[15] + d[16] + d[17] + d[18];
    const V Sdg = Gxy + Gxz + Gyz;
    const V Xax = d[1] - d[2], Xxy = d[7] - d[8] + d[9] - d[10], Xxz = d[11] - d[12] + d[13] - d[14];
    const V Yax = d[3] - d[4], Yxy = d[7] + d[8] - d[9] - d[10], Yyz = d[15] - d[16] + d[17] - d[18];
    const V Zax = d[5] - d[6], Zxz = d[11] + d[12] - d[13] - d[14], Zyz = d[15] + d[16] - d[17] - d[18];
    L.drho = d[0] + Sax + Sdg;
    L.mx = Xax + Xxy + Xxz;
    L.my = Yax + Yxy + Yyz;
    L.mz = Zax + Zxz + Zyz;
    L.M1 = V(-30.f) * d[0] - V(11.f) * Sax + V(8.f) * Sdg;
    L.M2 = V(12.f) * d[0] - V(4.f) * Sax + Sdg;
    L.E1 = V(19.f) * (Sdg - d[0]);
    L.E2 = V(9.f) * d[0] - V(7.f) * Sax - V(2.f) * Sdg;
    L.Qx = V(-4.f) * Xax + Xxy + Xxz;
    L.Qy = V(-4.f) * Yax + Yxy + Yyz;
    L.Qz = V(-4.f) * Zax + Zxz + Zyz;
    L.Kx = V(-2.f) * Xax + Xxy + Xxz;
    L.Ky = V(-2.f) * Yax + Yxy + Yyz;
    L.Kz = V(-2.f) * Zax + Zxz + Zyz;
    const V two(2.f);
    const V a9 = two * Ax - Ay - Az, g9 = Gxy + Gxz - two * Gyz;     // axis and diagonal parts of rows 9, 10
    const V a11 = Ay - Az, g11 = Gxy - Gxz;                          // ... of rows 11, 12
    L.P9 = a9 + g9;
    L.P10 = V(-2.f) * a9 + g9;
    L.P11 = a11 + g11;
    L.P12 = V(-2.f) * a11 + g11;
    L.P13 = d[7] - d[8] - d[9] + d[10];
    L.P14 = d[15] - d[16] - d[17] + d[18];
    L.P15 = d[11] - d[12] - d[13] + d[14];
    L.P16 = Xxy - Xxz;
    L.P17 = Yyz - Yxy;
    L.P18 = Zxz - Zyz;
    return L;
}

// Linear moments of a node: H of the populations (or of their exact high
// parts) and L of the low parts (PRECISE only; L is not read otherwise).
template <class V, bool PRECISE>
struct NodeMoments {
    Lin<V> H, L;
    __device__ __forceinline__ V drho() const { return PRECISE ? H.drho + L.drho : H.drho; }
};

// D3Q19 moment-space collision change om = T^-1 [-Lambda* (f^ - f^eq,*) +
// (I - Lambda*/2) S*] (Eqs. ppostcollision, prelax_term).  F is the total
// force; (jx, jy, jz) = m + F/(2 gamma) rounded to FP32.
template <class V, bool PRECISE>
__device__ __forceinline__ void flow_collide(const StepParams& p, const NodeMoments<V, PRECISE>& mm, V (&om)[19],
                                             V rho_inv, V jx, V jy, V jz, V Fx, V Fy, V Fz)
{
    const V ig(p.inv_gamma);
    const V gri = ig * rho_inv;                   // 1/(gamma rho)
    const V ux = jx * rho_inv, uy = jy * rho_inv, uz = jz * rho_inv;
    // the quadratic equilibrium terms j_a j_b / (gamma rho)
    const V gjx = jx * gri, gjy = jy * gri, gjz = jz * gri;
    const V xx = jx * gjx, yy = jy * gjy, zz = jz * gjz, jjg = xx + yy + zz;
    const Lin<V>& H = mm.H;
    const Lin<V>& L = mm.L;
#define GLBE_NK(hi, lo) (PRECISE ? (hi) + (lo) : (hi))
    // n_k = f^_k - f^eq,*_k; the rest state contributes -11 rho0 to row 1 and
    // 3 rho0 to row 2 only, so the deviations' moments enter directly
    const V n1 = GLBE_NK(H.E1 - V(19.f) * jjg, L.E1);
    const V n2 = GLBE_NK(H.E2 + V(5.5f) * jjg, L.E2);
    // heat-flux rows: n = q + (2/3) j with j = m + F/(2 gamma) is a
    // near-cancellation of two values of the size of j.  The precise forms
    // use n = (5/3) K + F/(3 gamma), K = (3 q + 2 m)/5 a linear moment of the
    // populations (exact on their high parts): n no longer carries the FP32
    // rounding of j, which otherwise moved the converged state by about one
    // unit in the last place every few steps (residual floor ~1.4e-8 on the
    // 64^3 duct at gamma = 0.1).
    V n4, n6, n8;
    if constexpr (PRECISE) {
        const V f3(5.f / 3.f), ig3(p.inv_gamma * (1.f / 3.f));
        n4 = vfma(f3, H.Kx + L.Kx, ig3 * Fx);
        n6 = vfma(f3, H.Ky + L.Ky, ig3 * Fy);
        n8 = vfma(f3, H.Kz + L.Kz, ig3 * Fz);
    } else {
        n4 = H.Qx + V(2.f / 3.f) * jx;
        n6 = H.Qy + V(2.f / 3.f) * jy;
        n8 = H.Qz + V(2.f / 3.f) * jz;
    }
    const V e9 = V(3.f) * xx - jjg;
    const V e11 = yy - zz;
    const V n9 = GLBE_NK(H.P9 - e9, L.P9);
    const V n10 = GLBE_NK(H.P10 + V(0.5f) * e9, L.P10);
    const V n11 = GLBE_NK(H.P11 - e11, L.P11);
    const V n12 = GLBE_NK(H.P12 + V(0.5f) * e11, L.P12);
    const V n13 = GLBE_NK(H.P13 - jx * gjy, L.P13);
    const V n14 = GLBE_NK(H.P14 - jy * gjz, L.P14);
    const V n15 = GLBE_NK(H.P15 - jx * gjz, L.P15);
    const V n16 = GLBE_NK(H.P16, L.P16);
    const V n17 = GLBE_NK(H.P17, L.P17);
    const V n18 = GLBE_NK(H.P18, L.P18);
#undef GLBE_NK

    // delta_k = [-s_k n_k + (1 - s_k/2) S*_k] / |row_k|^2 with the
    // preconditioned source moments S* = P_S S (App. A, Eq. precondsourceterm).
    // Per row the host folds -s_k/|row_k|^2 into p.rl_a[k] and
    // (1 - s_k/2) P_S,k c_k/|row_k|^2 into p.rl_b[k], where S_k = c_k R_k with
    // R_k one of the force-velocity products below (c_k: 38 and -11 on rows 1,
    // 2; -2/3 on 4, 6, 8; 2 and -1 on 9, 10 and 11, 12; 1 on 13-15).
    // Conserved rows: delta_3,5,7 = (F/gamma)/10 whatever the rate; delta_0 = 0.
    const V Fux = Fx * ux, Fuy = Fy * uy, Fuz = Fz * uz, Fu = Fux + Fuy + Fuz;
    const V R9 = V(2.f) * Fux - Fuy - Fuz, R11 = Fuy - Fuz;
    // Precise forms: q_k = delta_k/|row_k|^2, and om = T^t q is the change
    // added to f.  16-bit forms (RECON): q_k = (m_k + delta_k)/|row_k|^2, the
    // post-collision moments, and om = T^t q is f~ itself (T T^t = diag |row_k|^2, so
    // f = T^t diag(1/|row_k|^2) m); f is then dead once its moments are formed.
    // Per row p.rl_c[k] = rl_a[k] + 1/|row_k|^2 takes the moment's own share;
    // rows 1, 2 carry m_1 = E1 - 11 drho and m_2 = E2 + 3 drho, row 0 gives
    // q_0 = drho / 19.  The extra FP32 rounding (~1e-7 of the moments) is far
    // below that of the stored 16-bit values.
    constexpr bool RECON = !PRECISE;
#define GLBE_DK(k, nk, Rk) vfma(V(p.rl_a[k]), (nk), V(p.rl_b[k]) * (Rk))
#define GLBE_RK(k, hk, ek, Rk) vfma(V(p.rl_c[k]), (hk), vfma(V(-p.rl_a[k]), (ek), V(p.rl_b[k]) * (Rk)))
    V q1, q2, q3, q4, q5, q6, q7, q8, q9, q10, q11, q12, q13, q14, q15, q16, q17, q18, q0;
    if constexpr (RECON) {
        const V dr = H.drho;
        q0 = V(1.f / 19.f) * dr;
        q1 = vfma(V(p.rl_c[1]), H.E1, vfma(V(-19.f * p.rl_a[1]), jjg, vfma(V(p.rl_b[1]), Fu, V(-11.f / 2394.f) * dr)));
        q2 = vfma(V(p.rl_c[2]), H.E2, vfma(V(5.5f * p.rl_a[2]), jjg, vfma(V(p.rl_b[2]), Fu, V(3.f / 252.f) * dr)));
        q3 = vfma(V(0.1f), H.mx, Fx * V(p.rl_cons));
        q5 = vfma(V(0.1f), H.my, Fy * V(p.rl_cons));
        q7 = vfma(V(0.1f), H.mz, Fz * V(p.rl_cons));
        q4 = GLBE_RK(4, H.Qx, V(-2.f / 3.f) * jx, Fx);
        q6 = GLBE_RK(6, H.Qy, V(-2.f / 3.f) * jy, Fy);
        q8 = GLBE_RK(8, H.Qz, V(-2.f / 3.f) * jz, Fz);
        q9 = GLBE_RK(9, H.P9, e9, R9);
        q10 = GLBE_RK(10, H.P10, V(-0.5f) * e9, R9);
        q11 = GLBE_RK(11, H.P11, e11, R11);
        q12 = GLBE_RK(12, H.P12, V(-0.5f) * e11, R11);
        q13 = GLBE_RK(13, H.P13, jx * gjy, Fx * uy + Fy * ux);
        q14 = GLBE_RK(14, H.P14, jy * gjz, Fy * uz + Fz * uy);
        q15 = GLBE_RK(15, H.P15, jx * gjz, Fx * uz + Fz * ux);
        q16 = V(p.rl_c[16]) * H.P16;
        q17 = V(p.rl_c[17]) * H.P17;
        q18 = V(p.rl_c[18]) * H.P18;
    } else {
        q0 = V(0.f);
        q1 = GLBE_DK(1, n1, Fu);
        q2 = GLBE_DK(2, n2, Fu);
        q3 = Fx * V(p.rl_cons);
        q5 = Fy * V(p.rl_cons);
        q7 = Fz * V(p.rl_cons);
        q4 = GLBE_DK(4, n4, Fx);
        q6 = GLBE_DK(6, n6, Fy);
        q8 = GLBE_DK(8, n8, Fz);
        q9 = GLBE_DK(9, n9, R9);
        q10 = GLBE_DK(10, n10, R9);
        q11 = GLBE_DK(11, n11, R11);
        q12 = GLBE_DK(12, n12, R11);
        q13 = GLBE_DK(13, n13, Fx * uy + Fy * ux);
        q14 = GLBE_DK(14, n14, Fy * uz + Fz * uy);
        q15 = GLBE_DK(15, n15, Fx * uz + Fz * ux);
        q16 = V(p.rl_a[16]) * n16;
        q17 = V(p.rl_a[17]) * n17;
        q18 = V(p.rl_a[18]) * n18;
    }
#undef GLBE_DK
#undef GLBE_RK

    // om = T^t q  (columns of T read from the basis polynomials); row 0 adds
    // q_0 to every direction (RECON only)
    om[0] = RECON ? vfma(V(-30.f), q1, vfma(V(12.f), q2, q0)) : V(-30.f) * q1 + V(12.f) * q2;
    const V A = RECON ? vfma(V(-11.f), q1, vfma(V(-4.f), q2, q0)) : V(-11.f) * q1 - V(4.f) * q2;   // axis, c^2 = 1
    const V X9 = V(2.f) * q9 - V(4.f) * q10;           // 3c_x^2 - c^2 = 2 on +-x
    const V Y9 = V(2.f) * q10 - q9;                    // ... = -1 on +-y, +-z
    const V W11 = q11 - V(2.f) * q12;
    V t = q3 - V(4.f) * q4;
    om[1] = A + X9 + t;
    om[2] = A + X9 - t;
    t = q5 - V(4.f) * q6;
    om[3] = A + Y9 + W11 + t;
    om[4] = A + Y9 + W11 - t;
    t = q7 - V(4.f) * q8;
    om[5] = A + Y9 - W11 + t;
    om[6] = A + Y9 - W11 - t;
    const V Dg = RECON ? vfma(V(8.f), q1, q2 + q0) : V(8.f) * q1 + q2;   // diagonal directions, c^2 = 2
    const V P = q9 + q10, Q = q11 + q12;
    {   // (+-1, +-1, 0)
        const V b = Dg + P + Q, ax = q3 + q4 + q16, by = q5 + q6 - q17;
        om[7] = b + ax + by + q13;
        om[8] = b - ax + by - q13;
        om[9] = b + ax - by - q13;
        om[10] = b - ax - by + q13;
    }
    {   // (+-1, 0, +-1)
        const V b = Dg + P - Q, ax = q3 + q4 - q16, bz = q7 + q8 + q18;
        om[11] = b + ax + bz + q15;
        om[12] = b - ax + bz - q15;
        om[13] = b + ax - bz - q15;
        om[14] = b - ax - bz + q15;
    }
    {   // (0, +-1, +-1)
        const V b = Dg - V(2.f) * P, ay = q5 + q6 + q17, bz = q7 + q8 - q18;
        om[15] = b + ay + bz + q14;
        om[16] = b - ay + bz - q14;
        om[17] = b + ay - bz - q14;
        om[18] = b - ay - bz + q14;
    }
}

// The preconditioned SRT-LBE with forcing term (Sec. 3.1), the limiting form
// of the GLBE with all relaxation rates equal to 1/tau* (tau* = 1/s_nu*):
// f~_a = f_a - (f_a - f^eq,*_a)/tau* + (1 - 1/(2 tau*)) S*_a in particle
// velocity space, with
//   f^eq,*_a = w_a rho [1 + 3 e.u + 9/(2 gamma) (e.u)^2 - 3/(2 gamma) u.u]
// (the u.u coefficient as the moment tables of App. A fix it) and the
// preconditioned source of Eq. precondsourcecorrect,
//   S*_a = w_a [3 (e - u/gamma).F / gamma + 9 (e.u)(e.F) / gamma^2],
// or, COLL = 2, the naive source of Eq. precondsourceincorrect,
//   S_a = w_a [3 (e - u).F + 9 (e.u)(e.F)] / gamma,
// whose Chapman-Enskog expansion carries a spurious momentum term for
// gamma < 1 (kept for comparison).  u = j/rho with the half-force j of Eq.
// precondhydrofields.  om receives the change of each population (precise
// forms) or the post-collision deviation itself (16-bit forms).
__host__ __device__ constexpr int dir_ey(int a)
{
    return (a == 3 || a == 7 || a == 8 || a == 15 || a == 17) ? 1
           : (a == 4 || a == 9 || a == 10 || a == 16 || a == 18) ? -1 : 0;
}
__host__ __device__ constexpr int dir_ez(int a)
{
    return (a == 5 || a == 11 || a == 12 || a == 15 || a == 16) ? 1
           : (a == 6 || a == 13 || a == 14 || a == 17 || a == 18) ? -1 : 0;
}
template <class V, bool PRECISE, int COLL>
__device__ __forceinline__ void srt_collide(const StepParams& p, const V (&d)[19], const V (&dl)[19], bool comp,
                                            V (&om)[19], V rho, V drho, V ux, V uy, V uz, V Fx, V Fy, V Fz)
{
    const float ig = p.inv_gamma;
    const V omega(p.s[9]);                      // 1/tau*, the viscous rate
    const V keep(1.f - 0.5f * p.s[9]);          // 1 - 1/(2 tau*)
    const V uu = ux * ux + uy * uy + uz * uz, uF = ux * Fx + uy * Fy + uz * Fz;
    const V c2(4.5f * ig), c3(1.5f * ig);
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        const float ex = (float)dir_ex(a), ey = (float)dir_ey(a), ez = (float)dir_ez(a);
        const V w(a == 0 ? 1.f / 3.f : (a <= 6 ? 1.f / 18.f : 1.f / 36.f));
        const V eu = V(ex) * ux + V(ey) * uy + V(ez) * uz;
        const V eF = V(ex) * Fx + V(ey) * Fy + V(ez) * Fz;
        const V feq = w * (drho + rho * (V(3.f) * eu + c2 * eu * eu - c3 * uu));   // f^eq,* - w rho0
        V S;
        if constexpr (COLL == 1) S = w * (V(3.f * ig) * (eF - V(ig) * uF) + V(9.f * ig * ig) * eu * eF);
        else S = w * V(ig) * (V(3.f) * (eF - uF) + V(9.f) * eu * eF);
        const V f = comp ? d[a] + dl[a] : d[a];
        const V change = omega * (feq - f) + keep * S;
        om[a] = PRECISE ? change : d[a] + change;
    }
}

// Post-collision deviation of one population from the gathered one (f) and
// the collision output om of flow_collide: the precise forms add the change,
// the 16-bit forms get f~ itself (the moment-space reconstruction).
template <int ST, class V>
__device__ __forceinline__ V post_collision(V f, V om)
{
    if constexpr (ST == ST_F32 || ST == ST_F32C) return f + om;
    else return om;
}

// Result of one node's (or pair's) update besides the new populations.
// ulx, uly, ulz (the FP32 and compensated forms): the low parts of u, so
// that u = u_hi + u_lo resolves changes below one unit in the last place of
// u_hi.  The residual of a converged march in FP32 arithmetic is otherwise
// floored by u_hi's own rounding (a state that still moves by 1e-12 flips
// u_hi by one unit of 6e-8 at many nodes: r ~ 3e-8).
template <class V>
struct NodeState {
    V rho, drho, jx, jy, jz, ux, uy, uz;
    V ulx, uly, ulz;
    NodeMacro<V> mac;
};

// The whole update of a node (pair) from its gathered populations: moments,
// induction and Lorentz force, velocity, collision changes om (f) and og (g).
// With collide = false only the macroscopic fields are formed.
template <class V, int ST, bool MHD, int COLL = 0>
__device__ __forceinline__ void node_update(const StepParams& p, const V (&d)[19], const V (&dl)[19],
                                            const V (&q)[21], const V (&ql)[21], V FLpx, V FLpy, V FLpz, V Fx,
                                            V Fy, V Fz, bool collide, V (&om)[19], V (&og)[21], NodeState<V>& ns)
{
    using S = Store<ST>;
    // moments linear in the populations; density and bare first moment
    // (Eq. precondhydrofields)
    constexpr bool PRECISE = (ST == ST_F32 || ST == ST_F32C);
    NodeMoments<V, PRECISE> mm;
    if constexpr (PRECISE) {
        V dh[19], dlo[19];
#pragma unroll
        for (int a = 0; a < 19; ++a) {
            split_exact(d[a], dh[a], dlo[a]);
            if constexpr (S::COMP) dlo[a] += dl[a];
        }
        mm.H = linear_moments(dh);
        mm.L = linear_moments(dlo);
    } else {
        mm.H = linear_moments(d);
    }
    ns.drho = mm.drho();
    ns.rho = V(p.rho0) + ns.drho;
    const V rho_inv = vrcp(ns.rho);
    const V mxh = mm.H.mx, myh = mm.H.my, mzh = mm.H.mz;
    const V mxl = PRECISE ? mm.L.mx : V(0.f), myl = PRECISE ? mm.L.my : V(0.f), mzl = PRECISE ? mm.L.mz : V(0.f);
    ns.mac.Bx = ns.mac.By = ns.mac.Bz = V(0.f);
    ns.mac.FLx = ns.mac.FLy = ns.mac.FLz = V(0.f);
    if (MHD) {
        induction_collide<V, PRECISE, S::COMP>(p, q, ql, og, rho_inv, PRECISE ? mxh + mxl : mxh,
                                               PRECISE ? myh + myl : myh, PRECISE ? mzh + mzl : mzh, Fx, Fy, Fz,
                                               FLpx, FLpy, FLpz, ns.mac);
        Fx += ns.mac.FLx;
        Fy += ns.mac.FLy;
        Fz += ns.mac.FLz;
    }
    // j = m + F/(2 gamma): in the precise path the high parts and the
    // half-force are added by an exact two-sum before rounding once
    const V hg(0.5f * p.inv_gamma);
    V jlx(0.f), jly(0.f), jlz(0.f);
    if constexpr (PRECISE) {
        ns.jx = two_sum_round_lo(mxh, hg * Fx, mxl, jlx);
        ns.jy = two_sum_round_lo(myh, hg * Fy, myl, jly);
        ns.jz = two_sum_round_lo(mzh, hg * Fz, mzl, jlz);
    } else {
        ns.jx = mxh + hg * Fx;
        ns.jy = myh + hg * Fy;
        ns.jz = mzh + hg * Fz;
    }
    ns.ux = ns.jx * rho_inv;
    ns.uy = ns.jy * rho_inv;
    ns.uz = ns.jz * rho_inv;
    ns.ulx = ns.uly = ns.ulz = V(0.f);
    if constexpr (PRECISE) {
        // rho's low part: rho0 - rho is exact next to rho0, and so is its sum
        // with the high part of drho (both on the 2^-28 grid, small)
        const V rlo = vadd_rn(vadd_rn(vsub_rn(V(p.rho0), ns.rho), mm.H.drho), mm.L.drho);
        // u_lo = (j - u_hi rho + j_lo - u_hi rho_lo) / rho
        ns.ulx = (vfma(-ns.ux, ns.rho, ns.jx) + jlx - ns.ux * rlo) * rho_inv;
        ns.uly = (vfma(-ns.uy, ns.rho, ns.jy) + jly - ns.uy * rlo) * rho_inv;
        ns.ulz = (vfma(-ns.uz, ns.rho, ns.jz) + jlz - ns.uz * rlo) * rho_inv;
    }
    if (collide) {
        if constexpr (COLL == 0) flow_collide<V, PRECISE>(p, mm, om, rho_inv, ns.jx, ns.jy, ns.jz, Fx, Fy, Fz);
        else srt_collide<V, PRECISE, COLL>(p, d, dl, S::COMP, om, ns.rho, ns.drho, ns.ux, ns.uy, ns.uz, Fx, Fy, Fz);
    }
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Residual sums of a block into partials[k][block]: FP32 per node, warp and
// block (at most 256 terms, all of one node's FP32 quantities), FP64 from the
// partials on -- GB300's FP64 pipe is kept off the step kernel.
template <int NT>
__device__ __forceinline__ void block_partials(float (&acc)[7], double* partials)
{
    __shared__ float sh[NT / 32][7];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const float v = warp_sum(acc[k]);
        if (lane == 0) sh[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += sh[w][threadIdx.x];
        partials[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = (double)s;
    }
}

// Per-node inputs besides the populations: the lagged Lorentz force, the
// total external force and (residual steps) the previous velocity snapshot.
// They are loaded apart from the update so that a kernel can issue these
// loads early (before waiting on staged populations); the snapshot in
// particular must be read before the node's stores, which a later load would
// have to wait for (measured: the residual step took 5.3 ms instead of
// 1.3 ms on the 512 x 256 x 256 duct).
template <class V>
struct NodeIn {
    V FLx, FLy, FLz, Fx, Fy, Fz, us0, us1, us2;
    V ul0, ul1, ul2;   // low parts of the snapshot (b.snap_lo)
};

// FL_IN_F: the flow pass of a two-pass coupled update (coupled_induction_pass
// wrote this step's Lorentz force into b.FL): the total force is the external
// force plus b.FL, added as the one-pass update adds it.
template <bool MHD, int MODE, bool FL_IN_F = false>
__device__ __forceinline__ NodeIn<float> node_inputs(const StepParams& p, const StepBuffers& b, uint32_t n)
{
    const size_t N = p.N;
    NodeIn<float> in;
    in.FLx = in.FLy = in.FLz = 0.f;
    if (MHD) {
        in.FLx = b.FL[n];
        in.FLy = b.FL[N + n];
        in.FLz = b.FL[2 * N + n];
    }
    in.Fx = p.F[0];
    in.Fy = p.F[1];
    in.Fz = p.F[2];
    if (p.force_ncomp >= 1) in.Fx += __ldg(b.Ffield + n);
    if (p.force_ncomp == 3) {
        in.Fy += __ldg(b.Ffield + N + n);
        in.Fz += __ldg(b.Ffield + 2 * N + n);
    }
    if constexpr (FL_IN_F) {
        in.Fx += b.FL[n];
        in.Fy += b.FL[N + n];
        in.Fz += b.FL[2 * N + n];
    }
    in.us0 = in.us1 = in.us2 = 0.f;
    in.ul0 = in.ul1 = in.ul2 = 0.f;
    if (MODE == MODE_STEP_RESID && b.have_snap) {
        in.us0 = b.usnap[n];
        in.us1 = b.usnap[N + n];
        in.us2 = b.usnap[2 * N + n];
        if (b.snap_lo) {
            in.ul0 = b.usnap[3 * N + n];
            in.ul1 = b.usnap[4 * N + n];
            in.ul2 = b.usnap[5 * N + n];
        }
    }
    return in;
}

template <bool MHD, int MODE>
__device__ __forceinline__ NodeIn<F2> pair_inputs(const StepParams& p, const StepBuffers& b, uint32_t n0)
{
    const size_t N = p.N;
    NodeIn<F2> in;
    in.FLx = in.FLy = in.FLz = F2(0.f);
    if (MHD) {
        in.FLx = F2(*reinterpret_cast<const float2*>(b.FL + n0));
        in.FLy = F2(*reinterpret_cast<const float2*>(b.FL + N + n0));
        in.FLz = F2(*reinterpret_cast<const float2*>(b.FL + 2 * N + n0));
    }
    in.Fx = F2(p.F[0]);
    in.Fy = F2(p.F[1]);
    in.Fz = F2(p.F[2]);
    if (p.force_ncomp >= 1) in.Fx += F2(__ldg(reinterpret_cast<const float2*>(b.Ffield + n0)));
    if (p.force_ncomp == 3) {
        in.Fy += F2(__ldg(reinterpret_cast<const float2*>(b.Ffield + N + n0)));
        in.Fz += F2(__ldg(reinterpret_cast<const float2*>(b.Ffield + 2 * N + n0)));
    }
    in.us0 = in.us1 = in.us2 = F2(0.f);
    in.ul0 = in.ul1 = in.ul2 = F2(0.f);
    if (MODE == MODE_STEP_RESID && b.have_snap) {
        in.us0 = F2(*reinterpret_cast<const float2*>(b.usnap + n0));
        in.us1 = F2(*reinterpret_cast<const float2*>(b.usnap + N + n0));
        in.us2 = F2(*reinterpret_cast<const float2*>(b.usnap + 2 * N + n0));
        if (b.snap_lo) {
            in.ul0 = F2(*reinterpret_cast<const float2*>(b.usnap + 3 * N + n0));
            in.ul1 = F2(*reinterpret_cast<const float2*>(b.usnap + 4 * N + n0));
            in.ul2 = F2(*reinterpret_cast<const float2*>(b.usnap + 5 * N + n0));
        }
    }
    return in;
}

template <int ST, bool MHD, int MODE, bool DIR = false, int COLL = 0>
__device__ __forceinline__ void node_from_sources(const StepParams& p, const StepBuffers& b, const FieldOut& fo,
                                                  uint32_t n, const float (&d)[19], const float (&dl)[19],
                                                  const float (&q)[21], const float (&ql)[21],
                                                  const NodeIn<float>& in, float (&acc)[7]);

// Interior gather of f from the per-direction bases b.fsrc_dir (filled by
// the launcher): one base per direction, and the node's own offset (x-seam
// corrected for e_x = +-1) shared by all directions.
template <int ST>
__device__ __forceinline__ void load_f_interior_dir(const StepParams& p, const StepBuffers& b, uint32_t n, int wp,
                                                    int wm, float (&d)[19])
{
    using T = typename Store<ST>::T;
    const size_t n0 = n, np = (size_t)((long long)n + wp), nm = (size_t)((long long)n + wm);
#pragma unroll
    for (int a = 0; a < 19; ++a)
        d[a] = unscale<ST>(p, Store<ST>::ld(static_cast<const T*>(b.fsrc_dir[a]) + seam_src(a, n0, np, nm)));
}

// ---------------------------------------------------------------------------
// Scalar kernel: one node per thread, any geometry
// ---------------------------------------------------------------------------
// The update of node n (i < N) by one thread; accumulates the residual terms
// of MODE_STEP_RESID into acc.  Returns without work for solid nodes.
// DIR: the per-direction bases of b are filled (kernels launched by
// launch_mode); they serve the interior gather and the stores of f.
template <int ST, bool MHD, int MODE, bool CG = false, bool DIR = false, bool FL_IN_F = false, int COLL = 0>
__device__ __forceinline__ void scalar_node_step(const StepParams& p, const StepBuffers& b, const FieldOut& fo,
                                                 uint32_t i, float (&acc)[7])
{
    using S = Store<ST>;
    using T = typename S::T;
    const bool inb = i < p.N;
    const uint32_t n = inb ? i : 0u;
    const size_t N = p.N;
    float d[19], dl[19], q[21], ql[21];
    int wp = 0, wm = 0;
    if (inb && is_interior(p, n, wp, wm)) {
        // no solid node and no y or z wrap around: every source at a fixed
        // offset (x-seam sources corrected by wp, wm)
        if constexpr (DIR && !S::COMP && !CG) load_f_interior_dir<ST>(p, b, n, wp, wm, d);
        else load_f_interior<ST, CG>(p, static_cast<const T*>(b.fsrc), n, wp, wm, d, dl);
        if (MHD) load_g_interior<ST, CG>(p, static_cast<const T*>(b.gsrc), n, wp, wm, q, ql);
    } else {
        const Geo g = make_geo(p, n);
        if (!inb || g.solid) {
            if (MODE == MODE_FIELDS && inb) {
                if (fo.rho) fo.rho[n] = 0.f;
                if (fo.u) { fo.u[n] = 0.f; fo.u[N + n] = 0.f; fo.u[2 * N + n] = 0.f; }
                if (MHD && fo.B) { fo.B[n] = 0.f; fo.B[N + n] = 0.f; fo.B[2 * N + n] = 0.f; }
            }
            return;
        }
        load_f<ST, CG>(p, static_cast<const T*>(b.fsrc), g, d, dl);
        if (MHD) load_g<ST, CG>(p, static_cast<const T*>(b.gsrc), g, q, ql);
    }
    node_from_sources<ST, MHD, MODE, DIR, COLL>(p, b, fo, n, d, dl, q, ql, node_inputs<MHD, MODE, FL_IN_F>(p, b, n),
                                                 acc);
}

// Two-pass coupled update, pass 1 (the persistent batch kernel: one update
// of a coupled node does not fit its register budget).  Gathers f and g of
// node i, forms rho and m (Eq. precondhydrofields), runs the induction part
// exactly as node_update does (B, Lorentz force from the previous step's
// half-force velocity, D3Q7 collision; Sec. 4) and writes g~ and this step's
// Lorentz force into b.FL.  Pass 2 is scalar_node_step<ST, false, MODE, CG,
// false, true>: it gathers f again (from L2) and runs the flow update with
// F = F_ext + b.FL, which is the one-pass update's arithmetic in the same
// order, so the result is bit for bit the same.
template <int ST>
__device__ __forceinline__ void induction_from_sources(const StepParams& p, const StepBuffers& b, uint32_t n,
                                                      const float (&d)[19], const float (&dl)[19],
                                                      const float (&q)[21], const float (&ql)[21]);

template <int ST, bool CG>
__device__ __forceinline__ void coupled_induction_pass(const StepParams& p, const StepBuffers& b, uint32_t i)
{
    using S = Store<ST>;
    using T = typename S::T;
    constexpr bool PRECISE = (ST == ST_F32 || ST == ST_F32C);
    if (!(i < p.N)) return;
    const uint32_t n = i;
    const size_t N = p.N;
    float d[19], dl[19], q[21], ql[21];
    int wp = 0, wm = 0;
    if (is_interior(p, n, wp, wm)) {
        load_f_interior<ST, CG>(p, static_cast<const T*>(b.fsrc), n, wp, wm, d, dl);
        load_g_interior<ST, CG>(p, static_cast<const T*>(b.gsrc), n, wp, wm, q, ql);
    } else {
        const Geo g = make_geo(p, n);
        if (g.solid) return;
        load_f<ST, CG>(p, static_cast<const T*>(b.fsrc), g, d, dl);
        load_g<ST, CG>(p, static_cast<const T*>(b.gsrc), g, q, ql);
    }
    induction_from_sources<ST>(p, b, n, d, dl, q, ql);
}

// Pass 1 of the two-pass coupled update from the gathered populations of
// node n: rho and m, the induction part, and the stores of g~ and of this
// step's Lorentz force.
template <int ST>
__device__ __forceinline__ void induction_from_sources(const StepParams& p, const StepBuffers& b, uint32_t n,
                                                      const float (&d)[19], const float (&dl)[19],
                                                      const float (&q)[21], const float (&ql)[21])
{
    using S = Store<ST>;
    using T = typename S::T;
    constexpr bool PRECISE = (ST == ST_F32 || ST == ST_F32C);
    const size_t N = p.N;
    const NodeIn<float> in = node_inputs<true, MODE_STEP>(p, b, n);
    // rho and m as node_update forms them
    NodeMoments<float, PRECISE> mm;
    if constexpr (PRECISE) {
        float dh[19], dlo[19];
#pragma unroll
        for (int a = 0; a < 19; ++a) {
            split_exact(d[a], dh[a], dlo[a]);
            if constexpr (S::COMP) dlo[a] += dl[a];
        }
        mm.H = linear_moments(dh);
        mm.L = linear_moments(dlo);
    } else {
        mm.H = linear_moments(d);
    }
    const float rho = p.rho0 + mm.drho();
    const float rho_inv = vrcp(rho);
    const float mx = PRECISE ? mm.H.mx + mm.L.mx : mm.H.mx;
    const float my = PRECISE ? mm.H.my + mm.L.my : mm.H.my;
    const float mz = PRECISE ? mm.H.mz + mm.L.mz : mm.H.mz;
    float og[21];
    NodeMacro<float> mac;
    induction_collide<float, PRECISE, S::COMP>(p, q, ql, og, rho_inv, mx, my, mz, in.Fx, in.Fy, in.Fz, in.FLx,
                                              in.FLy, in.FLz, mac);
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
    b.FL[n] = mac.FLx;
    b.FL[N + n] = mac.FLy;
    b.FL[2 * N + n] = mac.FLz;
}

// The update of fluid node n from its gathered pre-collision populations
// (d, dl: f and, for F32C, its low parts; q, ql: g): reads the lagged Lorentz
// force and the force field, collides, writes the node's own slots of the
// destination buffers (or the fields in MODE_FIELDS) and adds the residual
// terms of MODE_STEP_RESID to acc.
template <int ST, bool MHD, int MODE, bool DIR, int COLL>
__device__ __forceinline__ void node_from_sources(const StepParams& p, const StepBuffers& b, const FieldOut& fo,
                                                  uint32_t n, const float (&d)[19], const float (&dl)[19],
                                                  const float (&q)[21], const float (&ql)[21],
                                                  const NodeIn<float>& in, float (&acc)[7])
{
    using S = Store<ST>;
    using T = typename S::T;
    const size_t N = p.N;
    float om[19], og[21];
    NodeState<float> ns;
    node_update<float, ST, MHD, COLL>(p, d, dl, q, ql, in.FLx, in.FLy, in.FLz, in.Fx, in.Fy, in.Fz, MODE != MODE_FIELDS, om,
                                og, ns);

    if (MODE == MODE_FIELDS) {
        if (fo.rho) fo.rho[n] = ns.rho;
        if (fo.u) { fo.u[n] = ns.ux; fo.u[N + n] = ns.uy; fo.u[2 * N + n] = ns.uz; }
        if (MHD && fo.B) { fo.B[n] = ns.mac.Bx; fo.B[N + n] = ns.mac.By; fo.B[2 * N + n] = ns.mac.Bz; }
        return;
    }
    // f~ = f + om, written to the node's own slot of the other buffer
    T* __restrict__ fd = static_cast<T*>(b.fdst);
    [[maybe_unused]] SrBits rb(n, step_seed<ST>(b));
    if constexpr (S::COMP) {
        __half* __restrict__ fdl = reinterpret_cast<__half*>(fd + 19 * N);
#pragma unroll
        for (int a = 0; a < 19; ++a) {
            float nh, nl;
            comp_add(d[a], dl[a], om[a], nh, nl);
            fd[(size_t)a * N + n] = nh;
            fdl[(size_t)a * N + n] = S::cv_lo(nl);
        }
    } else if constexpr (DIR) {
#pragma unroll
        for (int a = 0; a < 19; ++a)
            static_cast<T*>(b.fdst_dir[a])[n] = store_cv<ST>(toscale<ST>(p, post_collision<ST>(d[a], om[a])), rb);
    } else {
#pragma unroll
        for (int a = 0; a < 19; ++a) fd[(size_t)a * N + n] = store_cv<ST>(toscale<ST>(p, post_collision<ST>(d[a], om[a])), rb);
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
            for (int a = 0; a < 21; ++a) gd[(size_t)a * N + n] = store_cv<ST>(toscale<ST>(p, q[a] + og[a]), rb);
        }
        b.FL[n] = ns.mac.FLx;
        b.FL[N + n] = ns.mac.FLy;
        b.FL[2 * N + n] = ns.mac.FLz;
    }
    if (MODE == MODE_STEP_RESID) {
        if (b.have_snap) {
            // u_hi - us_hi is exact for nearby values; the low parts add what
            // u_hi cannot resolve (0 without b.snap_lo)
            const float dx = (ns.ux - in.us0) + (ns.ulx - in.ul0);
            const float dy = (ns.uy - in.us1) + (ns.uly - in.ul1);
            const float dz = (ns.uz - in.us2) + (ns.ulz - in.ul2);
            acc[0] += dx * dx + dy * dy + dz * dz;
        }
        acc[1] += ns.ux * ns.ux + ns.uy * ns.uy + ns.uz * ns.uz;
        acc[2] += ns.drho;             // the mass is rho0 * (fluid nodes) + sum drho
        acc[3] += ns.jx;
        acc[4] += ns.jy;
        acc[5] += ns.jz;
        acc[6] += vnonfinite(ns.ux + ns.uy + ns.uz);
        b.usnap[n] = ns.ux;
        b.usnap[N + n] = ns.uy;
        b.usnap[2 * N + n] = ns.uz;
        if (b.snap_lo) {
            b.usnap[3 * N + n] = ns.ulx;
            b.usnap[4 * N + n] = ns.uly;
            b.usnap[5 * N + n] = ns.ulz;
        }
    }
}

// L2 prefetch for a step: the block b.pf_ahead positions later (one resident
// wave of the kernel, so it starts about when this one ends) will gather
// NODES consecutive nodes.  One thread per row asks L2 for that block's
// segment of the row (bulk prefetch, no data enters the SM): threads 0..18
// the f rows, with the direction's source shift and one node of halo on
// each side; with induction the 21 g rows (shifted like their D3Q7
// direction) and the 3 rows of the lagged Lorentz force; the force rows; on
// residual steps the 3 rows of the velocity snapshot.  Ranges are clamped to
// their rows and trimmed to 16-byte boundaries.  Measured on the
// 512 x 256 x 256 duct: BF16 paired step 0.4516 against 0.4829 ms, F32
// one-node step 0.869 against 0.888 ms.
template <int ST, int NODES, bool MHD, bool RESID>
__device__ __forceinline__ void prefetch_ahead(const StepParams& p, const StepBuffers& b)
{
    using T = typename Store<ST>::T;
    constexpr int NG = MHD ? 21 : 0, NL = MHD ? 3 : 0;
    // the compensated form: the FP16 low rows of f and g as well
    constexpr int NFC = Store<ST>::COMP ? 19 : 0, NGC = Store<ST>::COMP ? NG : 0;
    const int NS = RESID ? (b.snap_lo ? 6 : 3) : 0;
    const int t = threadIdx.x;
    if (b.pf_ahead <= 0 || t >= 19 + NG + NFC + NGC + NL + 3 + NS) return;
    const long long N = p.N;
    const long long nb = ((long long)blockIdx.x + b.pf_ahead) * NODES;
    if (nb >= N) return;
    uintptr_t row;               // start of the row
    size_t esz;                  // bytes per element
    long long shift = 0, halo = 0;
    int r = t;
    if (r < 19) {
        row = reinterpret_cast<uintptr_t>(b.fsrc) + (uintptr_t)r * (uintptr_t)N * sizeof(T);
        esz = sizeof(T);
        shift = p.doff[r] - (long long)r * N;            // -(e_x + e_y nx + e_z nx ny)
        halo = 1;
    } else if ((r -= 19) < NG) {
        const int a = r % 7;
        row = reinterpret_cast<uintptr_t>(b.gsrc) + (uintptr_t)r * (uintptr_t)N * sizeof(T);
        esz = sizeof(T);
        shift = p.doff[a] - (long long)a * N;
        halo = 1;
    } else if ((r -= NG) < NFC) {
        row = reinterpret_cast<uintptr_t>(b.fsrc) + (uintptr_t)19 * (uintptr_t)N * sizeof(T) +
              (uintptr_t)r * (uintptr_t)N * sizeof(__half);
        esz = sizeof(__half);
        shift = p.doff[r] - (long long)r * N;
        halo = 1;
    } else if ((r -= NFC) < NGC) {
        const int a = r % 7;
        row = reinterpret_cast<uintptr_t>(b.gsrc) + (uintptr_t)21 * (uintptr_t)N * sizeof(T) +
              (uintptr_t)r * (uintptr_t)N * sizeof(__half);
        esz = sizeof(__half);
        shift = p.doff[a] - (long long)a * N;
        halo = 1;
    } else if ((r -= NGC) < NL) {
        row = reinterpret_cast<uintptr_t>(b.FL) + (uintptr_t)r * (uintptr_t)N * sizeof(float);
        esz = sizeof(float);
    } else if ((r -= NL) < 3) {
        if (r >= p.force_ncomp || b.Ffield == nullptr) return;
        row = reinterpret_cast<uintptr_t>(b.Ffield) + (uintptr_t)r * (uintptr_t)N * sizeof(float);
        esz = sizeof(float);
    } else {
        r -= 3;
        row = reinterpret_cast<uintptr_t>(b.usnap) + (uintptr_t)r * (uintptr_t)N * sizeof(float);
        esz = sizeof(float);
    }
    const long long s0 = nb + shift - halo, s1 = nb + NODES + shift + halo;
    uintptr_t lo = row + (uintptr_t)(s0 < 0 ? 0 : s0) * esz;
    uintptr_t hi = row + (uintptr_t)(s1 > N ? N : s1) * esz;
    lo = (lo + 15) & ~(uintptr_t)15;
    hi &= ~(uintptr_t)15;
    if (hi > lo)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((uint32_t)(hi - lo)) : "memory");
}

template <int ST, bool MHD, int MODE, int COLL = 0>
__device__ __forceinline__ void step_body(const StepParams& p, const StepBuffers& b, const FieldOut& fo)
{
    if (b.stop != nullptr && *b.stop) return;   // converged solve: remaining steps of the chunk are skipped
    if constexpr (MODE != MODE_FIELDS) advance_seed<ST>(b);
    // with induction only for F32 storage: coupled F32 step 0.1241 against
    // 0.1382 ms (half a wave ahead: 0.1200 ms), coupled BF16 step 0.0845
    // against 0.0829 ms (half a wave ahead: 0.0841 ms)
    if constexpr (MODE != MODE_FIELDS && (!MHD || ST == ST_F32))
        prefetch_ahead<ST, STEP_THREADS, MHD, MODE == MODE_STEP_RESID>(p, b);
    const uint32_t i = blockIdx.x * STEP_THREADS + threadIdx.x;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (MODE != MODE_STEP_RESID && !(i < p.N)) return;
    // per-direction bases for the plain BF16 steps only: measured on one
    // box against the plain addressing, BF16 0.598 vs 0.612 ms, but F16 0.679
    // vs 0.631 ms, F32 1.058 vs 0.898 ms (with induction they raise its
    // register count past a block per SM) and the BF16 residual step 0.914
    // vs 0.842 ms; the coupled BF16 step keeps 80 registers with them: f
    // 1.2586 against 1.3008 ms on the 512 x 256 x 256 duct (the 21 g rows
    // from such bases too: 1.3385 ms)
    scalar_node_step<ST, MHD, MODE, false, COLL == 0 && base_storage(ST) == ST_BF16 && MODE == MODE_STEP, false,
                     COLL>(p, b, fo, i, acc);
    if (MODE == MODE_STEP_RESID) block_partials<STEP_THREADS>(acc, b.partials);
}

template <int ST, bool MHD, int MODE>
__global__ void __launch_bounds__(STEP_THREADS) step_kernel(const StepParams p, const StepBuffers b, const FieldOut fo)
{
    step_body<ST, MHD, MODE>(p, b, fo);
}

// The preconditioned SRT-LBE step (Sec. 3.1; COLL = 1, or 2 with the naive
// source), one node per thread; the collision operator of
// glbe_params.collision = 1 or 2.
template <int ST, bool MHD, int MODE, int COLL>
__global__ void __launch_bounds__(STEP_THREADS) step_kernel_srt(const StepParams p, const StepBuffers b, const FieldOut fo)
{
    step_body<ST, MHD, MODE, COLL>(p, b, fo);
}

// The plain flow step held to MINB resident blocks of 256 threads per SM:
// with 16-bit storage it fits 48 registers (five blocks, 40 warps, instead of
// four).  A separate kernel because stating a minimum at all (even one block)
// changes the register allocation of the forms left free.  F32 stays free:
// held to 64 registers (four blocks) it measured slower than at 80 (three).
template <int ST, int MINB>
__global__ void __launch_bounds__(STEP_THREADS, MINB)
    step_kernel_dense(const StepParams p, const StepBuffers b, const FieldOut fo)
{
    step_body<ST, false, MODE_STEP>(p, b, fo);
}
template <int ST>
constexpr int step_dense_blocks()
{
    // 16-bit: 5 blocks (48 registers); F32C: 3 (80 registers, 32 B spilled);
    // 0: the free kernel
    return (base_storage(ST) == ST_BF16 || base_storage(ST) == ST_F16) ? 5 : (ST == ST_F32C ? 3 : 0);
}

// The coupled compensated step in two passes per thread (the batch's form):
// pass 1 gathers f and g, runs the induction part and writes g~ and this
// step's Lorentz force; pass 2 gathers f again (from L1 / L2) and runs the
// flow update with F = F_ext + F_L.  The arithmetic and its order are the
// one-pass update's, so the result is bit for bit the same, but the
// registers of the two parts are not live together: 172 registers in one
// pass (one block of 256 per SM) against at most 128 here (F32C; the F32
// and BF16 residual steps are held to three blocks).
template <int ST, int MODE>
__global__ void __launch_bounds__(STEP_THREADS, ST == ST_F32C ? 2 : 3)
    step_kernel_coupled2(const StepParams p, const StepBuffers b, const FieldOut fo)
{
    if (b.stop != nullptr && *b.stop) return;
    prefetch_ahead<ST, STEP_THREADS, true, MODE == MODE_STEP_RESID>(p, b);
    const uint32_t i = blockIdx.x * STEP_THREADS + threadIdx.x;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (MODE != MODE_STEP_RESID && !(i < p.N)) return;
    coupled_induction_pass<ST, false>(p, b, i);
    scalar_node_step<ST, false, MODE, false, false, true>(p, b, fo, i, acc);
    if (MODE == MODE_STEP_RESID) block_partials<STEP_THREADS>(acc, b.partials);
}

// The update of the fluid node pair (n0, n0 + 1) from its gathered
// pre-collision populations (packed FP32x2): the counterpart of
// node_from_sources for two nodes; adds the pair's residual terms to acc.
// DIR: the f stores address the per-direction bases b.fdst_dir.
template <int ST, bool MHD, int MODE, bool DIR = false>
__device__ __forceinline__ void pair_from_sources(const StepParams& p, const StepBuffers& b, uint32_t n0,
                                                  const F2 (&d)[19], const F2 (&dl)[19], const F2 (&q)[21],
                                                  const F2 (&ql)[21], const NodeIn<F2>& in, float (&acc)[7])
{
    using S = Store<ST>;
    using T = typename S::T;
    const size_t N = p.N;
    F2 om[19], og[21];
    NodeState<F2> ns;
    node_update<F2, ST, MHD>(p, d, dl, q, ql, in.FLx, in.FLy, in.FLz, in.Fx, in.Fy, in.Fz, true, om, og, ns);

    T* __restrict__ fd = static_cast<T*>(b.fdst);
    [[maybe_unused]] SrBits rb(n0, step_seed<ST>(b));
    if constexpr (S::COMP) {
        __half* __restrict__ fdl = reinterpret_cast<__half*>(fd + 19 * N);
#pragma unroll
        for (int a = 0; a < 19; ++a) {
            F2 nh, nl;
            comp_add(d[a], dl[a], om[a], nh, nl);
            S::st2(fd + (size_t)a * N + n0, nh);
            S::st2_lo(fdl + (size_t)a * N + n0, nl);
        }
    } else if constexpr (DIR) {
#pragma unroll
        for (int a = 0; a < 19; ++a)
            store_pair<ST>(static_cast<T*>(b.fdst_dir[a]) + n0, toscale<ST>(p, post_collision<ST>(d[a], om[a])), rb);
    } else {
#pragma unroll
        for (int a = 0; a < 19; ++a)
            store_pair<ST>(fd + (size_t)a * N + n0, toscale<ST>(p, post_collision<ST>(d[a], om[a])), rb);
    }
    if (MHD) {
        T* __restrict__ gd = static_cast<T*>(b.gdst);
        if constexpr (S::COMP) {
            __half* __restrict__ gdl = reinterpret_cast<__half*>(gd + 21 * N);
#pragma unroll
            for (int a = 0; a < 21; ++a) {
                F2 nh, nl;
                comp_add(q[a], ql[a], og[a], nh, nl);
                S::st2(gd + (size_t)a * N + n0, nh);
                S::st2_lo(gdl + (size_t)a * N + n0, nl);
            }
        } else {
#pragma unroll
            for (int a = 0; a < 21; ++a) store_pair<ST>(gd + (size_t)a * N + n0, toscale<ST>(p, q[a] + og[a]), rb);
        }
        *reinterpret_cast<float2*>(b.FL + n0) = ns.mac.FLx.v;
        *reinterpret_cast<float2*>(b.FL + N + n0) = ns.mac.FLy.v;
        *reinterpret_cast<float2*>(b.FL + 2 * N + n0) = ns.mac.FLz.v;
    }
    if (MODE == MODE_STEP_RESID) {
        float2* us = reinterpret_cast<float2*>(b.usnap + n0);
        float2* vs = reinterpret_cast<float2*>(b.usnap + N + n0);
        float2* ws = reinterpret_cast<float2*>(b.usnap + 2 * N + n0);
        if (b.have_snap) {
            const F2 dx = (ns.ux - in.us0) + (ns.ulx - in.ul0);
            const F2 dy = (ns.uy - in.us1) + (ns.uly - in.ul1);
            const F2 dz = (ns.uz - in.us2) + (ns.ulz - in.ul2);
            acc[0] += lane_sum(dx * dx + dy * dy + dz * dz);
        }
        acc[1] += lane_sum(ns.ux * ns.ux + ns.uy * ns.uy + ns.uz * ns.uz);
        acc[2] += lane_sum(ns.drho);
        acc[3] += lane_sum(ns.jx);
        acc[4] += lane_sum(ns.jy);
        acc[5] += lane_sum(ns.jz);
        acc[6] += vnonfinite(ns.ux + ns.uy + ns.uz);
        *us = ns.ux.v;
        *vs = ns.uy.v;
        *ws = ns.uz.v;
        if (b.snap_lo) {
            *reinterpret_cast<float2*>(b.usnap + 3 * N + n0) = ns.ulx.v;
            *reinterpret_cast<float2*>(b.usnap + 4 * N + n0) = ns.uly.v;
            *reinterpret_cast<float2*>(b.usnap + 5 * N + n0) = ns.ulz.v;
        }
    }
}

// Interior gather of f for the pair (x0, x0 + 1), x0 even, on a row whose
// nodes are all interior (x periodic, no wall among the neighbours, no y or z
// seam), from the per-direction bases b.fsrc_dir.  Direction a with x-shift
// e_x reads the aligned pair at fsrc_dir[a] + n0 + e_x, the source row's
// (x0, x0 + 1).  e_x = 0: the pair's own sources.  e_x = +1: node x0 + 1
// takes x0, node x0 takes x0 - 1 from the left lane's pair (a load of its own
// at a warp start, and across the x seam at x0 = 0).  e_x = -1: node x0 takes
// x0 + 1, node x0 + 1 takes x0 + 2 from the right lane (a load of its own at a
// warp end, and across the seam at x0 + 2 = nx).  Every lane of the warp
// takes this path or none (the shuffles), and every load is in bounds: the
// row's neighbour rows exist and are fluid.
template <int ST>
__device__ __forceinline__ void load_f_pair_interior(const StepParams& p, const StepBuffers& b, uint32_t n0, int x0,
                                                     F2 (&d)[19])
{
    using S = Store<ST>;
    using T = typename S::T;
    const int lane = threadIdx.x & 31;
    const bool left_own = lane == 0 || x0 == 0;
    const bool right_own = lane == 31 || x0 + 2 == p.nx;
    const long long nl = (long long)n0 + (x0 == 0 ? p.nx : 0);             // source x0 - 1 of node x0
    const long long nr = (long long)n0 + 1 + (x0 + 2 == p.nx ? -p.nx : 0);  // source x0 + 2 of node x0 + 1
#pragma unroll
    for (int a = 0; a < 19; ++a) {
        const T* __restrict__ base = static_cast<const T*>(b.fsrc_dir[a]);
        const int ex = dir_ex(a);
        const F2 v = unscale<ST>(p, S::ld2(base + ((long long)n0 + ex)));
        if (ex > 0) {
            const float t = __shfl_up_sync(0xffffffffu, v.v.y, 1);
            const float left = left_own ? unscale<ST>(p, S::ld(base + nl)) : t;
            d[a] = F2(left, v.v.x);
        } else if (ex < 0) {
            const float t = __shfl_down_sync(0xffffffffu, v.v.x, 1);
            const float right = right_own ? unscale<ST>(p, S::ld(base + nr)) : t;
            d[a] = F2(v.v.y, right);
        } else {
            d[a] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Paired kernel: two x-adjacent nodes per thread (x periodic, nx even)
// ---------------------------------------------------------------------------
template <int ST, bool MHD, int MODE>
__device__ __forceinline__ void pair_step_body(const StepParams& p, const StepBuffers& b)
{
    using S = Store<ST>;
    using T = typename S::T;
    if (b.stop != nullptr && *b.stop) return;
    advance_seed<ST>(b);
    if constexpr (!MHD && !S::COMP) prefetch_ahead<ST, 2 * PAIR_THREADS, false, MODE == MODE_STEP_RESID>(p, b);
    const uint32_t npairs = p.N >> 1;
    const uint32_t i = blockIdx.x * PAIR_THREADS + threadIdx.x;
    const bool inb = i < npairs;
    // lanes past the end mirror the last pair so that every lane takes part in
    // the shuffles; they write nothing
    const uint32_t n0 = 2u * (inb ? i : npairs - 1u);
    F2 d[19], dl[19], q[21], ql[21];
    bool fluid = inb;
    // interior rows (flow, 16-bit or F32 storage): fixed offsets, decided for
    // the whole warp so that every lane takes part in the shuffles
    constexpr bool FAST = !MHD && !S::COMP;
    int wp = 0, wm = 0;
    const bool interior = FAST && __all_sync(0xffffffffu, is_interior(p, n0, wp, wm));
    if (FAST && interior) {
        const int x0 = (int)(n0 - fdiv(n0, p.div_nx) * (uint32_t)p.nx);
        load_f_pair_interior<ST>(p, b, n0, x0, d);
    } else {
        const GeoP gp = make_geo_pair(p, n0);
        fluid = inb && !gp.g.solid;
        load_f_pair<ST>(p, static_cast<const T*>(b.fsrc), gp, d, dl);
        if (MHD) load_g_pair<ST>(p, static_cast<const T*>(b.gsrc), gp, q, ql);
    }

    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (fluid)
        pair_from_sources<ST, MHD, MODE, FAST>(p, b, n0, d, dl, q, ql, pair_inputs<MHD, MODE>(p, b, n0), acc);
    if (MODE == MODE_STEP_RESID) block_partials<PAIR_THREADS>(acc, b.partials);
}

template <int ST, bool MHD, int MODE>
__global__ void __launch_bounds__(PAIR_THREADS) step_pair_kernel(const StepParams p, const StepBuffers b)
{
    pair_step_body<ST, MHD, MODE>(p, b);
}

// The 16-bit flow forms held to MINB resident blocks of 128 threads per SM.
// The paired kernel is latency-bound: at its free 80 registers 24 warps per
// SM; held to 72 (7 blocks, 28 warps, a few spilled bytes) the BF16 plain
// step took 0.488 instead of 0.527 ms and the residual step 0.656 instead of
// 0.741 ms, measured alternately on one box (F16: 0.517 against 0.519 ms).
// Held to 6 blocks it was slower than free: stating a minimum changes the
// register allocation, hence a kernel of its own.
template <int ST, int MODE, int MINB>
__global__ void __launch_bounds__(PAIR_THREADS, MINB) step_pair_kernel_dense(const StepParams p, const StepBuffers b)
{
    pair_step_body<ST, false, MODE>(p, b);
}
// Held to 8 blocks (64 registers, 80 B spilled) the BF16 plain step took
// 0.491 against 0.484 ms, the F16 plain step 0.498 against 0.509 ms.
template <int ST, int MODE>
constexpr int pair_dense_blocks()
{
    if (base_storage(ST) == ST_F16) return MODE == MODE_STEP ? 8 : 7;
    // F32: plain step 4 (128 registers, 56 B spilled); the residual step stays
    // free (held to 4 it spills 176 B: 10 levels took 8.59 against 8.37 ms)
    if (ST == ST_F32) return MODE == MODE_STEP ? 4 : 0;
    return base_storage(ST) == ST_BF16 ? 7 : 0;   // 0: the free kernel
}

// The paired kernel serves x-periodic grids with an even nx: when asked for
// (variant 2), or by the automatic choice (variant 0) for the 16-bit flow
// steps, where it measured faster on the 512 x 256 x 256 duct: its interior
// rows issue about 310 instructions per node against 538 for the one-node
// kernel.  Plain step, BF16 0.485 against 0.598 ms, F16 0.509 against 0.631
// ms; residual step, BF16 0.655 against 0.838 ms.  F32 takes it too since
// the interior pair path: held to 4 blocks of 128 (128 registers) the plain
// step is 0.801 against 0.938 ms for one node per thread (at 142 registers,
// 3 blocks, it had measured 1.17 against 0.89 ms before that path).  The
// coupled forms and F32C have no interior pair path.
inline bool pair_eligible(const StepParams& p, bool mhd, int mode)
{
    if ((p.nx % 2 != 0) || p.wlo[0] || p.whi[0] || mode == MODE_FIELDS) return false;
    if (p.variant == 2) return true;
    if (p.variant != 0 || mhd) return false;
    return base_storage(p.storage) == ST_F16 || base_storage(p.storage) == ST_BF16 || p.storage == ST_F32;
}

// ---------------------------------------------------------------------------
// State transfer (not on the hot path; scalar)
// ---------------------------------------------------------------------------
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
        fs[s_] = Store<ST>::cv(toscale<ST>(p, df[(size_t)(a) * N + i]));                    \
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
        bj[s_] = Store<ST>::cv(toscale<ST>(p, v_));                                                  \
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

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
}  // namespace glbe
#include "glbe_tile.cuh"
#include "glbe_cavity.cuh"
namespace glbe {

// b with its per-direction bases filled (addresses formed as integers: a
// base may lie before the buffer, only base + n is ever read)
template <int ST>
StepBuffers with_dir_bases(const StepParams& p, StepBuffers b)
{
    const size_t e = sizeof(typename Store<ST>::T);
    for (int a = 0; a < 19; ++a) {
        b.fsrc_dir[a] = b.fsrc ? reinterpret_cast<const void*>(reinterpret_cast<uintptr_t>(b.fsrc) +
                                                               (uintptr_t)((long long)e * p.doff[a]))
                               : nullptr;
        b.fdst_dir[a] = b.fdst ? reinterpret_cast<void*>(reinterpret_cast<uintptr_t>(b.fdst) + e * (size_t)a * p.N)
                               : nullptr;
    }
    return b;
}

// Blocks of `kernel` resident on the whole device at once (one wave), from
// which the L2 prefetch distance is set.  Computed once per kernel (the first
// device that launches it); 0, and so no prefetch, if the runtime cannot tell.
// Measured on the 512 x 256 x 256 duct: the one-node plain steps prefetch one
// wave ahead (F32 0.875 ms; half a wave 0.886, two waves 0.957); the paired
// steps, the coupled steps and the residual steps half a wave ahead (BF16 plain 0.4528 against
// 0.4555 ms at one wave, BF16 residual 0.613 against 0.643 ms; two waves
// 0.505 ms, the prefetched rows then leave L2 before they are read).
template <class K>
long long resident_wave(K kernel, int threads)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) return 0;
    return (long long)sms * per_sm;
}

// Blocks of the one-pass coupled one-node kernel resident at once.  The
// two-pass form pays off on grids of several such waves; on a grid of about
// one wave its second gather only adds latency (F32C, 64 x 64 x 8 duct:
// 10.4 against 8.5 us per step; 64^3: 37.0 against 39.2 us).
template <int ST, int MODE>
long long one_pass_wave()
{
    static const long long w = resident_wave(step_kernel<ST, true, MODE>, STEP_THREADS);
    return w;
}

template <int ST, bool MHD, int MODE>
cudaError_t launch_mode(const StepParams& p, const StepBuffers& b_in, const FieldOut& fo, cudaStream_t st,
                        unsigned* nblocks)
{
    StepBuffers b = with_dir_bases<ST>(p, b_in);
    b.pf_ahead = 0;
    if constexpr (ST == ST_F32 || ST == ST_F32C || ST == ST_BF16) {
        if (p.cavity) {   // fluid box and / or moving lid: the one-node cavity kernel
            const unsigned grid = (unsigned)(((size_t)p.N + STEP_THREADS - 1) / STEP_THREADS);
            if (MODE != MODE_FIELDS && p.collision == 1) {
                if constexpr (ST == ST_F32) cavity_kernel<ST, MHD, MODE, 1><<<grid, STEP_THREADS, 0, st>>>(p, b, fo);
            } else if (MHD && (ST == ST_F32 || ST == ST_F32C) && MODE != MODE_FIELDS && p.variant == 0) {
                if constexpr (MHD && (ST == ST_F32 || ST == ST_F32C) && MODE != MODE_FIELDS)
                    cavity_kernel_coupled2<ST, MODE><<<grid, STEP_THREADS, 0, st>>>(p, b, fo);
            } else {
                cavity_kernel<ST, MHD, MODE, 0><<<grid, STEP_THREADS, 0, st>>>(p, b, fo);
            }
            if (nblocks) *nblocks = grid;
            return cudaGetLastError();
        }
    }
    if constexpr (MODE != MODE_FIELDS && (ST == ST_F32 || ST == ST_F32C || ST == ST_BF16)) {
        if (p.collision != 0) {   // preconditioned SRT-LBE: one node per thread
            const unsigned grid = (unsigned)(((size_t)p.N + STEP_THREADS - 1) / STEP_THREADS);
            if (p.collision == 1) step_kernel_srt<ST, MHD, MODE, 1><<<grid, STEP_THREADS, 0, st>>>(p, b, fo);
            else step_kernel_srt<ST, MHD, MODE, 2><<<grid, STEP_THREADS, 0, st>>>(p, b, fo);
            if (nblocks) *nblocks = grid;
            return cudaGetLastError();
        }
    }
    if constexpr (ST != ST_F32C && !Store<ST>::SR && MODE != MODE_FIELDS) {
        if (p.variant == 3 && tile_eligible(p, MODE)) return launch_tile<ST, MHD, MODE, false>(p, b, st, nblocks);
        if (p.variant == 4 && tile_eligible(p, MODE)) return launch_tile<ST, MHD, MODE, true>(p, b, st, nblocks);
    }
    if (pair_eligible(p, MHD, MODE)) {
        const unsigned grid = (unsigned)(((size_t)(p.N / 2) + PAIR_THREADS - 1) / PAIR_THREADS);
        constexpr int PMINB = pair_dense_blocks<ST, MODE>();
        if constexpr (!MHD && MODE != MODE_FIELDS && PMINB > 0) {
            static const long long wave = resident_wave(step_pair_kernel_dense<ST, MODE, PMINB>, PAIR_THREADS);
            b.pf_ahead = wave / 2;
            step_pair_kernel_dense<ST, MODE, PMINB><<<grid, PAIR_THREADS, 0, st>>>(p, b);
        } else {
            static const long long wave = resident_wave(step_pair_kernel<ST, MHD, MODE>, PAIR_THREADS);
            b.pf_ahead = wave / 2;
            step_pair_kernel<ST, MHD, MODE><<<grid, PAIR_THREADS, 0, st>>>(p, b);
        }
        if (nblocks) *nblocks = grid;
    } else {
        const unsigned grid = (unsigned)(((size_t)p.N + STEP_THREADS - 1) / STEP_THREADS);
        constexpr int MINB = step_dense_blocks<ST>();
        if constexpr (!MHD && MODE == MODE_STEP && MINB > 0) {
            static const long long wave = resident_wave(step_kernel_dense<ST, MINB>, STEP_THREADS);
            b.pf_ahead = wave;
            step_kernel_dense<ST, MINB><<<grid, STEP_THREADS, 0, st>>>(p, b, fo);
        } else if (MHD && (ST == ST_F32C || ((ST == ST_F32 || ST == ST_BF16) && MODE == MODE_STEP_RESID)) &&
                   MODE != MODE_FIELDS &&
                   p.variant == 0 && grid > 2 * one_pass_wave<ST, MODE>()) {
            // F32C: both steps; F32: the residual step only (its one-pass form
            // spills; the plain F32 step keeps one pass, 1.853 against 1.894 ms
            // on the 512 x 256 x 256 coupled duct, while the residual level
            // drops from about 3.3 to 2.3 ms); BF16: the residual step only
            // (one pass: 90 registers, two blocks per SM; two: 80, three
            // blocks; the residual level about 1.90 -> 1.73 ms)
            if constexpr (MHD && (ST == ST_F32C || ((ST == ST_F32 || ST == ST_BF16) && MODE == MODE_STEP_RESID)) &&
                          MODE != MODE_FIELDS) {
                // L2 prefetch half a wave ahead, on grids of several waves
                // (on a 48^3 duct it cost 0.0164 -> 0.0192 ms; on 144^3 it
                // took the step from 0.3235 to 0.3132 ms)
                // (not the BF16 residual step: the coupled BF16 steps are
                // slower with it)
                static const long long wave = resident_wave(step_kernel_coupled2<ST, MODE>, STEP_THREADS);
                b.pf_ahead = ST != ST_BF16 && (long long)grid > 4 * wave ? wave / 2 : 0;
                step_kernel_coupled2<ST, MODE><<<grid, STEP_THREADS, 0, st>>>(p, b, fo);
            }
        } else {
            static const long long wave = resident_wave(step_kernel<ST, MHD, MODE>, STEP_THREADS);
            b.pf_ahead = (MHD || MODE == MODE_STEP_RESID) ? wave / 2 : wave;
            step_kernel<ST, MHD, MODE><<<grid, STEP_THREADS, 0, st>>>(p, b, fo);
        }
        if (nblocks) *nblocks = grid;
    }
    return cudaGetLastError();
}

template <int ST>
cudaError_t launch_step_t(bool mhd, int mode, const StepParams& p, const StepBuffers& b, const FieldOut& fo,
                          cudaStream_t st, unsigned* nblocks)
{
    if (mhd) {
        if (mode == MODE_STEP) return launch_mode<ST, true, MODE_STEP>(p, b, fo, st, nblocks);
        if (mode == MODE_STEP_RESID) return launch_mode<ST, true, MODE_STEP_RESID>(p, b, fo, st, nblocks);
        return launch_mode<ST, true, MODE_FIELDS>(p, b, fo, st, nblocks);
    }
    if (mode == MODE_STEP) return launch_mode<ST, false, MODE_STEP>(p, b, fo, st, nblocks);
    if (mode == MODE_STEP_RESID) return launch_mode<ST, false, MODE_STEP_RESID>(p, b, fo, st, nblocks);
    return launch_mode<ST, false, MODE_FIELDS>(p, b, fo, st, nblocks);
}

template <int ST>
int tile_wait_error_t()
{
    return tile_wait_error_read();
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
