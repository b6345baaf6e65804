// glbe_adjoint.cuh -- reverse (transposed-Jacobian) form of one node's
// collision, written by hand from the forward arithmetic of glbe_kernels.cuh.
//
// Forward, per node (Eqs. ppostcollision, prelax_term, precondhydrofields of
// arXiv:0809.4730; Sec. 4 for the induction lattice):
//   rho = rho0 + sum d,  m = sum d e,  F = F_ext + F_L,  j = m + F/(2 gamma),
//   u = j/rho,  n_k = (T d)_k - eq_k(rho, j) on the relaxed rows,
//   delta_k = -s_k n_k + (1 - s_k/2) S_k(F, u),  delta_{3,5,7} = F/gamma,
//   f~ = d + T^t diag(1/|row_k|^2) delta.
// Reverse, with v = dL/df~ and mu = diag(1/|row_k|^2) T v (= dL/ddelta):
//   dL/dn_k = -s_k mu_k,  dL/dS_k = (1 - s_k/2) mu_k,  dL/dF += mu_{3,5,7}/gamma,
//   dL/drho and dL/dj collect the equilibrium and source derivatives,
//   dL/dd = v + T^t y with y_k = -s_k mu_k on the relaxed rows and
//   y_0 = dL/drho, y_{3,5,7} = dL/dj (the rows of T that give rho and m).
// The induction part is reversed through F_L = J x B, J = Jc (Lneq
// differences), Lneq = M - Lambda^eq(u0, B), u0 = (m + (F_ext + F_L^prev)/
// (2 gamma))/rho, B = B0 + sum g, and g~ = g + omega (g^eq - g).
#pragma once
#include "glbe_kernels.cuh"

namespace glbe {

// Cotangents leaving one node's reverse step.
struct NodeAdjoint {
    float d[19];     // dL/d(pre-collision df)
    float q[21];     // dL/d(pre-collision dg)
    float FLp[3];    // dL/d(lagged Lorentz force)
    float F[3];      // dL/d(external force at the node)
};

// Columns of T applied to y (Tt y)_a, the same group structure as the
// inverse transform of the forward collision (without the 1/|row|^2).
__device__ __forceinline__ void apply_Tt(const float (&y)[19], float (&out)[19])
{
    out[0] = y[0] - 30.f * y[1] + 12.f * y[2];
    const float A = y[0] - 11.f * y[1] - 4.f * y[2];
    const float X9 = 2.f * y[9] - 4.f * y[10];
    const float Y9 = 2.f * y[10] - y[9];
    const float W11 = y[11] - 2.f * y[12];
    float t = y[3] - 4.f * y[4];
    out[1] = A + X9 + t;
    out[2] = A + X9 - t;
    t = y[5] - 4.f * y[6];
    out[3] = A + Y9 + W11 + t;
    out[4] = A + Y9 + W11 - t;
    t = y[7] - 4.f * y[8];
    out[5] = A + Y9 - W11 + t;
    out[6] = A + Y9 - W11 - t;
    const float Dg = y[0] + 8.f * y[1] + y[2];
    const float P = y[9] + y[10], Q = y[11] + y[12];
    {
        const float b = Dg + P + Q, ax = y[3] + y[4] + y[16], by = y[5] + y[6] - y[17];
        out[7] = b + ax + by + y[13];
        out[8] = b - ax + by - y[13];
        out[9] = b + ax - by - y[13];
        out[10] = b - ax - by + y[13];
    }
    {
        const float b = Dg + P - Q, ax = y[3] + y[4] - y[16], bz = y[7] + y[8] + y[18];
        out[11] = b + ax + bz + y[15];
        out[12] = b - ax + bz - y[15];
        out[13] = b + ax - bz - y[15];
        out[14] = b - ax - bz + y[15];
    }
    {
        const float b = Dg - 2.f * P, ay = y[5] + y[6] + y[17], bz = y[7] + y[8] - y[18];
        out[15] = b + ay + bz + y[14];
        out[16] = b - ay + bz - y[14];
        out[17] = b + ay - bz - y[14];
        out[18] = b - ay - bz + y[14];
    }
}

// Forward quantities of one node that its reverse step needs, at the
// linearisation point: 1/rho, j = m + F/(2 gamma), the total force F and,
// with the induction lattice, B, u0 and the current J.  The reverse step is
// linear in the cotangents with coefficients formed from these 16 values
// alone, so a fixed linearisation point (the steady adjoint) can keep them
// resident instead of gathering the 40 populations again every iteration.
struct NodeLin {
    float ri;
    float j[3];
    float F[3];
    float B[3], u0[3], Jv[3];   // induction lattice only
};

// Rows of NodeLin stored per node ([rows][N] FP32): ri, j, F; + B, u0, J.
constexpr int LIN_ROWS_FLOW = 7;
constexpr int LIN_ROWS_MHD = 16;

// The forward part of the node update at (d, q, FLp, Fext): the moments, the
// induction lattice's B, u0, J and the Lorentz force, and j.
template <bool MHD>
__device__ __forceinline__ NodeLin node_linearise(const StepParams& p, const float (&d)[19], const float (&q)[21],
                                                  const float (&FLp)[3], const float (&Fext)[3])
{
    // (the precise FP32 moments of the forward step are not needed here: the
    // reverse is linear in the cotangents)
    NodeLin L;
    float drho = 0.f;
#pragma unroll
    for (int a = 0; a < 19; ++a) drho += d[a];
    const float rho = p.rho0 + drho, ri = 1.0f / rho;
    const float mx = (d[1] - d[2]) + (d[7] - d[8] + d[9] - d[10]) + (d[11] - d[12] + d[13] - d[14]);
    const float my = (d[3] - d[4]) + (d[7] + d[8] - d[9] - d[10]) + (d[15] - d[16] + d[17] - d[18]);
    const float mz = (d[5] - d[6]) + (d[11] + d[12] - d[13] - d[14]) + (d[15] + d[16] - d[17] - d[18]);
    const float hg = 0.5f * p.inv_gamma;
    float F[3] = {Fext[0], Fext[1], Fext[2]};
    // induction forward
    float B[3] = {0.f, 0.f, 0.f}, u0[3] = {0.f, 0.f, 0.f}, Jv[3] = {0.f, 0.f, 0.f};
    if (MHD) {
        float b[3] = {0.f, 0.f, 0.f};
        for (int j = 0; j < 3; ++j)
            for (int a = 0; a < 7; ++a) b[j] += q[j * 7 + a];
        for (int c = 0; c < 3; ++c) B[c] = p.B0[c] + b[c];
        u0[0] = (mx + hg * (Fext[0] + FLp[0])) * ri;
        u0[1] = (my + hg * (Fext[1] + FLp[1])) * ri;
        u0[2] = (mz + hg * (Fext[2] + FLp[2])) * ri;
        const float c = p.conv_coef;
        const float Lxy = c * (u0[0] * B[1] - B[0] * u0[1]);
        const float Lxz = c * (u0[0] * B[2] - B[0] * u0[2]);
        const float Lyz = c * (u0[1] * B[2] - B[1] * u0[2]);
        const float Nxy = (q[8] - q[9]) - Lxy, Nyx = (q[3] - q[4]) + Lxy;
        const float Nxz = (q[15] - q[16]) - Lxz, Nzx = (q[5] - q[6]) + Lxz;
        const float Nyz = (q[17] - q[18]) - Lyz, Nzy = (q[12] - q[13]) + Lyz;
        Jv[0] = p.J_coef * (Nyz - Nzy);
        Jv[1] = p.J_coef * (Nzx - Nxz);
        Jv[2] = p.J_coef * (Nxy - Nyx);
        F[0] += Jv[1] * B[2] - Jv[2] * B[1];
        F[1] += Jv[2] * B[0] - Jv[0] * B[2];
        F[2] += Jv[0] * B[1] - Jv[1] * B[0];
    }
    L.ri = ri;
    L.j[0] = mx + hg * F[0];
    L.j[1] = my + hg * F[1];
    L.j[2] = mz + hg * F[2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        L.F[c] = F[c];
        L.B[c] = B[c];
        L.u0[c] = u0[c];
        L.Jv[c] = Jv[c];
    }
    return L;
}

// Reverse of the whole node update (node_update + the stores f~ = d + om,
// g~ = q + og, F_L stored) at the linearisation point L.
// vf, vg, vFL: cotangents of f~, g~ and the stored F_L; wu: cotangent of the
// node's velocity u (the objective's weight, 0 for a plain step).
template <bool MHD>
__device__ __forceinline__ void node_reverse_at(const StepParams& p, const NodeLin& L, const float (&vf)[19],
                                                const float (&vg)[21], const float (&vFL)[3], const float (&wu)[3],
                                                NodeAdjoint& out)
{
    const float ri = L.ri;
    const float hg = 0.5f * p.inv_gamma;
    const float F[3] = {L.F[0], L.F[1], L.F[2]};
    const float B[3] = {L.B[0], L.B[1], L.B[2]};
    const float u0[3] = {L.u0[0], L.u0[1], L.u0[2]};
    const float Jv[3] = {L.Jv[0], L.Jv[1], L.Jv[2]};
    const float j[3] = {L.j[0], L.j[1], L.j[2]};
    const float u[3] = {j[0] * ri, j[1] * ri, j[2] * ri};
    const float ig = p.inv_gamma, ig2 = p.inv_gamma2, gri = ig * ri;
    const float jj = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
    const float e9 = (3.f * j[0] * j[0] - jj) * gri, e11 = (j[1] * j[1] - j[2] * j[2]) * gri;
    const float e13 = j[0] * j[1] * gri, e14 = j[1] * j[2] * gri, e15 = j[0] * j[2] * gri;

    // ---- reverse of the flow collision
    // mu_k = (T v)_k / |row_k|^2
    float vv[19];
#pragma unroll
    for (int a = 0; a < 19; ++a) vv[a] = vf[a];
    const Lin<float> Tv = linear_moments(vv);
    float mu[19];
    mu[0] = Tv.drho / 19.f;
    mu[1] = Tv.M1 / 2394.f;
    mu[2] = Tv.M2 / 252.f;
    mu[3] = Tv.mx / 10.f;
    mu[4] = Tv.Qx / 40.f;
    mu[5] = Tv.my / 10.f;
    mu[6] = Tv.Qy / 40.f;
    mu[7] = Tv.mz / 10.f;
    mu[8] = Tv.Qz / 40.f;
    mu[9] = Tv.P9 / 36.f;
    mu[10] = Tv.P10 / 72.f;
    mu[11] = Tv.P11 / 12.f;
    mu[12] = Tv.P12 / 24.f;
    mu[13] = Tv.P13 / 4.f;
    mu[14] = Tv.P14 / 4.f;
    mu[15] = Tv.P15 / 4.f;
    mu[16] = Tv.P16 / 8.f;
    mu[17] = Tv.P17 / 8.f;
    mu[18] = Tv.P18 / 8.f;
    float nu_[19], sg[19];
#pragma unroll
    for (int k = 0; k < 19; ++k) {
        nu_[k] = -p.s[k] * mu[k];               // dL/dn_k
        sg[k] = (1.f - 0.5f * p.s[k]) * mu[k];  // dL/dS_k
    }
    // equilibrium part: n_k = m^_k - eq_k  =>  dL/drho -= sum nu_k deq_k/drho, dL/dj -= sum nu_k deq_k/dj
    const float n9c = nu_[9] - 0.5f * nu_[10], n11c = nu_[11] - 0.5f * nu_[12];
    float Grho = -(nu_[1] * (-11.f - 19.f * jj * gri * ri) + nu_[2] * (3.f + 5.5f * jj * gri * ri) +
                   n9c * (-e9 * ri) + n11c * (-e11 * ri) + nu_[13] * (-e13 * ri) + nu_[14] * (-e14 * ri) +
                   nu_[15] * (-e15 * ri));
    float Gj[3];
    Gj[0] = -(38.f * nu_[1] * j[0] * gri - 11.f * nu_[2] * j[0] * gri - (2.f / 3.f) * nu_[4] +
              n9c * 4.f * j[0] * gri + nu_[13] * j[1] * gri + nu_[15] * j[2] * gri);
    Gj[1] = -(38.f * nu_[1] * j[1] * gri - 11.f * nu_[2] * j[1] * gri - (2.f / 3.f) * nu_[6] -
              n9c * 2.f * j[1] * gri + n11c * 2.f * j[1] * gri + nu_[13] * j[0] * gri + nu_[14] * j[2] * gri);
    Gj[2] = -(38.f * nu_[1] * j[2] * gri - 11.f * nu_[2] * j[2] * gri - (2.f / 3.f) * nu_[8] -
              n9c * 2.f * j[2] * gri - n11c * 2.f * j[2] * gri + nu_[14] * j[1] * gri + nu_[15] * j[0] * gri);
    // source part: S_k(F, u)
    const float A = 38.f * sg[1] - 11.f * sg[2];          // coefficient of F.u
    const float B9 = 2.f * sg[9] - sg[10];                 // of (2 Fx ux - Fy uy - Fz uz)
    const float B11 = 2.f * sg[11] - sg[12];               // of (Fy uy - Fz uz)
    float Gu[3];
    Gu[0] = ig2 * (A * F[0] + 2.f * B9 * F[0] + sg[13] * F[1] + sg[15] * F[2]);
    Gu[1] = ig2 * (A * F[1] - B9 * F[1] + B11 * F[1] + sg[13] * F[0] + sg[14] * F[2]);
    Gu[2] = ig2 * (A * F[2] - B9 * F[2] - B11 * F[2] + sg[14] * F[1] + sg[15] * F[0]);
    float GF[3];
    GF[0] = ig2 * (A * u[0] + 2.f * B9 * u[0] + sg[13] * u[1] + sg[15] * u[2]) - (2.f / 3.f) * ig * sg[4] + mu[3] * ig;
    GF[1] = ig2 * (A * u[1] - B9 * u[1] + B11 * u[1] + sg[13] * u[0] + sg[14] * u[2]) - (2.f / 3.f) * ig * sg[6] + mu[5] * ig;
    GF[2] = ig2 * (A * u[2] - B9 * u[2] - B11 * u[2] + sg[14] * u[1] + sg[15] * u[0]) - (2.f / 3.f) * ig * sg[8] + mu[7] * ig;
    // the objective's weight on u joins the source's
    for (int c = 0; c < 3; ++c) Gu[c] += wu[c];
    // u = j / rho
    for (int c = 0; c < 3; ++c) {
        Gj[c] += Gu[c] * ri;
        Grho -= Gu[c] * u[c] * ri;
    }
    // j = m + F/(2 gamma)
    for (int c = 0; c < 3; ++c) GF[c] += Gj[c] * hg;
    float Gm[3] = {Gj[0], Gj[1], Gj[2]};
    // dL/dd from the relaxed rows (y_k = nu_k) and the conserved ones (rho, m)
    float y[19];
#pragma unroll
    for (int k = 0; k < 19; ++k) y[k] = nu_[k];
    y[0] = 0.f;
    y[3] = y[5] = y[7] = 0.f;

    float qbar[21];
#pragma unroll
    for (int i = 0; i < 21; ++i) qbar[i] = 0.f;
    float FLpbar[3] = {0.f, 0.f, 0.f};
    float Fextbar[3] = {GF[0], GF[1], GF[2]};
    if (MHD) {
        // F = Fext + FL; the stored F_L is also an output
        const float FLbar[3] = {GF[0] + vFL[0], GF[1] + vFL[1], GF[2] + vFL[2]};
        // FL = J x B
        float Jbar[3], Bbar[3];
        Jbar[0] = B[1] * FLbar[2] - B[2] * FLbar[1];
        Jbar[1] = B[2] * FLbar[0] - B[0] * FLbar[2];
        Jbar[2] = B[0] * FLbar[1] - B[1] * FLbar[0];
        Bbar[0] = FLbar[1] * Jv[2] - FLbar[2] * Jv[1];
        Bbar[1] = FLbar[2] * Jv[0] - FLbar[0] * Jv[2];
        Bbar[2] = FLbar[0] * Jv[1] - FLbar[1] * Jv[0];
        // J = Jc (Nyz - Nzy, Nzx - Nxz, Nxy - Nyx)
        const float Jc = p.J_coef;
        const float Nyzb = Jc * Jbar[0], Nzyb = -Jc * Jbar[0];
        const float Nzxb = Jc * Jbar[1], Nxzb = -Jc * Jbar[1];
        const float Nxyb = Jc * Jbar[2], Nyxb = -Jc * Jbar[2];
        // N = M -+ L
        qbar[8] += Nxyb; qbar[9] -= Nxyb;
        qbar[3] += Nyxb; qbar[4] -= Nyxb;
        qbar[15] += Nxzb; qbar[16] -= Nxzb;
        qbar[5] += Nzxb; qbar[6] -= Nzxb;
        qbar[17] += Nyzb; qbar[18] -= Nyzb;
        qbar[12] += Nzyb; qbar[13] -= Nzyb;
        float Lxyb = -Nxyb + Nyxb, Lxzb = -Nxzb + Nzxb, Lyzb = -Nyzb + Nzyb;
        // g~ = q + omega (W_a b_j + conv - q)
        const float w = p.omega_m;
        float bbar[3] = {0.f, 0.f, 0.f};
        for (int i = 0; i < 21; ++i) {
            const int jj2 = i / 7, a = i % 7;
            const float W = a == 0 ? 0.25f : 0.125f;
            qbar[i] += vg[i] * (1.f - w);
            bbar[jj2] += w * W * vg[i];
        }
        // conv terms: A = L/2 with the signs of the forward table
        const float Axyb = w * (-vg[3] + vg[4] + vg[8] - vg[9]);
        const float Axzb = w * (-vg[5] + vg[6] + vg[15] - vg[16]);
        const float Ayzb = w * (-vg[12] + vg[13] + vg[17] - vg[18]);
        Lxyb += 0.5f * Axyb;
        Lxzb += 0.5f * Axzb;
        Lyzb += 0.5f * Ayzb;
        // L = c (u0 (x) B - B (x) u0)
        const float c = p.conv_coef;
        float u0b[3] = {0.f, 0.f, 0.f};
        u0b[0] += c * (Lxyb * B[1] + Lxzb * B[2]);
        u0b[1] += c * (-Lxyb * B[0] + Lyzb * B[2]);
        u0b[2] += c * (-Lxzb * B[0] - Lyzb * B[1]);
        Bbar[0] += c * (-Lxyb * u0[1] - Lxzb * u0[2]);
        Bbar[1] += c * (Lxyb * u0[0] - Lyzb * u0[2]);
        Bbar[2] += c * (Lxzb * u0[0] + Lyzb * u0[1]);
        // B = B0 + b
        for (int c2 = 0; c2 < 3; ++c2) bbar[c2] += Bbar[c2];
        for (int i = 0; i < 21; ++i) qbar[i] += bbar[i / 7];
        // u0 = (m + hg (Fext + FLp)) / rho
        for (int c2 = 0; c2 < 3; ++c2) {
            Gm[c2] += u0b[c2] * ri;
            Fextbar[c2] += hg * u0b[c2] * ri;
            FLpbar[c2] += hg * u0b[c2] * ri;
            Grho -= u0b[c2] * u0[c2] * ri;
        }
    }
    y[0] = Grho;
    y[3] = Gm[0];
    y[5] = Gm[1];
    y[7] = Gm[2];
    float tt[19];
    apply_Tt(y, tt);
#pragma unroll
    for (int a = 0; a < 19; ++a) out.d[a] = vf[a] + tt[a];
    for (int i = 0; i < 21; ++i) out.q[i] = MHD ? qbar[i] : 0.f;
    for (int c2 = 0; c2 < 3; ++c2) {
        out.FLp[c2] = FLpbar[c2];
        out.F[c2] = Fextbar[c2];
    }
}

// Reverse of the node update at (d, q, FLp, Fext): node_reverse_at at the
// linearisation point node_linearise gives there.
template <bool MHD>
__device__ __forceinline__ void node_reverse(const StepParams& p, const float (&d)[19], const float (&q)[21],
                                             const float (&FLp)[3], const float (&Fext)[3], const float (&vf)[19],
                                             const float (&vg)[21], const float (&vFL)[3], const float (&wu)[3],
                                             NodeAdjoint& out)
{
    node_reverse_at<MHD>(p, node_linearise<MHD>(p, d, q, FLp, Fext), vf, vg, vFL, wu, out);
}

}  // namespace glbe
