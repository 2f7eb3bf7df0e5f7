// adjoint_math.cuh -- transposed Jacobians of the per-node operations of one
// stream-collide step (reverse mode; the paper has no adjoint).
//
// Forward (lbm_math.cuh): source node y holds M(y); its populations are
// g_i = w_i sum_k h_ik A_k(M(y)) with the 17 Hermite coefficients A = make_coef(M);
// destination x pulls g*_i(x) = g_i(M(x - c_i)) (or its own opposite population
// at a wall), projects p = P g* and collides M' = C(p, F).
// Reverse, given lambda' = dL/dM'(x):
//   collide_vjp:   lambda_p = (dC/dp)^T lambda',  lambda_F = (dC/dF)^T lambda'
//   gbar_i(x)      = lambda_drho + c_i . lambda_j + H2(c_i) : lambda_Pi
//   adjoint_moments: ghat_k(y) = sum_i w_i h_ik gbar(dest of g_i(y))
//   coef_vjp:      dL/dM(y) = (dA/dM)^T ghat(y)
#pragma once
#include "lbm_math.cuh"

namespace hlbm {

// Adjoint of collide() (same variables, same order of operations).
template <typename R>
__device__ __forceinline__ void collide_vjp(const PreMom<R>& p, R fx, R fy, R fz, R om, const Mom<R>& lo,
                                            PreMom<R>& lp, R& lfx, R& lfy, R& lfz) {
  const R rho = R(1) + p.drho;
  const R ir = R(1) / rho;
  const R v[3] = {p.jx + R(0.5) * fx, p.jy + R(0.5) * fy, p.jz + R(0.5) * fz};
  const R u[3] = {v[0] * ir, v[1] * ir, v[2] * ir};
  const R F[3] = {fx, fy, fz};
  const R a = R(1) - om, cf = R(1) - R(0.5) * om;
  const R Pi[3][3] = {{p.pxx, p.pxy, p.pxz}, {p.pxy, p.pyy, p.pyz}, {p.pxz, p.pyz, p.pzz}};
  const R lS[3][3] = {{lo.sxx, lo.sxy, lo.sxz}, {lo.sxy, lo.syy, lo.syz}, {lo.sxz, lo.syz, lo.szz}};
  const R lu_out[3] = {lo.ux, lo.uy, lo.uz};
  R lu[3] = {lu_out[0], lu_out[1], lu_out[2]};
  R lF[3] = {R(0.5) * ir * lu_out[0], R(0.5) * ir * lu_out[1], R(0.5) * ir * lu_out[2]};
  R lir = R(0.5) * (lu_out[0] * F[0] + lu_out[1] * F[1] + lu_out[2] * F[2]);
  R lrho = R(0);
  R lPi[3][3];
  // S'_ab = (a Pi_ab + om rho u_a u_b + cf (u_a F_b + F_a u_b)) ir over the 6 stored pairs
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const R l = lS[i][j];
      lPi[i][j] = a * ir * l;
      const R num = a * Pi[i][j] + om * rho * u[i] * u[j] + cf * (u[i] * F[j] + F[i] * u[j]);
      lir += l * num;
      lrho += l * om * u[i] * u[j] * ir;
      lu[i] += l * (om * rho * u[j] + cf * F[j]) * ir;
      lu[j] += l * (om * rho * u[i] + cf * F[i]) * ir;
      lF[j] += l * cf * u[i] * ir;
      lF[i] += l * cf * u[j] * ir;
    }
  // u = v ir, v = j + F / 2
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    lir += lu[i] * v[i];
    lF[i] += R(0.5) * lu[i] * ir;
  }
  lrho -= lir * ir * ir;
  lp.drho = lo.drho + lrho;
  lp.jx = lu[0] * ir;
  lp.jy = lu[1] * ir;
  lp.jz = lu[2] * ir;
  lp.pxx = lPi[0][0];
  lp.pyy = lPi[1][1];
  lp.pzz = lPi[2][2];
  lp.pxy = lPi[0][1];
  lp.pxz = lPi[0][2];
  lp.pyz = lPi[1][2];
  lfx = lF[0];
  lfy = lF[1];
  lfz = lF[2];
}

// Adjoint of the projection for one direction: dL/dg*_J.
template <int J, typename R>
__device__ __forceinline__ R gbar(const PreMom<R>& l) {
  constexpr int cx = Dir<J>::cx, cy = Dir<J>::cy, cz = Dir<J>::cz;
  R v = l.drho;
  if constexpr (cx != 0) v = v + R(cx) * l.jx;
  if constexpr (cy != 0) v = v + R(cy) * l.jy;
  if constexpr (cz != 0) v = v + R(cz) * l.jz;
  v = v + R(cx * cx - 1.0 / 3.0) * l.pxx + R(cy * cy - 1.0 / 3.0) * l.pyy + R(cz * cz - 1.0 / 3.0) * l.pzz;
  if constexpr (cx * cy != 0) v = v + R(cx * cy) * l.pxy;
  if constexpr (cx * cz != 0) v = v + R(cx * cz) * l.pxz;
  if constexpr (cy * cz != 0) v = v + R(cy * cz) * l.pyz;
  return v;
}

// ghat_k = sum_i w_i h_ik gb[i]: weighted moments up to third order, by
// tensor-product sums (D3Q27 weights factor as w(cx) w(cy) w(cz), w(0) = 2/3,
// w(+-1) = 1/6).  Returns the 17 coefficient adjoints in Coef order.
template <typename R>
__device__ __forceinline__ Coef<R> adjoint_moments(const R (&gb)[27]) {
  const R w0 = R(2.0 / 3.0), w1 = R(1.0 / 6.0);
  // x sums per line l = (cy+1) + 3 (cz+1): X0 = sum w g, X1 = sum w c g, X2 = sum w c^2 g
  R X0[9], X1[9], X2[9];
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const R gm = gb[3 * l], g0 = gb[3 * l + 1], gp = gb[3 * l + 2];
    X2[l] = w1 * (gp + gm);
    X1[l] = w1 * (gp - gm);
    X0[l] = X2[l] + w0 * g0;
  }
  // y sums per z index k = cz+1: Y[a][b] = sum_cy w(cy) cy^b X_a
  R Y[3][3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R* Xs[3] = {X0, X1, X2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const R m = Xs[a][3 * k], z = Xs[a][3 * k + 1], pl = Xs[a][3 * k + 2];
      Y[k][a][2] = w1 * (pl + m);
      Y[k][a][1] = w1 * (pl - m);
      Y[k][a][0] = Y[k][a][2] + w0 * z;
    }
  }
  // z sums: M[a][b][c] = sum_cz w(cz) cz^c Y[cz][a][b]
  auto Mz = [&](int a, int b, int c) -> R {
    const R m = Y[0][a][b], z = Y[1][a][b], pl = Y[2][a][b];
    if (c == 0) return w1 * (pl + m) + w0 * z;
    if (c == 1) return w1 * (pl - m);
    return w1 * (pl + m);
  };
  const R t = R(1.0 / 3.0);
  Coef<R> g;
  g.K0 = Mz(0, 0, 0);
  g.Ux = Mz(1, 0, 0);
  g.Uy = Mz(0, 1, 0);
  g.Uz = Mz(0, 0, 1);
  g.Dx = Mz(2, 0, 0);
  g.Dy = Mz(0, 2, 0);
  g.Dz = Mz(0, 0, 2);
  g.Oxy = Mz(1, 1, 0);
  g.Oxz = Mz(1, 0, 1);
  g.Oyz = Mz(0, 1, 1);
  g.Gxxy = Mz(2, 1, 0) - t * g.Uy;
  g.Gxyy = Mz(1, 2, 0) - t * g.Ux;
  g.Gxxz = Mz(2, 0, 1) - t * g.Uz;
  g.Gxzz = Mz(1, 0, 2) - t * g.Ux;
  g.Gyzz = Mz(0, 1, 2) - t * g.Uy;
  g.Gyyz = Mz(0, 2, 1) - t * g.Uz;
  g.Gxyz = Mz(1, 1, 1);
  return g;
}

// (dA/dM)^T ghat for A = make_coef(M, kxyz).
template <typename R>
__device__ __forceinline__ Mom<R> coef_vjp(const Mom<R>& m, const Coef<R>& g, R kxyz) {
  const R rho = R(1) + m.drho;
  const R u[3] = {m.ux, m.uy, m.uz};
  const R S[3][3] = {{m.sxx, m.sxy, m.sxz}, {m.sxy, m.syy, m.syz}, {m.sxz, m.syz, m.szz}};
  R ld = R(0), lu[3] = {R(0), R(0), R(0)}, lS[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) lS[i][j] = R(0);
  const R tr = m.sxx + m.syy + m.szz;
  // K0 = drho - 3/2 rho tr S
  ld = ld + g.K0 * (R(1) - R(1.5) * tr);
  for (int i = 0; i < 3; ++i) lS[i][i] = lS[i][i] - R(1.5) * rho * g.K0;
  // U_a = 3 rho u_a, D_a = 9/2 rho S_aa
  const R gU[3] = {g.Ux, g.Uy, g.Uz}, gD[3] = {g.Dx, g.Dy, g.Dz};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    ld = ld + R(3) * u[i] * gU[i] + R(4.5) * S[i][i] * gD[i];
    lu[i] = lu[i] + R(3) * rho * gU[i];
    lS[i][i] = lS[i][i] + R(4.5) * rho * gD[i];
  }
  // O_ab = 9 rho S_ab
  ld = ld + R(9) * (m.sxy * g.Oxy + m.sxz * g.Oxz + m.syz * g.Oyz);
  lS[0][1] = lS[0][1] + R(9) * rho * g.Oxy;
  lS[0][2] = lS[0][2] + R(9) * rho * g.Oxz;
  lS[1][2] = lS[1][2] + R(9) * rho * g.Oyz;
  // G_aab = 27/2 rho Gamma_aab, Gamma_aab = S_aa u_b + 2 S_ab u_a - 2 u_a^2 u_b
  const int ta[6] = {0, 1, 0, 2, 2, 1}, tb[6] = {1, 0, 2, 0, 1, 2};  // xxy xyy xxz xzz yzz yyz
  const R gG[6] = {g.Gxxy, g.Gxyy, g.Gxxz, g.Gxzz, g.Gyzz, g.Gyyz};
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int A = ta[t], B = tb[t];
    const R gam = S[A][A] * u[B] + R(2) * S[A][B] * u[A] - R(2) * u[A] * u[A] * u[B];
    ld = ld + R(13.5) * gam * gG[t];
    const R q = R(13.5) * rho * gG[t];
    lS[A][A] = lS[A][A] + q * u[B];
    if (A < B)
      lS[A][B] = lS[A][B] + R(2) * q * u[A];
    else
      lS[B][A] = lS[B][A] + R(2) * q * u[A];
    lu[A] = lu[A] + q * (R(2) * S[A][B] - R(4) * u[A] * u[B]);
    lu[B] = lu[B] + q * (S[A][A] - R(2) * u[A] * u[A]);
  }
  // G_xyz = kxyz rho Gamma_xyz
  {
    const R gam = m.sxy * u[2] + m.sxz * u[1] + m.syz * u[0] - R(2) * u[0] * u[1] * u[2];
    ld = ld + kxyz * gam * g.Gxyz;
    const R q = kxyz * rho * g.Gxyz;
    lS[0][1] = lS[0][1] + q * u[2];
    lS[0][2] = lS[0][2] + q * u[1];
    lS[1][2] = lS[1][2] + q * u[0];
    lu[0] = lu[0] + q * (m.syz - R(2) * u[1] * u[2]);
    lu[1] = lu[1] + q * (m.sxz - R(2) * u[0] * u[2]);
    lu[2] = lu[2] + q * (m.sxy - R(2) * u[0] * u[1]);
  }
  Mom<R> r;
  r.drho = ld;
  r.ux = lu[0];
  r.uy = lu[1];
  r.uz = lu[2];
  r.sxx = lS[0][0];
  r.syy = lS[1][1];
  r.szz = lS[2][2];
  r.sxy = lS[0][1];
  r.sxz = lS[0][2];
  r.syz = lS[1][2];
  return r;
}

}  // namespace hlbm
