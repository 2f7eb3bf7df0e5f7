// lbm_math.cuh -- per-node arithmetic of the moment-encoded D3Q27 scheme.
//
// * reconstruction f_i(M) of Eq. (three_order_f), evaluated per direction class
//   (rest, 6 faces, 12 edges, 8 corners) with sign butterflies;
// * moment projection of Eq. (rho_u_stress) by tensor-product partial sums;
// * BGK collision in Hermite-moment space with Guo forcing and the mixture
//   relaxation time eps*tau (Sec. 3.1 "Collision and Streaming", Sec. 4).
//
// Every population is handled as its deviation g_i = f_i - w_i from the rest
// state (rho = 1, u = 0, S = 0): the stored density is delta_rho = rho - 1 and
// sums of g never carry the O(1) background, so FP32 keeps full relative
// precision in the small moments.
#pragma once
#include <cstdint>

namespace hlbm {

// Direction index j = (c_x+1) + 3 (c_y+1) + 9 (c_z+1); rest is 13, opposite 26-j.
template <int J>
struct Dir {
  static constexpr int cx = J % 3 - 1;
  static constexpr int cy = (J / 3) % 3 - 1;
  static constexpr int cz = J / 9 - 1;
};

// a * b + c and 1 / a for the scalar types (the packed type V2 has its own).
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float inv(float a) { return 1.0f / a; }
__device__ __forceinline__ double inv(double a) { return 1.0 / a; }

template <typename R>
struct Mom {
  R drho, ux, uy, uz, sxx, syy, szz, sxy, sxz, syz;
};

// Hermite coefficients of one source node (all multiplied by rho):
//   K0 = drho - (3/2) rho tr S            constant part
//   U_a = 3 rho u_a                        first order (c.u / c_s^2)
//   D_a = (9/2) rho S_aa                   diagonal second order
//   O_ab = 9 rho S_ab                      off-diagonal second order (counted twice in H2:S)
//   G_t = k_t rho Gamma_t                  third order, k_t = 1/(2 c_s^6) for the mixed
//                                          triples, kxyz for xyz
template <typename R>
struct Coef {
  R K0, Ux, Uy, Uz, Dx, Dy, Dz, Oxy, Oxz, Oyz;
  R Gxxy, Gxyy, Gxxz, Gxzz, Gyzz, Gyyz, Gxyz;
};

template <typename R>
__device__ __forceinline__ Coef<R> make_coef(const Mom<R>& m, R kxyz) {
  const R rho = R(1) + m.drho;
  Coef<R> c;
  c.K0 = m.drho - R(1.5) * rho * (m.sxx + m.syy + m.szz);
  const R r3 = R(3) * rho, r45 = R(4.5) * rho, r9 = R(9) * rho, r135 = R(13.5) * rho;
  c.Ux = r3 * m.ux;
  c.Uy = r3 * m.uy;
  c.Uz = r3 * m.uz;
  c.Dx = r45 * m.sxx;
  c.Dy = r45 * m.syy;
  c.Dz = r45 * m.szz;
  c.Oxy = r9 * m.sxy;
  c.Oxz = r9 * m.sxz;
  c.Oyz = r9 * m.syz;
  const R ux = m.ux, uy = m.uy, uz = m.uz;
  const R m2 = R(-2);
  // Gamma_abg = S_ab u_g + S_ag u_b + S_bg u_a - 2 u_a u_b u_g
  const R sxy2 = m.sxy + m.sxy, sxz2 = m.sxz + m.sxz, syz2 = m.syz + m.syz;
  const R uxx = m2 * ux * ux, uyy = m2 * uy * uy, uzz = m2 * uz * uz;
  c.Gxxy = r135 * mad(m.sxx + uxx, uy, sxy2 * ux);  // u_y (S_xx - 2 u_x^2) + 2 S_xy u_x
  c.Gxyy = r135 * mad(m.syy + uyy, ux, sxy2 * uy);
  c.Gxxz = r135 * mad(m.sxx + uxx, uz, sxz2 * ux);
  c.Gxzz = r135 * mad(m.szz + uzz, ux, sxz2 * uz);
  c.Gyzz = r135 * mad(m.szz + uzz, uy, syz2 * uz);
  c.Gyyz = r135 * mad(m.syy + uyy, uz, syz2 * uy);
  c.Gxyz = kxyz * rho * mad(m.sxy, uz, mad(m.sxz, uy, mad(m2 * ux, uy * uz, m.syz * ux)));
  return c;
}

// Emit g_j = f_j - w_j of one source node to sink.put<J>(value) for all 27 j.
// A sink that ignores some J lets the compiler drop their arithmetic.
//
// With H3_aab(c) = (c_a^2 - 1/3) c_b and H3_xyz = c_x c_y c_z the bracket of
// Eq. (three_order_f) per class is (s = +-1 components):
//   rest   : K0
//   face a : K0 + D_a + s (U_a - (G_abb + G_acc)/3)
//   edge ab: K0 + D_a + D_b + s_a X + s_b Y + s_a s_b O_ab
//   corner : K0 + D_x + D_y + D_z + sum_a s_a X_a + sum_{a<b} s_a s_b O_ab + s_x s_y s_z G_xyz
// with the third-order corrections folded into X / X_a.
template <typename R, typename Sink>
__device__ __forceinline__ void emit_all(const Coef<R>& c, Sink& s) {
  const R w0 = R(8.0 / 27.0), wf = R(2.0 / 27.0), we = R(1.0 / 54.0), wc = R(1.0 / 216.0);
  const R t2 = R(2.0 / 3.0), mt1 = R(-1.0 / 3.0);
  s.template put<13>(w0 * c.K0);
  {  // faces x
    const R E = c.K0 + c.Dx, O = mad(mt1, c.Gxyy + c.Gxzz, c.Ux);
    s.template put<14>(wf * (E + O));
    s.template put<12>(wf * (E - O));
  }
  {  // faces y
    const R E = c.K0 + c.Dy, O = mad(mt1, c.Gxxy + c.Gyzz, c.Uy);
    s.template put<16>(wf * (E + O));
    s.template put<10>(wf * (E - O));
  }
  {  // faces z
    const R E = c.K0 + c.Dz, O = mad(mt1, c.Gxxz + c.Gyyz, c.Uz);
    s.template put<22>(wf * (E + O));
    s.template put<4>(wf * (E - O));
  }
  {  // edges xy (c_z = 0): j = (sx+1) + 3 (sy+1) + 9
    const R E = c.K0 + c.Dx + c.Dy;
    const R X = mad(t2, c.Gxyy, mad(mt1, c.Gxzz, c.Ux));
    const R Y = mad(t2, c.Gxxy, mad(mt1, c.Gyzz, c.Uy));
    const R a = E + c.Oxy, b = E - c.Oxy, p = X + Y, m = X - Y;
    s.template put<17>(we * (a + p));  // (+,+)
    s.template put<9>(we * (a - p));   // (-,-)
    s.template put<11>(we * (b + m));  // (+,-)
    s.template put<15>(we * (b - m));  // (-,+)
  }
  {  // edges xz (c_y = 0): j = (sx+1) + 3 + 9 (sz+1)
    const R E = c.K0 + c.Dx + c.Dz;
    const R X = mad(t2, c.Gxzz, mad(mt1, c.Gxyy, c.Ux));
    const R Z = mad(t2, c.Gxxz, mad(mt1, c.Gyyz, c.Uz));
    const R a = E + c.Oxz, b = E - c.Oxz, p = X + Z, m = X - Z;
    s.template put<23>(we * (a + p));  // (+,+)
    s.template put<3>(we * (a - p));   // (-,-)
    s.template put<5>(we * (b + m));   // (+,-)
    s.template put<21>(we * (b - m));  // (-,+)
  }
  {  // edges yz (c_x = 0): j = 1 + 3 (sy+1) + 9 (sz+1)
    const R E = c.K0 + c.Dy + c.Dz;
    const R Y = mad(t2, c.Gyzz, mad(mt1, c.Gxxy, c.Uy));
    const R Z = mad(t2, c.Gyyz, mad(mt1, c.Gxxz, c.Uz));
    const R a = E + c.Oyz, b = E - c.Oyz, p = Y + Z, m = Y - Z;
    s.template put<25>(we * (a + p));  // (+,+)
    s.template put<1>(we * (a - p));   // (-,-)
    s.template put<7>(we * (b + m));   // (+,-)
    s.template put<19>(we * (b - m));  // (-,+)
  }
  {  // corners: value = P(sx,sy) + sz Q(sx,sy)
    const R E = c.K0 + c.Dx + c.Dy + c.Dz;
    const R X = mad(t2, c.Gxyy + c.Gxzz, c.Ux);
    const R Y = mad(t2, c.Gxxy + c.Gyzz, c.Uy);
    const R Z = mad(t2, c.Gxxz + c.Gyyz, c.Uz);
    const R pa = E + c.Oxy, pb = E - c.Oxy, pp = X + Y, pm = X - Y;
    const R Ppp = pa + pp, Pmm = pa - pp, Ppm = pb + pm, Pmp = pb - pm;
    const R qa = Z + c.Gxyz, qb = Z - c.Gxyz, qp = c.Oxz + c.Oyz, qm = c.Oxz - c.Oyz;
    const R Qpp = qa + qp, Qmm = qa - qp, Qpm = qb + qm, Qmp = qb - qm;
    // j = (sx+1) + 3 (sy+1) + 9 (sz+1)
    s.template put<26>(wc * (Ppp + Qpp));  // (+,+,+)
    s.template put<8>(wc * (Ppp - Qpp));   // (+,+,-)
    s.template put<18>(wc * (Pmm + Qmm));  // (-,-,+)
    s.template put<0>(wc * (Pmm - Qmm));   // (-,-,-)
    s.template put<20>(wc * (Ppm + Qpm));  // (+,-,+)
    s.template put<2>(wc * (Ppm - Qpm));   // (+,-,-)
    s.template put<24>(wc * (Pmp + Qmp));  // (-,+,+)
    s.template put<6>(wc * (Pmp - Qmp));   // (-,+,-)
  }
}

// Pre-collision moments (deviation form) of 27 pulled populations g[j]:
// drho* = sum g, j*_a = sum c_a g, Pi*_ab = sum (c_a c_b - delta_ab/3) g.
template <typename R>
struct PreMom {
  R drho, jx, jy, jz, pxx, pyy, pzz, pxy, pxz, pyz;
};

template <typename R>
__device__ __forceinline__ PreMom<R> project(const R (&g)[27]) {
  // sums along x for each line l = (cy+1) + 3 (cz+1): j = 3 l + (cx+1)
  R s0[9], s1[9], s2[9];
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const R gm = g[3 * l], g0 = g[3 * l + 1], gp = g[3 * l + 2];
    s2[l] = gp + gm;
    s1[l] = gp - gm;
    s0[l] = s2[l] + g0;
  }
  R A0[3], A1[3], A2[3], B0[3], B1[3], C0[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {  // k = cz + 1, lines 3k + (cy+1)
    A2[k] = s0[3 * k + 2] + s0[3 * k];
    A1[k] = s0[3 * k + 2] - s0[3 * k];
    A0[k] = A2[k] + s0[3 * k + 1];
    B1[k] = s1[3 * k + 2] - s1[3 * k];
    B0[k] = s1[3 * k + 2] + s1[3 * k] + s1[3 * k + 1];
    C0[k] = s2[3 * k + 2] + s2[3 * k] + s2[3 * k + 1];
  }
  PreMom<R> p;
  p.drho = A0[0] + A0[1] + A0[2];
  p.jz = A0[2] - A0[0];
  const R mzz = A0[2] + A0[0];
  p.jy = A1[0] + A1[1] + A1[2];
  p.pyz = A1[2] - A1[0];
  const R myy = A2[0] + A2[1] + A2[2];
  p.jx = B0[0] + B0[1] + B0[2];
  p.pxz = B0[2] - B0[0];
  p.pxy = B1[0] + B1[1] + B1[2];
  const R mxx = C0[0] + C0[1] + C0[2];
  const R d3 = p.drho * R(1.0 / 3.0);
  p.pxx = mxx - d3;
  p.pyy = myy - d3;
  p.pzz = mzz - d3;
  return p;
}

// BGK collision in moment space with Guo forcing (Sec. 3.1; Sec. 4 with
// tau_e = eps tau).  u = (j* + F/2)/rho*, the stored velocity is u + F/(2 rho*),
// S' = [(1-om) Pi* + om rho* u u + (1 - om/2)(u F + F u)] / rho*, om = 1/tau_e.
template <typename R>
__device__ __forceinline__ Mom<R> collide(const PreMom<R>& p, R fx, R fy, R fz, R om) {
  const R rho = R(1) + p.drho;
  const R ir = inv(rho);
  const R h = R(0.5);
  const R ux = mad(h, fx, p.jx) * ir;
  const R uy = mad(h, fy, p.jy) * ir;
  const R uz = mad(h, fz, p.jz) * ir;
  const R a = R(1) - om, b = om * rho, cf = R(1) - h * om;
  const R bux = b * ux, buy = b * uy, buz = b * uz;
  const R cfx = cf * fx, cfy = cf * fy, cfz = cf * fz;
  Mom<R> m;
  m.drho = p.drho;
  m.sxx = mad(a, p.pxx, mad(bux, ux, (cfx + cfx) * ux)) * ir;
  m.syy = mad(a, p.pyy, mad(buy, uy, (cfy + cfy) * uy)) * ir;
  m.szz = mad(a, p.pzz, mad(buz, uz, (cfz + cfz) * uz)) * ir;
  m.sxy = mad(a, p.pxy, mad(bux, uy, mad(cfy, ux, cfx * uy))) * ir;
  m.sxz = mad(a, p.pxz, mad(bux, uz, mad(cfz, ux, cfx * uz))) * ir;
  m.syz = mad(a, p.pyz, mad(buy, uz, mad(cfz, uy, cfy * uz))) * ir;
  const R hir = h * ir;
  m.ux = mad(hir, fx, ux);
  m.uy = mad(hir, fy, uy);
  m.uz = mad(hir, fz, uz);
  return m;
}

}  // namespace hlbm
