// Coordinated-turn bearings-only model (Sec. 6.2) and its square-root
// statistical linear regression (Sec. 4.2 Taylor, Sec. 4.3 cubature), one
// thread per time step, plus the IPLS loop of Alg. 3.
//
// Model: x = (p_x, p_y, v_x, v_y, w), a = w dt,
//   p' = p + [[S, -C], [C, S]] v,  v' = [[cos a, -sin a], [sin a, cos a]] v,
//   w' = w,  S = sin(a)/w,  C = (1 - cos a)/w = 2 sin^2(a/2)/w
//   (Taylor series of sin(a)/a and (1 - cos a)/a^2 for |a| <= 1/4);
//   process noise factor in closed form; bearings
//   atan2(p_y - s_y, p_x - s_x) with noise sigma.
//
// Cubature (third-degree spherical-radial rule, points m +- sqrt(nx) N e_i,
// weights 1/(2 nx)).  Two exact rewritings of Sec. 4.3 are used:
//  * because X_i - m = +-sqrt(nx) N e_i, the regression matrix
//    sum_i w (Z_i - z)(X_i - m)^T (N N^T)^{-1} equals D N^{-1} with
//    D e_i = (Z_i^+ - Z_i^-)/(2 sqrt(nx));
//  * the noise factor DownDate(Tria([sqrt(w) S, ..., Z_x]), F N) of eqs.
//    lambda-prime / sqr-lambda-sigma-point has the same product as
//    Tria([S, s_1/sqrt(nx), ..., s_nx/sqrt(nx)]) with
//    s_i = (Z_i^+ + Z_i^-)/2 - z_bar (the residual Z_i - z_bar - F(X_i - m)
//    of both points of pair i); this needs no downdate and cannot fail.
// Transformed points are evaluated as differences from the mean's image in
// a form without cancellation (for f, of its non-identity part f(x) - x, whose
// regression is added to I), and bearings of the points as the signed angle
// from the mean's line of sight, which also takes them on the branch nearest
// h(m).  d absorbs the 2 pi multiple that moves y
// onto that branch.
#pragma once

#include "engine.cuh"

namespace sqsm {

template <typename T>
struct CTParams {
  T dt;
  T sx[2], sy[2];
  T sigma[2];    // bearing noise standard deviation of each sensor
  T SQ[25];      // lower Cholesky factor of the process noise
};

SQSM_DEV void sq_sincos(float a, float* s, float* c) { sincosf(a, s, c); }
SQSM_DEV void sq_sincos(double a, double* s, double* c) { sincos(a, s, c); }
SQSM_DEV float sq_atan2(float y, float x) { return atan2f(y, x); }
SQSM_DEV double sq_atan2(double y, double x) { return atan2(y, x); }
SQSM_DEV float sq_floor(float x) { return floorf(x); }
SQSM_DEV double sq_floor(double x) { return floor(x); }

// Parameters from theta = (log sigma_1, log q_c, log q_w, log sigma_2)
// (bearing noise standard deviation of each sensor; closed-form factor of
// q_c [[dt^3/3, dt^2/2], [dt^2/2, dt]] per axis and q_w dt).
template <typename T>
__global__ void ct_params_kernel(double th0, double th1, double th2, double th3, double dt,
                                 double s1x, double s1y, double s2x, double s2y, CTParams<T>* P) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double qc = exp(th1), qw = exp(th2);
  CTParams<T> p;
  p.dt = (T)dt;
  p.sx[0] = (T)s1x; p.sy[0] = (T)s1y; p.sx[1] = (T)s2x; p.sy[1] = (T)s2y;
  p.sigma[0] = (T)exp(th0);
  p.sigma[1] = (T)exp(th3);
  for (int i = 0; i < 25; ++i) p.SQ[i] = T(0);
  const double a = sqrt(qc * dt * dt * dt / 3.0);
  const double b = sqrt(qc) * sqrt(3.0 * dt) / 2.0;
  const double c = sqrt(qc) * sqrt(dt) / 2.0;
  for (int i = 0; i < 2; ++i) {
    p.SQ[i * 5 + i] = (T)a;
    p.SQ[(i + 2) * 5 + i] = (T)b;
    p.SQ[(i + 2) * 5 + i + 2] = (T)c;
  }
  p.SQ[24] = (T)sqrt(qw * dt);
  *P = p;
}

// sin(a)/a and (1 - cos a)/a^2 by their Taylor series in a^2, for
// |a| <= kSeriesMaxAngle: the first omitted term is below half an ulp of the
// result (a^2 <= 1/16; FP32 keeps 4 terms, FP64 7).
constexpr double kSeriesMaxAngle = 0.25;

template <typename T>
SQSM_DEV void sinc_cosc(T a2, T& sinc, T& cosc) {
  if constexpr (sizeof(T) == 4) {
    sinc = T(1) + a2 * (T(-1.0 / 6) + a2 * (T(1.0 / 120) + a2 * T(-1.0 / 5040)));
    cosc = T(0.5) + a2 * (T(-1.0 / 24) + a2 * (T(1.0 / 720) + a2 * T(-1.0 / 40320)));
  } else {
    sinc = T(1) + a2 * (T(-1.0 / 6) + a2 * (T(1.0 / 120) + a2 * (T(-1.0 / 5040) +
           a2 * (T(1.0 / 362880) + a2 * (T(-1.0 / 39916800) + a2 * T(1.0 / 6227020800.0))))));
    cosc = T(0.5) + a2 * (T(-1.0 / 24) + a2 * (T(1.0 / 720) + a2 * (T(-1.0 / 40320) +
           a2 * (T(1.0 / 3628800) + a2 * (T(-1.0 / 479001600) + a2 * T(1.0 / 87178291200.0))))));
  }
}

// sin a and 1 - cos a of a small angle (series), else from one sincos of
// a/2 (sin a = 2 s c, 1 - cos a = 2 s^2): both without cancellation.
template <typename T>
SQSM_DEV void sin_omc(T a, T& sa, T& omc) {
  if (fabs(a) <= T(kSeriesMaxAngle)) {
    T sinc, cosc;
    sinc_cosc(a * a, sinc, cosc);
    sa = a * sinc;
    omc = a * a * cosc;
  } else {
    T sh, ch;
    sq_sincos(T(0.5) * a, &sh, &ch);
    sa = T(2) * sh * ch;
    omc = T(2) * sh * sh;
  }
}

// Turn coefficients of a = w dt: S = sin(a)/w, C = (1 - cos a)/w,
// ca = cos a, sa = sin a, omc = 1 - cos a.  Small angles (the usual case:
// |w| dt <= 1/4) take the series of sin(a)/a and (1 - cos a)/a^2, which need
// neither a sincos nor a division; larger ones one sincos of a/2 and two
// divisions.
template <typename T>
struct Turn {
  T S, C, ca, sa, omc;
};

template <typename T>
SQSM_DEV Turn<T> turn(T w, T dt) {
  Turn<T> r;
  const T a = w * dt;
  if (fabs(a) <= T(kSeriesMaxAngle)) {
    T sinc, cosc;
    sinc_cosc(a * a, sinc, cosc);
    r.sa = a * sinc;
    r.omc = a * a * cosc;
    r.S = dt * sinc;
    r.C = dt * a * cosc;
  } else {
    T sh, ch;
    sq_sincos(T(0.5) * a, &sh, &ch);
    r.sa = T(2) * sh * ch;
    r.omc = T(2) * sh * sh;
    r.S = r.sa / w;
    r.C = r.omc / w;
  }
  r.ca = T(1) - r.omc;
  return r;
}

template <typename T>
SQSM_DEV void turn_coeffs(T w, T dt, T& S, T& C, T& ca, T& sa) {
  const Turn<T> r = turn(w, dt);
  S = r.S;
  C = r.C;
  ca = r.ca;
  sa = r.sa;
}

// dS/dw and dC/dw: series in a for |a| < 0.1, closed forms otherwise.
template <typename T>
SQSM_DEV void turn_coeff_derivs(T w, T dt, T& dS, T& dC) {
  const T a = w * dt;
  T dsa, dca;
  if (fabs(a) < T(0.1)) {
    const T a2 = a * a;
    dsa = a * (T(-1) / T(3) + a2 * (T(1) / T(30) + a2 * (T(-1) / T(840) + a2 / T(45360))));
    dca = T(0.5) + a2 * (T(-1) / T(8) + a2 * (T(1) / T(144) + a2 * (T(-1) / T(5760) + a2 / T(403200))));
  } else {
    T sh, ch;
    sq_sincos(T(0.5) * a, &sh, &ch);
    const T sa = T(2) * sh * ch, omc = T(2) * sh * sh;
    dsa = (a * (T(1) - omc) - sa) / (a * a);
    dca = (a * sa - omc) / (a * a);
  }
  dS = dt * dt * dsa;
  dC = dt * dt * dca;
}

template <typename T>
SQSM_DEV void ct_f(const CTParams<T>& P, const T* x, T* o) {
  T S, C, ca, sa;
  turn_coeffs(x[4], P.dt, S, C, ca, sa);
  o[0] = x[0] + S * x[2] - C * x[3];
  o[1] = x[1] + C * x[2] + S * x[3];
  o[2] = ca * x[2] - sa * x[3];
  o[3] = sa * x[2] + ca * x[3];
  o[4] = x[4];
}

// f(x) - x: the CT step has no position term in it, so this is exact
// however large the position (1 - cos a = 2 sin^2(a/2)).
template <typename T>
SQSM_DEV void ct_f_minus_x(const CTParams<T>& P, const T* x, T* o) {
  const Turn<T> t = turn(x[4], P.dt);
  o[0] = t.S * x[2] - t.C * x[3];
  o[1] = t.C * x[2] + t.S * x[3];
  o[2] = -t.omc * x[2] - t.sa * x[3];
  o[3] = t.sa * x[2] - t.omc * x[3];
  o[4] = T(0);
}

// g(m + dl) - g(m) for g(x) = f(x) - x, the part of the CT step that is not
// the identity, written so that no term cancels against a larger one:
//   positions:  K(w_x) dl_v + (K(w_x) - K(w_m)) v_m,  K = [[S, -C], [C, S]],
//   velocities: (R(a_x) - I) dl_v + R(a_m) (R(da) - I) v_m,
//   with R(b) - I = [[-2 sin^2(b/2), -sin b], [sin b, -2 sin^2(b/2)]] and
//   da = dl_w dt formed from the small increment itself; omega: 0.
// (The cubature regression of f is then I + the regression of g.)
template <typename T>
SQSM_DEV void ct_g_delta(const CTParams<T>& P, const Turn<T>& tm, const T* m, const T* dl, T* o) {
  const Turn<T> tx = turn(m[4] + dl[4], P.dt);
  T sd, omd;
  sin_omc(dl[4] * P.dt, sd, omd);
  const T ux = -omd * m[2] - sd * m[3], uy = sd * m[2] - omd * m[3];
  o[0] = (tx.S * dl[2] - tx.C * dl[3]) + ((tx.S - tm.S) * m[2] - (tx.C - tm.C) * m[3]);
  o[1] = (tx.C * dl[2] + tx.S * dl[3]) + ((tx.C - tm.C) * m[2] + (tx.S - tm.S) * m[3]);
  o[2] = (-tx.omc * dl[2] - tx.sa * dl[3]) + (tm.ca * ux - tm.sa * uy);
  o[3] = (tx.sa * dl[2] - tx.omc * dl[3]) + (tm.sa * ux + tm.ca * uy);
  o[4] = T(0);
}

// The same differences evaluated the way the SLR formulas are printed: the
// function at the sigma point and at the mean in absolute coordinates, then
// subtracted (g(m + dl) - g(m) with g(x) = f(x) - x).  Their FP32 rounding
// is that of the absolute values (positions of size ~100), which the
// textbook comparator of the robustness experiment keeps on purpose.
template <typename T>
SQSM_DEV void ct_g_delta_naive(const CTParams<T>& P, const T* m, const T* dl, T* o) {
  T xa[5], fa[5], f0[5];
#pragma unroll
  for (int r = 0; r < 5; ++r) xa[r] = m[r] + dl[r];
  ct_f(P, xa, fa);
  ct_f(P, m, f0);
#pragma unroll
  for (int r = 0; r < 5; ++r) o[r] = (fa[r] - xa[r]) - (f0[r] - m[r]);
}

template <typename T>
SQSM_DEV void ct_jac_f(const CTParams<T>& P, const T* x, T* J) {
  T S, C, ca, sa, dS, dC;
  const T dt = P.dt;
  turn_coeffs(x[4], dt, S, C, ca, sa);
  turn_coeff_derivs(x[4], dt, dS, dC);
  const T vx = x[2], vy = x[3];
  const T r[25] = {T(1), T(0), S, -C, vx * dS - vy * dC,
                   T(0), T(1), C, S, vx * dC + vy * dS,
                   T(0), T(0), ca, -sa, -dt * sa * vx - dt * ca * vy,
                   T(0), T(0), sa, ca, dt * ca * vx - dt * sa * vy,
                   T(0), T(0), T(0), T(0), T(1)};
#pragma unroll
  for (int i = 0; i < 25; ++i) J[i] = r[i];
}

// Second derivatives of the turn coefficients in w: d2S/dw2 = dt^3 u''(a)
// with u(a) = sin(a)/a and d2C/dw2 = dt^3 v''(a) with v(a) = (1 - cos a)/a
// (a = w dt): series for |a| < 0.1, closed forms otherwise.
template <typename T>
SQSM_DEV void turn_coeff_derivs2(T w, T dt, T& d2S, T& d2C) {
  const T a = w * dt;
  T u2, v2;
  if (fabs(a) < T(0.1)) {
    const T a2 = a * a;
    u2 = T(-1) / T(3) + a2 * (T(1) / T(10) + a2 * (T(-1) / T(168) + a2 / T(6480)));
    v2 = a * (T(-1) / T(4) + a2 * (T(1) / T(36) + a2 * (T(-1) / T(960) + a2 / T(50400))));
  } else {
    T sh, ch;
    sq_sincos(T(0.5) * a, &sh, &ch);
    const T sa = T(2) * sh * ch, omc = T(2) * sh * sh, ca = T(1) - omc;
    const T a3 = a * a * a;
    u2 = (-a * a * sa - T(2) * a * ca + T(2) * sa) / a3;
    v2 = (a * a * ca - T(2) * a * sa + T(2) * omc) / a3;
  }
  d2S = dt * dt * dt * u2;
  d2C = dt * dt * dt * v2;
}

// Contraction of the second derivatives of f with a cotangent of its
// Jacobian: out_k += sum_ij Jb_ij d J_ij / d x_k, J = ct_jac_f (the
// derivative of the Taylor linearisation F = J(m) in m, Sec. 4.2).
template <typename T>
SQSM_DEV void ct_jac_f_vjp(const CTParams<T>& P, const T* x, const T* Jb, T* out) {
  T S, C, ca, sa, dS, dC, d2S, d2C;
  const T dt = P.dt;
  turn_coeffs(x[4], dt, S, C, ca, sa);
  turn_coeff_derivs(x[4], dt, dS, dC);
  turn_coeff_derivs2(x[4], dt, d2S, d2C);
  const T vx = x[2], vy = x[3];
  // d/dvx, d/dvy: only the omega column depends on v
  out[2] += Jb[0 * 5 + 4] * dS + Jb[1 * 5 + 4] * dC + Jb[2 * 5 + 4] * (-dt * sa) +
            Jb[3 * 5 + 4] * (dt * ca);
  out[3] += Jb[0 * 5 + 4] * (-dC) + Jb[1 * 5 + 4] * dS + Jb[2 * 5 + 4] * (-dt * ca) +
            Jb[3 * 5 + 4] * (-dt * sa);
  // d/dw of every omega-dependent entry (d ca/dw = -dt sa, d sa/dw = dt ca)
  const T dt2 = dt * dt;
  out[4] += Jb[0 * 5 + 2] * dS + Jb[0 * 5 + 3] * (-dC) + Jb[0 * 5 + 4] * (vx * d2S - vy * d2C) +
            Jb[1 * 5 + 2] * dC + Jb[1 * 5 + 3] * dS + Jb[1 * 5 + 4] * (vx * d2C + vy * d2S) +
            Jb[2 * 5 + 2] * (-dt * sa) + Jb[2 * 5 + 3] * (-dt * ca) +
            Jb[2 * 5 + 4] * (-dt2 * ca * vx + dt2 * sa * vy) +
            Jb[3 * 5 + 2] * (dt * ca) + Jb[3 * 5 + 3] * (-dt * sa) +
            Jb[3 * 5 + 4] * (-dt2 * sa * vx - dt2 * ca * vy);
}

// The same for the bearings: J_h row j = (-dy, dx, 0, 0, 0) / r^2 with
// (dx, dy) = p - s_j, whose derivatives in (p_x, p_y) are
// [[2 dx dy, dy^2 - dx^2], [dy^2 - dx^2, -2 dx dy]] / r^4.
template <typename T>
SQSM_DEV void ct_jac_h_vjp(const CTParams<T>& P, const T* x, const T* Jb, T* out) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T dx = x[0] - P.sx[j], dy = x[1] - P.sy[j];
    const T r2 = dx * dx + dy * dy;
    const T i4 = T(1) / (r2 * r2);
    const T a = Jb[j * 5 + 0], b = Jb[j * 5 + 1];
    out[0] += (a * T(2) * dx * dy + b * (dy * dy - dx * dx)) * i4;
    out[1] += (a * (dy * dy - dx * dx) - b * T(2) * dx * dy) * i4;
  }
}

template <typename T>
SQSM_DEV void ct_h(const CTParams<T>& P, const T* x, T* o) {
#pragma unroll
  for (int j = 0; j < 2; ++j) o[j] = sq_atan2(x[1] - P.sy[j], x[0] - P.sx[j]);
}

// Signed angle from the line of sight of m to that of m + dl (= the bearing
// of m + dl on the branch nearest h(m), minus h(m)).
template <typename T>
SQSM_DEV void ct_h_delta(const CTParams<T>& P, const T* m, const T* dl, T* o) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T ux = m[0] - P.sx[j], uy = m[1] - P.sy[j];
    const T cross = ux * dl[1] - uy * dl[0];
    const T dot = ux * ux + uy * uy + ux * dl[0] + uy * dl[1];
    o[j] = sq_atan2(cross, dot);
  }
}

// Bearing of m + dl minus the bearing of m, both from absolute positions
// (atan2), wrapped into (-pi, pi] (textbook comparator, see above).
template <typename T>
SQSM_DEV void ct_h_delta_naive(const CTParams<T>& P, const T* m, const T* dl, T* o) {
  const T twopi = T(6.283185307179586476925286766559);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T a = sq_atan2(m[1] + dl[1] - P.sy[j], m[0] + dl[0] - P.sx[j]);
    const T a0 = sq_atan2(m[1] - P.sy[j], m[0] - P.sx[j]);
    const T d = a - a0;
    o[j] = d - twopi * sq_floor(d / twopi + T(0.5));
  }
}

template <typename T>
SQSM_DEV void ct_jac_h(const CTParams<T>& P, const T* x, T* J) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T dx = x[0] - P.sx[j], dy = x[1] - P.sy[j];
    const T r2 = dx * dx + dy * dy;
    J[j * 5 + 0] = -dy / r2;
    J[j * 5 + 1] = dx / r2;
    J[j * 5 + 2] = T(0);
    J[j * 5 + 3] = T(0);
    J[j * 5 + 4] = T(0);
  }
}

// 2 pi multiple that moves y onto the branch nearest the reference bearing.
template <typename T>
SQSM_DEV T branch_shift(T y, T ref) {
  const T twopi = T(6.283185307179586476925286766559);
  return twopi * sq_floor((y - ref) / twopi + T(0.5));
}

// Cubature regression of a function about (m, N): G = D N^{-1} (+ I when
// ADD_I), noise factor Tria([Sc, s_i / sqrt(5)]) and the offset
//   off = gm + dbar - G m   (subtract_Gm: absolute form z_bar - G m), or
//   off = gm + dbar         (deviation form, gm already relative),
// where dbar is the mean of the point differences.  DG(m, dl, out) returns
// the difference at m + dl; with ADD_I it returns that difference minus dl
// (the regression of x itself is exactly I, and the pair means and
// residuals are unchanged because the +-dl of a pair cancel).
// Sigma-point rules with the pair structure m, m +- s N e_i: the cubature
// rule (s^2 = n_x, no centre point) and the unscented transform with
// alpha = 1, beta = 0, kappa = 1 (s^2 = n_x + 1, centre weight
// 1 / (n_x + 1), pair weights 1 / (2 (n_x + 1))).
enum SigmaRule { kCubature = 0, kUnscented = 1 };
constexpr double kUtKappa = 1.0;

template <typename T, int NO, bool ADD_I, typename DG, int RULE = kCubature>
SQSM_DEV void cubature_regress(const T* m, const T* N, const T* gm, bool subtract_Gm,
                               const T* Sc, DG dg, T* G, T* off, T* Sout) {
  constexpr int NX = 5;
  // pair scale s, pair weight w = 1 / (2 s^2), centre weight w0
  constexpr double s2 = RULE == kUnscented ? NX + kUtKappa : NX;
  constexpr double w0 = RULE == kUnscented ? kUtKappa / (NX + kUtKappa) : 0.0;
  const T sq = sq_sqrt(T(s2));
  T D[NO * NX], Hs[NO * NX], dsum[NO];
#pragma unroll
  for (int r = 0; r < NO; ++r) dsum[r] = T(0);
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    T dp[NX], dn[NX], zp[NO], zn[NO];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      dp[r] = sq * N[r * NX + i];
      dn[r] = -dp[r];
    }
    dg(m, dp, zp);
    dg(m, dn, zn);
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      D[r * NX + i] = (zp[r] - zn[r]) / (T(2) * sq);
      Hs[r * NX + i] = T(0.5) * (zp[r] + zn[r]);
      dsum[r] += zp[r] + zn[r];
    }
  }
  // z_bar - g(m): the centre point's difference is 0
  T dbar[NO];
#pragma unroll
  for (int r = 0; r < NO; ++r) dbar[r] = dsum[r] / T(2 * s2);
  rsolve<T, NO, NX>(D, N);           // G = D N^{-1}
  if constexpr (ADD_I) {
    static_assert(NO == NX, "identity split needs a square regression");
#pragma unroll
    for (int r = 0; r < NO; ++r) D[r * NX + r] += T(1);
  }
#pragma unroll
  for (int r = 0; r < NO; ++r) {
    T s = gm[r] + dbar[r];
    if (subtract_Gm) {
#pragma unroll
      for (int k = 0; k < NX; ++k) s -= D[r * NX + k] * m[k];
    }
    off[r] = s;
#pragma unroll
    for (int k = 0; k < NX; ++k) G[r * NX + k] = D[r * NX + k];
  }
  // residual columns sqrt(2 w) ((Z_i^+ + Z_i^-) / 2 - z_bar) (both points of
  // pair i have the same residual), and sqrt(w0) (Z_0 - z_bar) for a centre
  constexpr int C = NO + NX + (w0 > 0.0 ? 1 : 0);
  T B[NO * C];
#pragma unroll
  for (int r = 0; r < NO; ++r) {
#pragma unroll
    for (int j = 0; j < NO; ++j) B[r * C + j] = Sc[r * NO + j];
#pragma unroll
    for (int i = 0; i < NX; ++i) B[r * C + NO + i] = (Hs[r * NX + i] - dbar[r]) / sq;
    if constexpr (w0 > 0.0) B[r * C + NO + NX] = -T(sqrt(w0)) * dbar[r];
  }
  tria<T, NO, C>(B);
  take_lower<T, NO, C>(B, Sout);
}

// The same regression with the tensor-product three-point Gauss-Hermite
// rule (3^n_x points m + N xi, xi_k in {0, +sqrt 3, -sqrt 3}, weights
// prod 2/3, 1/6, 1/6), in two passes over the points because the residuals
// need z_bar and G first: pass 1 accumulates z_bar - g(m) and
// D = sum w (Z - z_bar) xi^T (= the regression times N, as sum w xi xi^T = I);
// pass 2 evaluates the points again and folds the residual columns
// sqrt(w) (Z - z_bar - D xi) into the noise factor K at a time,
// L <- Tria([L, columns]).
template <typename T, int NO, bool ADD_I, typename DG>
SQSM_DEV void gauss_hermite_regress(const T* m, const T* N, const T* gm, bool subtract_Gm,
                                    const T* Sc, DG dg, T* G, T* off, T* Sout) {
  constexpr int NX = 5, NP = 243, K = 5;
  const T r3 = sq_sqrt(T(3));
  auto node = [&](int digit) { return digit == 0 ? T(0) : (digit == 1 ? r3 : -r3); };
  auto weight = [&](int digit) { return digit == 0 ? T(2.0 / 3.0) : T(1.0 / 6.0); };
  T D[NO * NX], dbar[NO];
#pragma unroll
  for (int i = 0; i < NO * NX; ++i) D[i] = T(0);
#pragma unroll
  for (int r = 0; r < NO; ++r) dbar[r] = T(0);
  // the point: xi from the base-3 digits of p, delta = N xi, its weight
  auto point = [&](int p, T* xi, T* dl) -> T {
    T w = T(1);
    int q = p;
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      const int dgt = q % 3;
      q /= 3;
      xi[k] = node(dgt);
      w *= weight(dgt);
    }
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      T a = T(0);
#pragma unroll
      for (int k = 0; k <= r; ++k) a += N[r * NX + k] * xi[k];
      dl[r] = a;
    }
    return w;
  };
#pragma unroll 1
  for (int p = 0; p < NP; ++p) {
    T xi[NX], dl[NX], z[NO];
    const T w = point(p, xi, dl);
    dg(m, dl, z);
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      dbar[r] += w * z[r];
#pragma unroll
      for (int k = 0; k < NX; ++k) D[r * NX + k] += w * z[r] * xi[k];
    }
  }
  // G = D N^{-1} (+ I); the offset as in cubature_regress
#pragma unroll
  for (int i = 0; i < NO * NX; ++i) G[i] = D[i];
  rsolve<T, NO, NX>(G, N);
  if constexpr (ADD_I) {
    static_assert(NO == NX, "identity split needs a square regression");
#pragma unroll
    for (int r = 0; r < NO; ++r) G[r * NX + r] += T(1);
  }
#pragma unroll
  for (int r = 0; r < NO; ++r) {
    T a = gm[r] + dbar[r];
    if (subtract_Gm) {
#pragma unroll
      for (int k = 0; k < NX; ++k) a -= G[r * NX + k] * m[k];
    }
    off[r] = a;
  }
  // pass 2: residual columns folded into L, K points at a time
  T L[NO * NO];
#pragma unroll
  for (int i = 0; i < NO * NO; ++i) L[i] = Sc[i];
  constexpr int C = NO + K;
#pragma unroll 1
  for (int p0 = 0; p0 < NP; p0 += K) {
    T B[NO * C];
#pragma unroll
    for (int r = 0; r < NO; ++r)
#pragma unroll
      for (int j = 0; j < NO; ++j) B[r * C + j] = L[r * NO + j];
#pragma unroll
    for (int q = 0; q < K; ++q) {
      T xi[NX], dl[NX], z[NO];
      const bool valid = p0 + q < NP;   // the last group is partial: zero columns
      const T w = point(valid ? p0 + q : 0, xi, dl);
      dg(m, dl, z);
      const T sw = valid ? sq_sqrt(w) : T(0);
#pragma unroll
      for (int r = 0; r < NO; ++r) {
        T res = z[r] - dbar[r];
#pragma unroll
        for (int k = 0; k < NX; ++k) res -= D[r * NX + k] * xi[k];
        B[r * C + NO + q] = sw * res;
      }
    }
    tria<T, NO, C>(B);
#pragma unroll
    for (int r = 0; r < NO; ++r)
#pragma unroll
      for (int j = 0; j < NO; ++j) L[r * NO + j] = j <= r ? B[r * C + j] : T(0);
  }
#pragma unroll
  for (int i = 0; i < NO * NO; ++i) Sout[i] = L[i];
}

// One thread per step s: the transition is linearised at state row s + b
// (k - 1) and the observation at row s + b + 1 (k) of the nominal trajectory
// `nom`.  PACKED writes one PRec record per step to F (c, SQ, H, d, SR
// unused); otherwise the six arrays are written in the sqsm_ct_linearize
// layout (full matrices, row-major, one per step).
//
// centered = 0: eq. Gamma-s as printed (c = z_bar - F m, d = z_bar - H m).
// centered = 1: the same linear model written for the deviation
// dx_k = x_k - m_k from the nominal trajectory, which keeps every scan
// quantity small in FP32 however large the positions:
//   dx_k = F dx_{k-1} + c~ + q,  c~ = z_bar_x - m_k
//        = (m_{k-1} - m_k) + (f(m_{k-1}) - m_{k-1}) + dbar_x,
//   y_k  = H dx_k + d~ + v,      d~ = H m_k + d = z_bar_y (+ branch shift).
// Steps are independent: one thread per step, addressed as (leaf chunk,
// position in chunk) so that the chunk table gives the sequence; launch
// n_chunks * leaf threads.
//
// Resident blocks per SM the kernel is compiled for: in FP32 the cubature,
// Taylor and unscented rules take five (96 registers, a spill of a few
// words), whose extra warps hide more of the latency of the
// transcendental-heavy model code (5-8% faster than at 120 registers);
// FP64 and the 243-point Gauss-Hermite rule keep their registers.
template <typename T, int LIN> constexpr int slr_min_blocks() {
  return sizeof(T) == 4 && LIN != 3 ? 5 : 1;
}

template <typename T, bool PACKED, typename NO, int LIN, bool TB = false>
__global__ void __launch_bounds__(kBlock, (slr_min_blocks<T, LIN>()))
ct_slr_kernel_lin(DevLevel lv, int leaf, DevSeqs sq, const CTParams<T>* __restrict__ Pp,
              int centered, NO nom, const T* __restrict__ y, T* __restrict__ F,
              T* __restrict__ c, T* __restrict__ SQo, T* __restrict__ H, T* __restrict__ d,
              T* __restrict__ SRo) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ch = tid / leaf;
  if (ch >= lv.n_chunks) return;
  const int j = (int)(tid - ch * leaf);
  if (j >= lv.count[ch]) return;
  constexpr int NX = 5, NY = 2;
  const CTParams<T> P = *Pp;
  const int b = lv.seq[ch];
  {
    const int64_t s = lv.first[ch] + j;
    const int64_t rp = s + b, rk = s + b + 1;
    T m[NX], N[NX * NX];
    // transition at k - 1
    nom.load(rp, m, N);
    T Fm[NX * NX], cm[NX], Sl[NX * NX];
    T fm[NX];    // f(m_{k-1}) (absolute) or f(m_{k-1}) - m_k (deviation form)
    if (centered) {
      T mk[NX];
      nom.load_mean(rk, mk);
      ct_f_minus_x(P, m, fm);
#pragma unroll
      for (int r = 0; r < NX; ++r) fm[r] += m[r] - mk[r];
    } else {
      ct_f(P, m, fm);
    }
    const Turn<T> tm = turn(m[4], P.dt);
    auto gd = [&](const T* mm_, const T* dl, T* o) {
      if constexpr (TB) ct_g_delta_naive(P, mm_, dl, o);
      else ct_g_delta(P, tm, mm_, dl, o);
    };
    if constexpr (LIN == 0) {
      cubature_regress<T, NX, true>(m, N, fm, !centered, P.SQ, gd, Fm, cm, Sl);
    } else if constexpr (LIN == 2) {
      cubature_regress<T, NX, true, decltype(gd), kUnscented>(m, N, fm, !centered, P.SQ, gd, Fm,
                                                               cm, Sl);
    } else if constexpr (LIN == 3) {
      gauss_hermite_regress<T, NX, true>(m, N, fm, !centered, P.SQ, gd, Fm, cm, Sl);
    } else {
      ct_jac_f(P, m, Fm);
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        T sacc = fm[r];
        if (!centered) {
#pragma unroll
          for (int k = 0; k < NX; ++k) sacc -= Fm[r * NX + k] * m[k];
        }
        cm[r] = sacc;
      }
#pragma unroll
      for (int i = 0; i < NX * NX; ++i) Sl[i] = P.SQ[i];
    }
    if constexpr (PACKED) {
      Gamma<T, NX, NY> gg;
      copy<T, NX * NX>(Fm, gg.F);
      copy<T, NX>(cm, gg.c);
      copy<T, NX * NX>(Sl, gg.SQ);
      gg.store_transition(GammaPacked<T>{F}, s);
    } else {
      store<T, NX * NX>(F + s * NX * NX, Fm);
      store<T, NX>(c + s * NX, cm);
      store_lower<T, NX>(SQo + s * NX * NX, Sl);
    }
    // observation at k
    nom.load(rk, m, N);
    T hm[NY], Hm[NY * NX], dm[NY], So[NY * NY], ys[NY];
    load<T, NY>(y + s * NY, ys);
    ct_h(P, m, hm);
    const T Sr[NY * NY] = {P.sigma[0], T(0), T(0), P.sigma[1]};
    auto hd = [&](const T* mm_, const T* dl, T* o) {
      if constexpr (TB) ct_h_delta_naive(P, mm_, dl, o);
      else ct_h_delta(P, mm_, dl, o);
    };
    if constexpr (LIN == 0) {
      cubature_regress<T, NY, false>(m, N, hm, !centered, Sr, hd, Hm, dm, So);
    } else if constexpr (LIN == 2) {
      cubature_regress<T, NY, false, decltype(hd), kUnscented>(m, N, hm, !centered, Sr, hd, Hm, dm,
                                                                So);
    } else if constexpr (LIN == 3) {
      gauss_hermite_regress<T, NY, false>(m, N, hm, !centered, Sr, hd, Hm, dm, So);
    } else {
      ct_jac_h(P, m, Hm);
#pragma unroll
      for (int r = 0; r < NY; ++r) {
        T sacc = hm[r];
        if (!centered) {
#pragma unroll
          for (int k = 0; k < NX; ++k) sacc -= Hm[r * NX + k] * m[k];
        }
        dm[r] = sacc;
      }
      So[0] = P.sigma[0]; So[1] = T(0); So[2] = T(0); So[3] = P.sigma[1];
    }
#pragma unroll
    for (int r = 0; r < NY; ++r) dm[r] += branch_shift(ys[r], hm[r]);
    if constexpr (PACKED) {
      Gamma<T, NX, NY> gg;
      copy<T, NY * NX>(Hm, gg.H);
      copy<T, NY>(dm, gg.d);
      copy<T, NY * NY>(So, gg.SR);
      gg.store_observation(GammaPacked<T>{F}, s);
    } else {
      store<T, NY * NX>(H + s * NY * NX, Hm);
      store<T, NY>(d + s * NY, dm);
      store_lower<T, NY>(SRo + s * NY * NY, So);
    }
  }
}

// ct_slr_kernel_lin for a run-time linearisation (0 cubature, 1 Taylor,
// 2 unscented, 3 Gauss-Hermite): one instantiation per rule, so that each
// keeps its own register budget.
// textbook: the cubature rule with the differences of the printed formulas
// (ct_g_delta_naive, ct_h_delta_naive) instead of the cancellation-free ones.
template <typename T, bool PACKED, typename NO>
void launch_ct_slr(unsigned grid, cudaStream_t s, int linearization, DevLevel lv, int leaf,
                   DevSeqs sq, const CTParams<T>* Pp, int centered, NO nom, const T* y, T* F,
                   T* c, T* SQo, T* H, T* d, T* SRo, int textbook = 0) {
  if (textbook && linearization == 0) {
    ct_slr_kernel_lin<T, PACKED, NO, 0, true><<<grid, kBlock, 0, s>>>(lv, leaf, sq, Pp, centered,
                                                                       nom, y, F, c, SQo, H, d,
                                                                       SRo);
    return;
  }
  switch (linearization) {
    case 0:
      ct_slr_kernel_lin<T, PACKED, NO, 0><<<grid, kBlock, 0, s>>>(lv, leaf, sq, Pp, centered, nom,
                                                                   y, F, c, SQo, H, d, SRo);
      break;
    case 2:
      ct_slr_kernel_lin<T, PACKED, NO, 2><<<grid, kBlock, 0, s>>>(lv, leaf, sq, Pp, centered, nom,
                                                                   y, F, c, SQo, H, d, SRo);
      break;
    case 3:
      ct_slr_kernel_lin<T, PACKED, NO, 3><<<grid, kBlock, 0, s>>>(lv, leaf, sq, Pp, centered, nom,
                                                                   y, F, c, SQo, H, d, SRo);
      break;
    default:
      ct_slr_kernel_lin<T, PACKED, NO, 1><<<grid, kBlock, 0, s>>>(lv, leaf, sq, Pp, centered, nom,
                                                                   y, F, c, SQo, H, d, SRo);
      break;
  }
}

// Initial nominal trajectory (Alg. 3 input): the prior of each sequence
// broadcast to all of its state rows.  One thread per smoother leaf chunk.
template <typename T, int NX, typename SO>
__global__ void __launch_bounds__(kBlock)
broadcast_prior_kernel(DevLevel lv, const T* __restrict__ m0, const T* __restrict__ N0, SO so) {
  const int64_t ch = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ch >= lv.n_chunks) return;
  const int b = lv.seq[ch];
  T m[NX], N[NX * NX];
  load<T, NX>(m0 + (int64_t)b * NX, m);
  load_lower<T, NX>(N0 + (int64_t)b * NX * NX, N);
  for (int j = 0; j < lv.count[ch]; ++j) {
    so.store(lv.first[ch] + j, m, N);
  }
}

// Copy of state rows between layouts, one thread per row.
template <typename T, int NX, typename RI, typename RO>
__global__ void __launch_bounds__(kBlock) rows_copy_kernel(int64_t rows, RI in, RO out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= rows) return;
  T m[NX], N[NX * NX];
  in.load(e, m, N);
  out.store(e, m, N);
}

// Error-free transformations (Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005): TwoSum (Knuth) gives s + e = a + b
// exactly with s = fl(a + b); TwoProduct with an FMA gives p + e = a b
// exactly.  The explicit round-to-nearest intrinsics keep the compiler from
// contracting or reordering them.
SQSM_DEV void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
SQSM_DEV void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// r = x0 + sum_k A[k] (v_hi[k] + v_lo[k]) in the Dot2 scheme of the paper
// above: the leading sum carried by TwoSum / TwoProduct, every rounding error
// (and the products with v_lo) summed into a correction added once at the
// end -- as accurate as the sum computed in twice the working precision and
// then rounded.
template <int N>
SQSM_DEV float dot2(float s, float comp, const float* A, const float* vh, const float* vl) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float p, pe, e;
    two_prod(A[k], vh[k], p, pe);
    two_sum(s, p, s, e);
    comp = __fadd_rn(comp, __fadd_rn(e, pe));
    comp = __fmaf_rn(A[k], vl[k], comp);
  }
  return __fadd_rn(s, comp);
}

// Residual model of one refinement pass of the linear smoother (mixed
// precision iterative refinement).  The smoother of the linearised model in
// deviation coordinates about m (the iteration's nominal means, rows
// prev) returned n1 = m + dx; the correction delta = x - n1 solves the same
// linear-Gaussian model about n1, whose offsets are, with dx = n1 - m,
//   c' = F dx_{k-1} + c~ - dx_k,   d' = d~ + H dx_k
// (x_k = F x_{k-1} + c~ + q and y_k = H x_k + d~ + r written for x - dx);
// the prior's is dm0 - dx_0 (center_prior_kernel on n1).  The offsets are
// formed from the stored values beyond the working precision and rounded
// once when written back into the PRec records in place: in FP32, dx exactly
// as a TwoSum pair and the sums by Dot2 (FP64 arithmetic, far slower on this
// GPU, is not needed for that accuracy); in FP64, in plain FP64.  One thread
// per step.
template <typename T, int NX, int NY, typename RI>
__global__ void __launch_bounds__(kBlock)
refine_residual_kernel(DevLevel lv, int leaf, RI prev, RI now, T* __restrict__ rec) {
  using P = PRec<NX, NY>;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ch = tid / leaf;
  if (ch >= lv.n_chunks) return;
  const int j = (int)(tid - ch * leaf);
  if (j >= lv.count[ch]) return;
  const int b = lv.seq[ch];
  const int64_t s = lv.first[ch] + j;
  const int64_t rp = s + b, rk = s + b + 1;
  T m0v[NX], m1v[NX], k0v[NX], k1v[NX];
  prev.load_mean(rp, m0v);
  now.load_mean(rp, m1v);
  prev.load_mean(rk, k0v);
  now.load_mean(rk, k1v);
  // the record's 16-byte words that hold F, c (from word 0) and H, d (from
  // P::H), read whole; only the words holding c and d are written back
  static_assert(P::F == 0 && P::c == NX * NX && P::d == P::H + NY * NX && P::H % 4 == 0,
                "PRec layout");
  constexpr int LA = (P::c + NX + 3) / 4 * 4, LB = (NY * NX + NY + 3) / 4 * 4;
  constexpr int C0 = P::c / 4 * 4, D0 = NY * NX / 4 * 4;
  T* r = rec + s * P::size;
  T fa[LA], ha[LB];
  vload<T, LA>(r, fa);
  vload<T, LB>(r + P::H, ha);
  if constexpr (sizeof(T) == 4) {
    float dph[NX], dpl[NX], dkh[NX], dkl[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      two_sum(m1v[i], -m0v[i], dph[i], dpl[i]);
      two_sum(k1v[i], -k0v[i], dkh[i], dkl[i]);
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      float s0, e0;
      two_sum(fa[P::c + i], -dkh[i], s0, e0);
      fa[P::c + i] = dot2<NX>(s0, __fsub_rn(e0, dkl[i]), fa + i * NX, dph, dpl);
    }
#pragma unroll
    for (int i = 0; i < NY; ++i)
      ha[NY * NX + i] = dot2<NX>(ha[NY * NX + i], 0.f, ha + i * NX, dkh, dkl);
  } else {
    double dp[NX], dk[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      dp[i] = (double)m1v[i] - (double)m0v[i];
      dk[i] = (double)k1v[i] - (double)k0v[i];
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      double a = (double)fa[P::c + i] - dk[i];
#pragma unroll
      for (int k = 0; k < NX; ++k) a += (double)fa[i * NX + k] * dp[k];
      fa[P::c + i] = (T)a;
    }
#pragma unroll
    for (int i = 0; i < NY; ++i) {
      double a = (double)ha[NY * NX + i];
#pragma unroll
      for (int k = 0; k < NX; ++k) a += (double)ha[i * NX + k] * dk[k];
      ha[NY * NX + i] = (T)a;
    }
  }
  vstore<T, LA - C0>(r + C0, fa + C0);
  vstore<T, LB - D0>(r + P::H + D0, ha + D0);
}

// Prior of the deviation model: dm0[b] = m0[b] - m_0 (nominal row 0 of b).
template <typename T, int NX, typename RI>
__global__ void center_prior_kernel(DevSeqs sq, const T* __restrict__ m0, RI nom,
                                    T* __restrict__ dm0) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= sq.B) return;
  T mn[NX];
  nom.load_mean(sq.offsets[b] + b, mn);
#pragma unroll
  for (int i = 0; i < NX; ++i) dm0[(int64_t)b * NX + i] = m0[(int64_t)b * NX + i] - mn[i];
}

}  // namespace sqsm
