// Standard (covariance) form of the parallel filter and smoother -- the left
// columns of Tables 1-5 -- and of the cubature SLR (Sec. 4.1 with
// covariances), inside the same IPLS loop (Alg. 3) as the square-root form.
// It exists to measure what the paper's square-root form buys in FP32
// (Sec. 6: the standard form's covariances lose positive definiteness and
// the run diverges); the scan shape is the fold-only plan (4 items per thread
// at every upper level), the coordinates are the same deviation coordinates.
//
// Records reuse the square-root layouts with full symmetric matrices in the
// factor slots: filter (A, b, C, eta, J), smoother (E, g, L); the linearised
// model record holds Lambda and Omega (lower triangle, symmetric) where the
// square-root form holds S_Lambda and S_Omega; state rows hold (m, P) with P
// as its lower triangle.
#pragma once

#include "ct_model.cuh"
#include "dispatch.h"

namespace sqsm {

// ---------------------------------------------------------------------------
// small dense helpers
// ---------------------------------------------------------------------------

// B (N x M) <- (L L^T)^{-1} B for lower L.
template <typename T, int N, int M>
SQSM_DEV void chol_solve(const T* L, T* B) {
#pragma unroll
  for (int c = 0; c < M; ++c) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s = B[i * M + c];
#pragma unroll
      for (int k = 0; k < i; ++k) s -= L[i * N + k] * B[k * M + c];
      B[i * M + c] = s / L[i * N + i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      T s = B[i * M + c];
#pragma unroll
      for (int k = i + 1; k < N; ++k) s -= L[k * N + i] * B[k * M + c];
      B[i * M + c] = s / L[i * N + i];
    }
  }
}

// X = A^{-1} by Gauss-Jordan elimination with partial pivoting (rows are
// swapped by selection, so the code has no data-dependent branch); A is
// destroyed.
template <typename T, int N>
SQSM_DEV void gj_inverse(T* A, T* X) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) X[i * N + j] = i == j ? T(1) : T(0);
#pragma unroll
  for (int k = 0; k < N; ++k) {
    int p = k;
    T best = fabs(A[k * N + k]);
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const T v = fabs(A[i * N + k]);
      const bool bigger = v > best;
      best = bigger ? v : best;
      p = bigger ? i : p;
    }
#pragma unroll
    for (int i = k + 1; i < N; ++i) {
      const bool sw = i == p;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const T a = A[k * N + j], b = A[i * N + j];
        A[k * N + j] = sw ? b : a;
        A[i * N + j] = sw ? a : b;
        const T x = X[k * N + j], z = X[i * N + j];
        X[k * N + j] = sw ? z : x;
        X[i * N + j] = sw ? x : z;
      }
    }
    const T inv = T(1) / A[k * N + k];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      A[k * N + j] *= inv;
      X[k * N + j] *= inv;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const T f = A[i * N + k];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        A[i * N + j] -= f * A[k * N + j];
        X[i * N + j] -= f * X[k * N + j];
      }
    }
  }
}

// C = A B A^T for A (M x K), symmetric B (K x K).
template <typename T, int M, int K>
SQSM_DEV void abat(const T* A, const T* B, T* C) {
  T AB[M * K];
  mm<T, M, K, K>(A, B, AB);
  mmt<T, M, K, M>(AB, A, C);
}

// ---------------------------------------------------------------------------
// packed storage with symmetric matrices
// ---------------------------------------------------------------------------

// The linearised model of step t: F, c, Lambda (full), H, d, Omega (full).
template <typename T, int NX, int NY>
struct GammaStd {
  T F[NX * NX], c[NX], Q[NX * NX], H[NY * NX], d[NY], R[NY * NY];

  SQSM_DEV void load_transition(const GammaPacked<T>& g, int64_t t) {
    using P = PRec<NX, NY>;
    T v[P::H];
    vload<T, P::H>(g.rec + t * P::size, v);
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) F[i] = v[P::F + i];
#pragma unroll
    for (int i = 0; i < NX; ++i) c[i] = v[P::c + i];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) Q[i * NX + j] = Q[j * NX + i] = v[P::SQ + i * (i + 1) / 2 + j];
  }
  SQSM_DEV void load_all(const GammaPacked<T>& g, int64_t t) {
    using P = PRec<NX, NY>;
    load_transition(g, t);
    T v[P::size - P::H];
    vload<T, P::size - P::H>(g.rec + t * P::size + P::H, v);
#pragma unroll
    for (int i = 0; i < NY * NX; ++i) H[i] = v[i];
#pragma unroll
    for (int i = 0; i < NY; ++i) d[i] = v[P::d - P::H + i];
#pragma unroll
    for (int i = 0; i < NY; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j)
        R[i * NY + j] = R[j * NY + i] = v[P::SR - P::H + i * (i + 1) / 2 + j];
  }
};

// State rows (m, P) with P symmetric, packed as RowsPacked (lower triangle).
template <typename T, int NX>
struct RowsSym {
  T* rec;
  SQSM_DEV void load(int64_t e, T* mo, T* Po) const {
    using R = XRow<NX>;
    T v[R::size];
    vload<T, R::size>(rec + e * R::size, v);
#pragma unroll
    for (int i = 0; i < NX; ++i) mo[i] = v[i];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) Po[i * NX + j] = Po[j * NX + i] = v[NX + i * (i + 1) / 2 + j];
  }
  SQSM_DEV void load_mean(int64_t e, T* mo) const { RowsPacked<T, NX>{rec}.load_mean(e, mo); }
  SQSM_DEV void store(int64_t e, const T* mi, const T* Pi) const {
    RowsPacked<T, NX>{rec}.store(e, mi, Pi);   // keeps the lower triangle
  }
};

// Caller arrays (m, full symmetric P), m and P of one row contiguous.
template <typename T, int NX>
struct RowsSplitSym {
  T* m;
  T* P;
  SQSM_DEV void load(int64_t e, T* mo, T* Po) const {
    sqsm::load<T, NX>(m + e * NX, mo);
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) Po[i * NX + j] = Po[j * NX + i] = P[e * NX * NX + i * NX + j];
  }
  SQSM_DEV void load_mean(int64_t e, T* mo) const { sqsm::load<T, NX>(m + e * NX, mo); }
  SQSM_DEV void store(int64_t e, const T* mi, const T* Pi) const {
    sqsm::store<T, NX>(m + e * NX, mi);
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j < NX; ++j)
        P[e * NX * NX + i * NX + j] = j <= i ? Pi[i * NX + j] : Pi[j * NX + i];
  }
};

// ---------------------------------------------------------------------------
// elements and operators (left columns of Tables 1-5)
// ---------------------------------------------------------------------------

// K = P H^T S^{-1} with S = H P H^T + R (its Cholesky factor in Ls); a
// non-definite S gives NaN.
template <typename T, int NX, int NY>
SQSM_DEV void std_gain(const T* P, const T* H, const T* R, T* K, T* Ls) {
  T HP[NY * NX];
  mm<T, NY, NX, NX>(H, P, HP);
  mmt<T, NY, NX, NY>(HP, H, Ls);
#pragma unroll
  for (int i = 0; i < NY * NY; ++i) Ls[i] += R[i];
  chol_inplace<T, NY>(Ls);
  chol_solve<T, NY, NX>(Ls, HP);   // S^{-1} H P
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NY; ++j) K[i * NY + j] = HP[j * NX + i];
}

// Filter element, Table 1 (first) / Table 2, left column; b uses d_k, eta is
// read without the extra H (the readings of the square-root form).
template <typename T, int NX, int NY>
SQSM_DEV void std_filter_element(const GammaStd<T, NX, NY>& g, const T* y, bool first,
                                 const T* m0, const T* P0, T* e) {
  using R = FRec<NX>;
  T mp[NX], Pp[NX * NX];
  if (first) {
    mv<T, NX, NX>(g.F, m0, mp);
#pragma unroll
    for (int i = 0; i < NX; ++i) mp[i] += g.c[i];
    abat<T, NX, NX>(g.F, P0, Pp);
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) Pp[i] += g.Q[i];
  } else {
#pragma unroll
    for (int i = 0; i < NX; ++i) mp[i] = g.c[i];
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) Pp[i] = g.Q[i];
  }
  T K[NX * NY], Ls[NY * NY];
  std_gain<T, NX, NY>(Pp, g.H, g.R, K, Ls);
  // innovation about the predicted mean (k = 1) / about c (k > 1)
  T v[NY];
  mv<T, NY, NX>(g.H, mp, v);
#pragma unroll
  for (int i = 0; i < NY; ++i) v[i] = y[i] - v[i] - g.d[i];
  T Kv[NX];
  mv<T, NX, NY>(K, v, Kv);
#pragma unroll
  for (int i = 0; i < NX; ++i) e[R::b + i] = mp[i] + Kv[i];
  // I - K H
  T IKH[NX * NX];
  mm<T, NX, NY, NX>(K, g.H, IKH);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) IKH[i] = (i % (NX + 1) == 0 ? T(1) : T(0)) - IKH[i];
  if (first) {
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) e[R::A + i] = T(0);
  } else {
    mm<T, NX, NX, NX>(IKH, g.F, e + R::A);
  }
  mm<T, NX, NX, NX>(IKH, Pp, e + R::U);   // C = (I - K H) P^-
  // eta = (HF)^T S^{-1} (y - H c - d), J = (HF)^T S^{-1} H F
  T HF[NY * NX], Si_HF[NY * NX], r[NY];
  mm<T, NY, NX, NX>(g.H, g.F, HF);
#pragma unroll
  for (int i = 0; i < NY * NX; ++i) Si_HF[i] = HF[i];
  chol_solve<T, NY, NX>(Ls, Si_HF);
  mv<T, NY, NX>(g.H, g.c, r);
#pragma unroll
  for (int i = 0; i < NY; ++i) r[i] = y[i] - r[i] - g.d[i];
  chol_solve<T, NY, 1>(Ls, r);
  mtv<T, NY, NX>(HF, r, e + R::eta);
  mtm<T, NX, NY, NX>(HF, Si_HF, e + R::Z);
  zero_pad<T, R::Z + NX * NX, R::size>(e);
}

// Table 3, left column: out = e_i (x) e_j, with M = (I + C_i J_j)^{-1} and
// (I + J_j C_i)^{-1} = M^T (C, J symmetric).
template <typename T, int NX>
SQSM_DEV void std_filter_combine(const T* ei, const T* ej, T* out) {
  using R = FRec<NX>;
  T W[NX * NX], Mi[NX * NX];
  mm<T, NX, NX, NX>(ei + R::U, ej + R::Z, W);
#pragma unroll
  for (int i = 0; i < NX; ++i) W[i * NX + i] += T(1);
  gj_inverse<T, NX>(W, Mi);
  T AjM[NX * NX];
  mm<T, NX, NX, NX>(ej + R::A, Mi, AjM);
  mm<T, NX, NX, NX>(AjM, ei + R::A, out + R::A);
  T u[NX], t[NX];
  mv<T, NX, NX>(ei + R::U, ej + R::eta, u);
#pragma unroll
  for (int i = 0; i < NX; ++i) u[i] += ei[R::b + i];
  mv<T, NX, NX>(AjM, u, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) out[R::b + i] = t[i] + ej[R::b + i];
  T AMC[NX * NX];
  mm<T, NX, NX, NX>(AjM, ei + R::U, AMC);
  mmt<T, NX, NX, NX>(AMC, ej + R::A, out + R::U);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) out[R::U + i] += ej[R::U + i];
  // MA = M A_i: eta_ij = (M A_i)^T (eta_j - J_j b_i) + eta_i,
  //             J_ij   = (M A_i)^T J_j A_i + J_i
  T MA[NX * NX];
  mm<T, NX, NX, NX>(Mi, ei + R::A, MA);
  mv<T, NX, NX>(ej + R::Z, ei + R::b, u);
#pragma unroll
  for (int i = 0; i < NX; ++i) u[i] = ej[R::eta + i] - u[i];
  mtv<T, NX, NX>(MA, u, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) out[R::eta + i] = t[i] + ei[R::eta + i];
  T JA[NX * NX];
  mm<T, NX, NX, NX>(ej + R::Z, ei + R::A, JA);
  mtm<T, NX, NX, NX>(MA, JA, out + R::Z);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) out[R::Z + i] += ei[R::Z + i];
  zero_pad<T, R::Z + NX * NX, R::size>(out);
}

// Table 3 left with a filtering distribution (m, P) on the left (A_i = 0):
// (m, P) <- (b_ij, C_ij).
template <typename T, int NX>
SQSM_DEV void std_filter_apply(T* m, T* P, const T* ej) {
  using R = FRec<NX>;
  T W[NX * NX], Mi[NX * NX];
  mm<T, NX, NX, NX>(P, ej + R::Z, W);
#pragma unroll
  for (int i = 0; i < NX; ++i) W[i * NX + i] += T(1);
  gj_inverse<T, NX>(W, Mi);
  T AjM[NX * NX];
  mm<T, NX, NX, NX>(ej + R::A, Mi, AjM);
  T u[NX], t[NX];
  mv<T, NX, NX>(P, ej + R::eta, u);
#pragma unroll
  for (int i = 0; i < NX; ++i) u[i] += m[i];
  mv<T, NX, NX>(AjM, u, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) m[i] = t[i] + ej[R::b + i];
  T AMP[NX * NX];
  mm<T, NX, NX, NX>(AjM, P, AMP);
  mmt<T, NX, NX, NX>(AMP, ej + R::A, P);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) P[i] += ej[R::U + i];
}

// Covariance Kalman step (Table 1 left with (m0, P0) replaced by (m, P));
// returns l_k.
template <typename T, int NX, int NY>
SQSM_DEV T std_kf_step(const GammaStd<T, NX, NY>& g, const T* y, T* m, T* P) {
  T mp[NX], Pp[NX * NX];
  mv<T, NX, NX>(g.F, m, mp);
#pragma unroll
  for (int i = 0; i < NX; ++i) mp[i] += g.c[i];
  abat<T, NX, NX>(g.F, P, Pp);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) Pp[i] += g.Q[i];
  T K[NX * NY], Ls[NY * NY], v[NY];
  std_gain<T, NX, NY>(Pp, g.H, g.R, K, Ls);
  mv<T, NY, NX>(g.H, mp, v);
#pragma unroll
  for (int i = 0; i < NY; ++i) v[i] = y[i] - v[i] - g.d[i];
  T Kv[NX];
  mv<T, NX, NY>(K, v, Kv);
#pragma unroll
  for (int i = 0; i < NX; ++i) m[i] = mp[i] + Kv[i];
  T KH[NX * NX];
  mm<T, NX, NY, NX>(K, g.H, KH);
  T KHP[NX * NX];
  mm<T, NX, NX, NX>(KH, Pp, KHP);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) P[i] = Pp[i] - KHP[i];
  // l = -1/2 (ny log 2 pi + log det S + v^T S^{-1} v), S = Ls Ls^T
  T w[NY], ld = T(0), q = T(0);
#pragma unroll
  for (int i = 0; i < NY; ++i) {
    T s = v[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= Ls[i * NY + k] * w[k];
    w[i] = s / Ls[i * NY + i];
    q += w[i] * w[i];
    ld += sq_log(Ls[i * NY + i]);
  }
  return T(-0.5) * (T(NY) * T(kLog2Pi) + T(2) * ld + q);
}

// Table 4, left column (0 <= k < n): E = P F^T (F P F^T + Q)^{-1},
// g = m - E (F m + c), L = P - E F P.
template <typename T, int NX, int NY>
SQSM_DEV void std_smoother_element(const GammaStd<T, NX, NY>& g, const T* mf, const T* Pf, T* e) {
  using R = SRec<NX>;
  T Pp[NX * NX], FP[NX * NX];
  abat<T, NX, NX>(g.F, Pf, Pp);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) Pp[i] += g.Q[i];
  chol_inplace<T, NX>(Pp);
  mm<T, NX, NX, NX>(g.F, Pf, FP);
  T X[NX * NX];
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) X[i] = FP[i];
  chol_solve<T, NX, NX>(Pp, X);   // (F P F^T + Q)^{-1} F P = E^T
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) e[R::E + i * NX + j] = X[j * NX + i];
  T fm[NX], t[NX];
  mv<T, NX, NX>(g.F, mf, fm);
#pragma unroll
  for (int i = 0; i < NX; ++i) fm[i] += g.c[i];
  mv<T, NX, NX>(e + R::E, fm, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) e[R::g + i] = mf[i] - t[i];
  T EFP[NX * NX];
  mm<T, NX, NX, NX>(e + R::E, FP, EFP);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) e[R::D + i] = Pf[i] - EFP[i];
  zero_pad<T, R::D + NX * NX, R::size>(e);
}

template <typename T, int NX>
SQSM_DEV void std_smoother_element_last(const T* mf, const T* Pf, T* e) {
  using R = SRec<NX>;
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) {
    e[R::E + i] = T(0);
    e[R::D + i] = Pf[i];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) e[R::g + i] = mf[i];
  zero_pad<T, R::D + NX * NX, R::size>(e);
}

// Table 5, left column: (E_i E_j, E_i g_j + g_i, E_i L_j E_i^T + L_i).
template <typename T, int NX>
SQSM_DEV void std_smoother_combine(const T* ei, const T* ej, T* out) {
  using R = SRec<NX>;
  mm<T, NX, NX, NX>(ei + R::E, ej + R::E, out + R::E);
  T t[NX];
  mv<T, NX, NX>(ei + R::E, ej + R::g, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) out[R::g + i] = t[i] + ei[R::g + i];
  abat<T, NX, NX>(ei + R::E, ej + R::D, out + R::D);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) out[R::D + i] += ei[R::D + i];
  zero_pad<T, R::D + NX * NX, R::size>(out);
}

// Table 5 left with a smoothing distribution (g, L) on the right (E_j = 0).
template <typename T, int NX>
SQSM_DEV void std_smoother_apply(const T* ei, T* g, T* L) {
  using R = SRec<NX>;
  T t[NX], EL[NX * NX];
  mv<T, NX, NX>(ei + R::E, g, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) g[i] = t[i] + ei[R::g + i];
  abat<T, NX, NX>(ei + R::E, L, EL);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) L[i] = EL[i] + ei[R::D + i];
}

// ---------------------------------------------------------------------------
// covariance-form cubature SLR (Sec. 4.1 with covariances)
// ---------------------------------------------------------------------------

// As cubature_regress, but with the noise covariance
//   Lambda = Phi - G P G^T + Qc,  Phi = sum_i w (Z_i - z_bar)(Z_i - z_bar)^T
// in place of the square-root residual factor.  ADD_I: dg returns
// differences of f(x) - x, so Z_i - z_bar = (X_i - m) + (dg_i - dbar).
template <typename T, int NO, bool ADD_I, typename DG>
SQSM_DEV void cubature_regress_std(const T* m, const T* N, const T* P, const T* gm,
                                   const T* Qc, DG dg, T* G, T* off, T* Lam) {
  constexpr int NX = 5;
  const T sq = sq_sqrt(T(NX));
  const T w = T(1) / T(2 * NX);
  T D[NO * NX], dsum[NO], Phi2[NO * NO];   // Phi2 = sum over points of u u^T (before / w)
#pragma unroll
  for (int r = 0; r < NO; ++r) dsum[r] = T(0);
#pragma unroll
  for (int i = 0; i < NO * NO; ++i) Phi2[i] = T(0);
  T zs[2 * NX][NO];
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    T dp[NX], dn[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      dp[r] = sq * N[r * NX + i];
      dn[r] = -dp[r];
    }
    dg(m, dp, zs[2 * i]);
    dg(m, dn, zs[2 * i + 1]);
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      D[r * NX + i] = (zs[2 * i][r] - zs[2 * i + 1][r]) / (T(2) * sq);
      dsum[r] += zs[2 * i][r] + zs[2 * i + 1][r];
    }
  }
  T dbar[NO];
#pragma unroll
  for (int r = 0; r < NO; ++r) dbar[r] = dsum[r] / T(2 * NX);
#pragma unroll
  for (int p = 0; p < 2 * NX; ++p) {
    T u[NO];
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      T x = zs[p][r] - dbar[r];
      if constexpr (ADD_I) x += (p % 2 == 0 ? sq : -sq) * N[r * NX + p / 2];
      u[r] = x;
    }
#pragma unroll
    for (int r = 0; r < NO; ++r)
#pragma unroll
      for (int q = 0; q < NO; ++q) Phi2[r * NO + q] += u[r] * u[q];
  }
  rsolve<T, NO, NX>(D, N);           // G = D N^{-1}
  if constexpr (ADD_I) {
#pragma unroll
    for (int r = 0; r < NO; ++r) D[r * NX + r] += T(1);
  }
#pragma unroll
  for (int r = 0; r < NO; ++r) {
    off[r] = gm[r] + dbar[r];
#pragma unroll
    for (int k = 0; k < NX; ++k) G[r * NX + k] = D[r * NX + k];
  }
  T GPG[NO * NO];
  abat<T, NO, NX>(D, P, GPG);
#pragma unroll
  for (int i = 0; i < NO * NO; ++i) Lam[i] = w * Phi2[i] - GPG[i] + Qc[i];
}

// One thread per step: the covariance-form linearisation of step s about
// the nominal rows (m, P), cubature (linearization 0: Sec. 4.1 with sigma
// points) or Taylor (1: Jacobians, Lambda = Q, Omega = R); centered as in
// ct_slr_kernel (1: deviation form, 0: the printed absolute form).
template <typename T, typename NO, bool TB = false>
__global__ void __launch_bounds__(kBlock)
std_slr_kernel(DevLevel lv, int leaf, DevSeqs sq, const CTParams<T>* __restrict__ Pp, NO nom,
               int linearization, int centered, const T* __restrict__ y, T* __restrict__ gam) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ch = tid / leaf;
  if (ch >= lv.n_chunks) return;
  const int j = (int)(tid - ch * leaf);
  if (j >= lv.count[ch]) return;
  constexpr int NX = 5, NY = 2;
  const CTParams<T> P = *Pp;
  const int b = lv.seq[ch];
  const int64_t s = lv.first[ch] + j;
  const int64_t rp = s + b, rk = s + b + 1;
  Gamma<T, NX, NY> out;   // stored through the packed record (lower triangles)
  {
    T m[NX], Pc[NX * NX], N[NX * NX], mk[NX], fm[NX];
    nom.load(rp, m, Pc);
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) N[i] = Pc[i];
    chol_inplace<T, NX>(N);
    if (centered) {
      nom.load_mean(rk, mk);
      ct_f_minus_x(P, m, fm);
#pragma unroll
      for (int r = 0; r < NX; ++r) fm[r] += m[r] - mk[r];
    } else {
      ct_f(P, m, fm);
    }
    T Qc[NX * NX];
    mmt<T, NX, NX, NX>(P.SQ, P.SQ, Qc);   // Q = S_Q S_Q^T
    if (linearization == 0) {
      const Turn<T> tm = turn(m[4], P.dt);
      cubature_regress_std<T, NX, true>(
          m, N, Pc, fm, Qc,
          [&](const T* mm_, const T* dl, T* o) {
            if constexpr (TB) ct_g_delta_naive(P, mm_, dl, o);
            else ct_g_delta(P, tm, mm_, dl, o);
          },
          out.F, out.c, out.SQ);
    } else {
      ct_jac_f(P, m, out.F);
#pragma unroll
      for (int i = 0; i < NX * NX; ++i) out.SQ[i] = Qc[i];
#pragma unroll
      for (int r = 0; r < NX; ++r) out.c[r] = fm[r];
    }
    if (!centered) {   // c = z_bar - F m
#pragma unroll
      for (int r = 0; r < NX; ++r)
#pragma unroll
        for (int k = 0; k < NX; ++k) out.c[r] -= out.F[r * NX + k] * m[k];
    }
    out.store_transition(GammaPacked<T>{gam}, s);
  }
  {
    T m[NX], Pc[NX * NX], N[NX * NX];
    nom.load(rk, m, Pc);
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) N[i] = Pc[i];
    chol_inplace<T, NX>(N);
    T hm[NY], ys[NY];
    load<T, NY>(y + s * NY, ys);
    ct_h(P, m, hm);
    const T Rc[NY * NY] = {P.sigma[0] * P.sigma[0], T(0), T(0), P.sigma[1] * P.sigma[1]};
    if (linearization == 0) {
      cubature_regress_std<T, NY, false>(
          m, N, Pc, hm, Rc,
          [&](const T* mm_, const T* dl, T* o) {
            if constexpr (TB) ct_h_delta_naive(P, mm_, dl, o);
            else ct_h_delta(P, mm_, dl, o);
          },
          out.H, out.d, out.SR);
    } else {
      ct_jac_h(P, m, out.H);
#pragma unroll
      for (int i = 0; i < NY * NY; ++i) out.SR[i] = Rc[i];
#pragma unroll
      for (int r = 0; r < NY; ++r) out.d[r] = hm[r];
    }
    if (!centered) {   // d = z_bar - H m
#pragma unroll
      for (int r = 0; r < NY; ++r)
#pragma unroll
        for (int k = 0; k < NX; ++k) out.d[r] -= out.H[r * NX + k] * m[k];
    }
#pragma unroll
    for (int r = 0; r < NY; ++r) out.d[r] += branch_shift(ys[r], hm[r]);
    out.store_observation(GammaPacked<T>{gam}, s);
  }
}

// ---------------------------------------------------------------------------
// scan kernels (fold-only plan: every level folds up to R items per thread)
// ---------------------------------------------------------------------------

template <typename T, int NX, int NY>
__global__ void __launch_bounds__(kBlock)
std_filter_leaf_up(DevLevel lv, DevSeqs sq, GammaPacked<T> gv, const T* __restrict__ y,
                   const T* __restrict__ m0, const T* __restrict__ P0, T* __restrict__ items) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = FRec<NX>::size;
  const int b = lv.seq[c];
  const int64_t s0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t off = sq.offsets[b];
  T agg[REC], el[REC], tmp[REC];
  T m0b[NX], P0b[NX * NX];
  load<T, NX>(m0 + (int64_t)b * NX, m0b);
  load<T, NX * NX>(P0 + (int64_t)b * NX * NX, P0b);
  for (int j = 0; j < cnt; ++j) {
    const int64_t s = s0 + j;
    GammaStd<T, NX, NY> g;
    g.load_all(gv, s);
    T ys[NY];
    load<T, NY>(y + s * NY, ys);
    std_filter_element<T, NX, NY>(g, ys, s == off, m0b, P0b, j == 0 ? agg : el);
    if (j > 0) {
      std_filter_combine<T, NX>(agg, el, tmp);
      copy<T, REC>(tmp, agg);
    }
  }
  vstore<T, REC>(items + c * REC, agg);
}

template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
std_filter_up(DevLevel lv, const T* __restrict__ in, T* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = FRec<NX>::size;
  const int64_t i0 = lv.first[c];
  T agg[REC], el[REC], tmp[REC];
  vload<T, REC>(in + i0 * REC, agg);
  for (int j = 1; j < lv.count[c]; ++j) {
    vload<T, REC>(in + (i0 + j) * REC, el);
    std_filter_combine<T, NX>(agg, el, tmp);
    copy<T, REC>(tmp, agg);
  }
  vstore<T, REC>(out + c * REC, agg);
}

// Carries (b, C) = the filtering distribution before each item; flag 0: none.
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
std_filter_down(DevLevel lv, const T* __restrict__ items, const T* __restrict__ cin,
                const int* __restrict__ fin, T* __restrict__ cout, int* __restrict__ fout) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = FRec<NX>::size, CREC = NX + NX * NX;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  int flag = fin[c];
  T m[NX], P[NX * NX];
  load<T, NX>(cin + c * CREC, m);
  load<T, NX * NX>(cin + c * CREC + NX, P);
  for (int j = 0; j < cnt; ++j) {
    const int64_t i = i0 + j;
    store<T, NX>(cout + i * CREC, m);
    store<T, NX * NX>(cout + i * CREC + NX, P);
    fout[i] = flag;
    if (j + 1 < cnt) {
      T el[REC];
      vload<T, REC>(items + i * REC, el);
      if (flag) {
        std_filter_apply<T, NX>(m, P, el);
      } else {
        copy<T, NX>(el + FRec<NX>::b, m);
        copy<T, NX * NX>(el + FRec<NX>::U, P);
        flag = 1;
      }
    }
  }
}

template <typename T, int NX, int NY>
__global__ void __launch_bounds__(kBlock)
std_filter_leaf_down(DevLevel lv, DevSeqs sq, GammaPacked<T> gv, const T* __restrict__ y,
                     const T* __restrict__ m0, const T* __restrict__ P0,
                     const T* __restrict__ carry, const int* __restrict__ flag, RowsSym<T, NX> fo,
                     double* __restrict__ partial, int* status) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int CREC = NX + NX * NX;
  const int b = lv.seq[c];
  const int64_t s0 = lv.first[c];
  const int cnt = lv.count[c];
  T m[NX], P[NX * NX];
  if (flag[c]) {
    load<T, NX>(carry + c * CREC, m);
    load<T, NX * NX>(carry + c * CREC + NX, P);
  } else {
    load<T, NX>(m0 + (int64_t)b * NX, m);
    load<T, NX * NX>(P0 + (int64_t)b * NX * NX, P);
    fo.store(sq.offsets[b] + b, m, P);   // k = 0
  }
  double acc = 0.0;
  bool ok = true;
  for (int j = 0; j < cnt; ++j) {
    const int64_t s = s0 + j;
    GammaStd<T, NX, NY> g;
    g.load_all(gv, s);
    T ys[NY];
    load<T, NY>(y + s * NY, ys);
    acc += (double)std_kf_step<T, NX, NY>(g, ys, m, P);
    fo.store(s + b + 1, m, P);
#pragma unroll
    for (int i = 0; i < NX; ++i) ok = ok && finite(m[i]);
  }
  if (partial) partial[c] = acc;
  if (!ok) flag_status(status, 8);
}

template <typename T, int NX, int NY>
__global__ void __launch_bounds__(kBlock)
std_smoother_leaf_up(DevLevel lv, DevSeqs sq, GammaPacked<T> gv, RowsSym<T, NX> fo,
                     T* __restrict__ items) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = SRec<NX>::size;
  const int b = lv.seq[c];
  const int64_t e0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t r0 = sq.offsets[b] + b;
  const int64_t nb = sq.offsets[b + 1] - sq.offsets[b];
  T agg[REC], el[REC], tmp[REC];
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t e = e0 + j;
    const int64_t k = e - r0;
    T m[NX], P[NX * NX];
    fo.load(e, m, P);
    T* dst = (j == cnt - 1) ? agg : el;
    if (k == nb) {
      std_smoother_element_last<T, NX>(m, P, dst);
    } else {
      GammaStd<T, NX, NY> g;
      g.load_transition(gv, sq.offsets[b] + k);
      std_smoother_element<T, NX, NY>(g, m, P, dst);
    }
    if (j != cnt - 1) {
      std_smoother_combine<T, NX>(el, agg, tmp);
      copy<T, REC>(tmp, agg);
    }
  }
  vstore<T, REC>(items + c * REC, agg);
}

template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
std_smoother_up(DevLevel lv, const T* __restrict__ in, T* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = SRec<NX>::size;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T agg[REC], el[REC], tmp[REC];
  vload<T, REC>(in + (i0 + cnt - 1) * REC, agg);
  for (int j = cnt - 2; j >= 0; --j) {
    vload<T, REC>(in + (i0 + j) * REC, el);
    std_smoother_combine<T, NX>(el, agg, tmp);
    copy<T, REC>(tmp, agg);
  }
  vstore<T, REC>(out + c * REC, agg);
}

// Carries (g, L) = the smoothing distribution after each item; flag 0: none.
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
std_smoother_down(DevLevel lv, const T* __restrict__ items, const T* __restrict__ cin,
                  const int* __restrict__ fin, T* __restrict__ cout, int* __restrict__ fout) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = SRec<NX>::size, CREC = NX + NX * NX;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  int flag = fin[c];
  T g[NX], L[NX * NX];
  load<T, NX>(cin + c * CREC, g);
  load<T, NX * NX>(cin + c * CREC + NX, L);
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t i = i0 + j;
    store<T, NX>(cout + i * CREC, g);
    store<T, NX * NX>(cout + i * CREC + NX, L);
    fout[i] = flag;
    if (j > 0) {
      T el[REC];
      vload<T, REC>(items + i * REC, el);
      if (flag) {
        std_smoother_apply<T, NX>(el, g, L);
      } else {
        copy<T, NX>(el + SRec<NX>::g, g);
        copy<T, NX * NX>(el + SRec<NX>::D, L);
        flag = 1;
      }
    }
  }
}

// Leaf down-sweep: covariance RTS steps from the chunk's carry; writes the
// new nominal into `nom` (previous nominal + deviation with add_nominal).
template <typename T, int NX, int NY>
__global__ void __launch_bounds__(kBlock)
std_smoother_leaf_down(DevLevel lv, DevSeqs sq, GammaPacked<T> gv, RowsSym<T, NX> fo,
                       const T* __restrict__ carry, const int* __restrict__ flag,
                       RowsSym<T, NX> nom, int* status, bool add_nominal) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = SRec<NX>::size, CREC = NX + NX * NX;
  const int b = lv.seq[c];
  const int64_t e0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t r0 = sq.offsets[b] + b;
  const int64_t nb = sq.offsets[b + 1] - sq.offsets[b];
  T g[NX], L[NX * NX];
  if (flag[c]) {
    load<T, NX>(carry + c * CREC, g);
    load<T, NX * NX>(carry + c * CREC + NX, L);
  }
  bool ok = true;
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t e = e0 + j;
    const int64_t k = e - r0;
    T m[NX], P[NX * NX];
    fo.load(e, m, P);
    if (k == nb) {
      copy<T, NX>(m, g);
      copy<T, NX * NX>(P, L);
    } else {
      GammaStd<T, NX, NY> gm;
      gm.load_transition(gv, sq.offsets[b] + k);
      T el[REC];
      std_smoother_element<T, NX, NY>(gm, m, P, el);
      std_smoother_apply<T, NX>(el, g, L);
    }
    T out[NX];
    if (add_nominal) {
      nom.load_mean(e, out);
#pragma unroll
      for (int i = 0; i < NX; ++i) out[i] += g[i];
    } else {
      copy<T, NX>(g, out);
    }
    nom.store(e, out, L);
#pragma unroll
    for (int i = 0; i < NX; ++i) ok = ok && finite(g[i]);
  }
  if (!ok) flag_status(status, 8);
}

// (m0, P0) of each sequence broadcast to its rows (initial nominal).
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
std_broadcast_prior(DevLevel lv, const T* __restrict__ m0, const T* __restrict__ P0,
                    RowsSym<T, NX> nom) {
  const int64_t ch = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (ch >= lv.n_chunks) return;
  const int b = lv.seq[ch];
  T m[NX], P[NX * NX];
  load<T, NX>(m0 + (int64_t)b * NX, m);
  load<T, NX * NX>(P0 + (int64_t)b * NX * NX, P);
  for (int j = 0; j < lv.count[ch]; ++j) nom.store(lv.first[ch] + j, m, P);
}

// One Alg. 3 run in the standard form (M iterations), fold-only plan.
template <typename T>
void std_ipls_enqueue(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s) {
  constexpr int NX = 5, NY = 2;
  const int64_t rows = Ls.n_items[0];
  const RowsSym<T, NX> nom{(T*)a.nrows}, fr{(T*)a.frows};
  const GammaPacked<T> gv{(T*)a.F};
  const T* P0 = (const T*)a.N0;   // the standard form takes prior covariances
  std_broadcast_prior<T, NX><<<grid_for(Ls.lv[0].n_chunks), kBlock, 0, s>>>(
      Ls.lv[0], (const T*)a.m0, P0, nom);
  for (int it = 0; it < a.M; ++it) {
    if (a.textbook && a.linearization == 0)
      std_slr_kernel<T, RowsSym<T, NX>, true><<<grid_for(Lf.lv[0].n_chunks * a.leaf), kBlock, 0, s>>>(
          Lf.lv[0], a.leaf, sq, (const CTParams<T>*)a.params, nom, a.linearization, a.centered,
          (const T*)a.y, (T*)a.F);
    else
      std_slr_kernel<T><<<grid_for(Lf.lv[0].n_chunks * a.leaf), kBlock, 0, s>>>(
          Lf.lv[0], a.leaf, sq, (const CTParams<T>*)a.params, nom, a.linearization, a.centered,
          (const T*)a.y, (T*)a.F);
    if (a.centered)
      center_prior_kernel<T, NX><<<(sq.B + 127) / 128, 128, 0, s>>>(sq, (const T*)a.m0, nom,
                                                                     (T*)a.dm0);
    const T* prior = (const T*)(a.centered ? a.dm0 : a.m0);
    // filter
    const int Lc = (int)Lf.lv.size();
    if (Lc > 1) {
      std_filter_leaf_up<T, NX, NY><<<grid_for(Lf.lv[0].n_chunks), kBlock, 0, s>>>(
          Lf.lv[0], sq, gv, (const T*)a.y, prior, P0, (T*)Wf.items[1]);
      for (int l = 1; l < Lc; ++l)
        std_filter_up<T, NX><<<grid_for(Lf.lv[l].n_chunks), kBlock, 0, s>>>(
            Lf.lv[l], (const T*)Wf.items[l], (T*)Wf.items[l + 1]);
    }
    cudaMemsetAsync(Wf.flag[Lc], 0, sizeof(int) * Lf.n_items[Lc], s);
    for (int l = Lc - 1; l >= 1; --l)
      std_filter_down<T, NX><<<grid_for(Lf.lv[l].n_chunks), kBlock, 0, s>>>(
          Lf.lv[l], (const T*)Wf.items[l], (const T*)Wf.carry[l + 1], Wf.flag[l + 1],
          (T*)Wf.carry[l], Wf.flag[l]);
    std_filter_leaf_down<T, NX, NY><<<grid_for(Lf.lv[0].n_chunks), kBlock, 0, s>>>(
        Lf.lv[0], sq, gv, (const T*)a.y, prior, P0, (const T*)Wf.carry[1], Wf.flag[1], fr, partial,
        status);
    // smoother
    const int Sc = (int)Ls.lv.size();
    if (Sc > 1) {
      std_smoother_leaf_up<T, NX, NY><<<grid_for(Ls.lv[0].n_chunks), kBlock, 0, s>>>(
          Ls.lv[0], sq, gv, fr, (T*)Ws.items[1]);
      for (int l = 1; l < Sc; ++l)
        std_smoother_up<T, NX><<<grid_for(Ls.lv[l].n_chunks), kBlock, 0, s>>>(
            Ls.lv[l], (const T*)Ws.items[l], (T*)Ws.items[l + 1]);
    }
    cudaMemsetAsync(Ws.flag[Sc], 0, sizeof(int) * Ls.n_items[Sc], s);
    for (int l = Sc - 1; l >= 1; --l)
      std_smoother_down<T, NX><<<grid_for(Ls.lv[l].n_chunks), kBlock, 0, s>>>(
          Ls.lv[l], (const T*)Ws.items[l], (const T*)Ws.carry[l + 1], Ws.flag[l + 1],
          (T*)Ws.carry[l], Ws.flag[l]);
    std_smoother_leaf_down<T, NX, NY><<<grid_for(Ls.lv[0].n_chunks), kBlock, 0, s>>>(
        Ls.lv[0], sq, gv, fr, (const T*)Ws.carry[1], Ws.flag[1], nom, status, a.centered != 0);
  }
  const RowsSplitSym<T, NX> user{(T*)a.ms, (T*)a.Ns};
  rows_copy_kernel<T, NX><<<grid_for(rows), kBlock, 0, s>>>(rows, nom, user);
  if (a.loglik) enqueue_loglik_reduce(sq, partial, a.loglik, status, s, nullptr);
}

}  // namespace sqsm
