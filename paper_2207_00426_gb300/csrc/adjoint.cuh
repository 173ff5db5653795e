// Reverse-mode adjoint of one iteration of Alg. 3 and of the pseudo
// log-likelihood, for the gradient of Sec. 5.2 (eq. implicity_function_theorem,
// Alg. 4) in its reverse (vector-Jacobian) form:
//   lambda <- (dKS/dn)^T lambda + (d l/dn)^T   (fixed point),
//   d l/d theta = (d l/d theta)^T + (dKS/d theta)^T lambda.
//
// One reverse pass, with cotangents lambda on the smoother output
// (m^s_k, N^s_k) and lbar on the log-likelihood, runs in covariance form
// (the square-root and covariance recursions are the same function):
//  1. N^s = chol(P^s): P^s-bar = sym(L^{-T} Phi(L^T L-bar) L^{-1}), Phi = lower
//     triangle with half diagonal (the factors are full rank here);
//  2. the RTS recursion read backwards is a forward linear recurrence
//     x_{k+1} = (G_k^T m, G_k^T P G_k) + direct_{k+1};
//  3. local VJP of each RTS step;
//  4. the filter recursion read backwards is a backward linear recurrence
//     x_{k-1} = (A_k^T m + s_k, A_k^T P A_k + sym(A_k^T m w_k^T) + S_k) with
//     A_k = (I - K_k H_k) F_{k-1}, w_k = F^T H^T S_k^{-1} v_k and sources from
//     lbar and from step 3;
//  5. local VJP of each Kalman step (-> linearised-model cotangents) and of
//     the cubature SLR (-> nominal-trajectory cotangents and theta).
// Both recurrences use one family of affine maps
//   x = (m, P) -> (B^T m + s, B^T P B + sym(B^T m r^T) + S),
// closed under composition, so they run as the same segmented
// reduce-then-scan as the forward filter and smoother (no thread waits on
// another).  The first map of the forward recurrence and the last of the
// backward one absorb their boundary value (B = 0), which makes a chunk that
// holds them independent of its carry.  Every iteration of Alg. 4 runs on
// the same linearisation, so what steps 2-5 need of it (the Kalman and RTS
// quantities, the fixed parts of both maps, the cubature regressions' G and
// residual columns) is computed once per evaluation into per-step tables
// (adj_tables.h); an iteration then does only the work that depends on
// lambda.
#pragma once

#include "adj_tables.h"
#include "ct_model.cuh"

namespace sqsm {

template <int NX> struct MapRec {
  static constexpr int B = 0, r = NX * NX, s = NX * NX + NX, S = NX * NX + 2 * NX,
                       size = 2 * NX * NX + 2 * NX;
};
template <int NX> struct XRec {
  static constexpr int m = 0, P = NX, size = NX + NX * NX;
};

// x_out = map(x_in)
template <typename T, int NX>
SQSM_DEV void map_apply(const T* mp, const T* xin, T* xout) {
  using R = MapRec<NX>;
  T bm[NX];
  mtv<T, NX, NX>(mp + R::B, xin, bm);             // B^T m
  T BP[NX * NX];
  mtm<T, NX, NX, NX>(mp + R::B, xin + NX, BP);    // B^T P
#pragma unroll
  for (int i = 0; i < NX; ++i) xout[i] = bm[i] + mp[R::s + i];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) acc += BP[i * NX + k] * mp[R::B + k * NX + j];
      xout[NX + i * NX + j] =
          acc + T(0.5) * (bm[i] * mp[R::r + j] + mp[R::r + i] * bm[j]) + mp[R::S + i * NX + j];
    }
}

// out = second o first (first applied first):
//   B = B_f B_s, r = B_s^T r_f + r_s, s = B_s^T s_f + s_s,
//   S = B_s^T S_f B_s + sym(B_s^T s_f r_s^T) + S_s.
template <typename T, int NX>
SQSM_DEV void map_compose(const T* f, const T* sc, T* out) {
  using R = MapRec<NX>;
  mm<T, NX, NX, NX>(f + R::B, sc + R::B, out + R::B);
  T t[NX];
  mtv<T, NX, NX>(sc + R::B, f + R::r, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) out[R::r + i] = t[i] + sc[R::r + i];
  T bs[NX];
  mtv<T, NX, NX>(sc + R::B, f + R::s, bs);
#pragma unroll
  for (int i = 0; i < NX; ++i) out[R::s + i] = bs[i] + sc[R::s + i];
  T BS[NX * NX];
  mtm<T, NX, NX, NX>(sc + R::B, f + R::S, BS);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) acc += BS[i * NX + k] * sc[R::B + k * NX + j];
      out[R::S + i * NX + j] =
          acc + T(0.5) * (bs[i] * sc[R::r + j] + sc[R::r + i] * bs[j]) + sc[R::S + i * NX + j];
    }
}

// Fold a boundary value into a map: the result ignores its input.
template <typename T, int NX>
SQSM_DEV void map_make_constant(T* mp, const T* x0) {
  using R = MapRec<NX>;
  T x1[XRec<NX>::size];
  map_apply<T, NX>(mp, x0, x1);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) {
    mp[R::B + i] = T(0);
    mp[R::S + i] = x1[NX + i];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    mp[R::r + i] = T(0);
    mp[R::s + i] = x1[i];
  }
}

// A A^T for lower A.
template <typename T, int N>
SQSM_DEV void gram_lower(const T* A, T* P) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (k <= i && k <= j) s += A[i * N + k] * A[j * N + k];
      P[i * N + j] = s;
    }
}

// Inverse of a lower-triangular N x N matrix (lower).
template <typename T, int N>
SQSM_DEV void inv_lower(const T* L, T* Li) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T col[N];
#pragma unroll
    for (int i = 0; i < N; ++i) col[i] = i == j ? T(1) : T(0);
    lsolve<T, N>(L, col);
#pragma unroll
    for (int i = 0; i < N; ++i) Li[i * N + j] = col[i];
  }
}

// (F N) with N lower (NX x NX), then N^- = Tria([F N, SQ]).
template <typename T, int NX>
SQSM_DEV void predict_factor(const T* F, const T* N, const T* SQ, T* Nm) {
  T P[NX * 2 * NX];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < NX; ++k) s += F[i * NX + k] * N[k * NX + j];
      P[i * 2 * NX + j] = s;
      P[i * 2 * NX + NX + j] = SQ[i * NX + j];
    }
  tria<T, NX, 2 * NX>(P);
  take_lower<T, NX, 2 * NX>(P, Nm);
}

// The Kalman-step quantities the VJP reads, loaded from a KfTab record.
template <typename T, int NX, int NY>
struct KfQ {
  T mp[NX], Pp[NX * NX], W[NY * NY], U[NX * NY], K[NX * NY], v[NY], Pprev[NX * NX];
  SQSM_DEV void load(const T* t) {
    using KT = KfTab<NX, NY>;
#pragma unroll
    for (int i = 0; i < NX; ++i) mp[i] = t[KT::mp + i];
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) {
      Pp[i] = t[KT::Pp + i];
      Pprev[i] = t[KT::Pprev + i];
    }
#pragma unroll
    for (int i = 0; i < NY * NY; ++i) W[i] = t[KT::W + i];
#pragma unroll
    for (int i = 0; i < NX * NY; ++i) {
      U[i] = t[KT::U + i];
      K[i] = t[KT::K + i];
    }
#pragma unroll
    for (int i = 0; i < NY; ++i) v[i] = t[KT::v + i];
  }
};

// Both tables of one step from its linearised model g, observation y, the
// filter output (mf, Nf) at row e and the smoother output (msn, Nsn) at row
// e + 1.  The prediction (m^-, N^-) is shared by the Kalman and RTS steps.
template <typename T, int NX, int NY>
SQSM_DEV void adj_step_tables(const Gamma<T, NX, NY>& g, const T* y, const T* mf, const T* Nf,
                              const T* msn, const T* Nsn, T* kt, T* rt) {
  using KT = KfTab<NX, NY>;
  using RT = RtsTab<NX>;
  T mp[NX];
  mv<T, NX, NX>(g.F, mf, mp);
#pragma unroll
  for (int i = 0; i < NX; ++i) mp[i] += g.c[i];
  T Nm[NX * NX], Pp[NX * NX], Pf[NX * NX];
  predict_factor<T, NX>(g.F, Nf, g.SQ, Nm);
  gram_lower<T, NX>(Nm, Pp);
  gram_lower<T, NX>(Nf, Pf);
  // Kalman step
  T U[NX * NY], S[NY * NY], R[NY * NY];
  mmt<T, NX, NX, NY>(Pp, g.H, U);                  // P^- H^T
  mm<T, NY, NX, NY>(g.H, U, S);                    // H P^- H^T
  gram_lower<T, NY>(g.SR, R);
#pragma unroll
  for (int i = 0; i < NY * NY; ++i) S[i] += R[i];
  chol_inplace<T, NY>(S);                          // W = S^{-1} from its factor
  T Si[NY * NY], W[NY * NY], K[NX * NY], v[NY];
  inv_lower<T, NY>(S, Si);
  mtm<T, NY, NY, NY>(Si, Si, W);
  mm<T, NX, NY, NY>(U, W, K);
#pragma unroll
  for (int i = 0; i < NY; ++i) {
    T a = y[i] - g.d[i];
#pragma unroll
    for (int k = 0; k < NX; ++k) a -= g.H[i * NX + k] * mp[k];
    v[i] = a;
  }
  // fixed parts of the backward map
  T KH[NX * NX];
  mm<T, NX, NY, NX>(K, g.H, KH);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) KH[i] = ((i / NX) == (i % NX) ? T(1) : T(0)) - KH[i];
  mm<T, NX, NX, NX>(KH, g.F, kt + KT::A);
  T HF[NY * NX], al[NY], WHF[NY * NX];
  mm<T, NY, NX, NX>(g.H, g.F, HF);
  mv<T, NY, NY>(W, v, al);
  mtv<T, NY, NX>(HF, al, kt + KT::w);
  mm<T, NY, NY, NX>(W, HF, WHF);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T a = T(0);
#pragma unroll
      for (int k = 0; k < NY; ++k) a += HF[k * NX + i] * WHF[k * NX + j];
      kt[KT::C + i * NX + j] = a - kt[KT::w + i] * kt[KT::w + j];
    }
#pragma unroll
  for (int i = KT::C + NX * NX; i < KT::head; ++i) kt[i] = T(0);
#pragma unroll
  for (int i = 0; i < NY * NY; ++i) kt[KT::W + i] = W[i];
#pragma unroll
  for (int i = 0; i < NY; ++i) kt[KT::v + i] = v[i];
#pragma unroll
  for (int i = 0; i < NX * NY; ++i) {
    kt[KT::K + i] = K[i];
    kt[KT::U + i] = U[i];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) kt[KT::mp + i] = mp[i];
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) {
    kt[KT::Pp + i] = Pp[i];
    kt[KT::Pprev + i] = Pf[i];
  }
#pragma unroll
  for (int i = KT::Pprev + NX * NX; i < KT::size; ++i) kt[i] = T(0);
  // RTS step
  T Li[NX * NX], PFt[NX * NX];
  inv_lower<T, NX>(Nm, Li);
  mtm<T, NX, NX, NX>(Li, Li, rt + RT::Wp);
  mmt<T, NX, NX, NX>(Pf, g.F, PFt);
  mm<T, NX, NX, NX>(PFt, rt + RT::Wp, rt + RT::G);
#pragma unroll
  for (int i = RT::G + NX * NX; i < RT::head; ++i) rt[i] = T(0);
  T Ps1[NX * NX];
  gram_lower<T, NX>(Nsn, Ps1);
#pragma unroll
  for (int i = 0; i < NX; ++i) rt[RT::dm + i] = msn[i] - mp[i];
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) {
    rt[RT::Pf + i] = Pf[i];
    rt[RT::D + i] = Ps1[i] - Pp[i];
  }
#pragma unroll
  for (int i = RT::D + NX * NX; i < RT::size; ++i) rt[i] = T(0);
}

// Linearised-model cotangent record of one step: F | c | Lambda | H | d | Omega.
template <int NX, int NY> struct GRec {
  static constexpr int F = 0, c = NX * NX, L = NX * NX + NX, H = 2 * NX * NX + NX,
                       d = 2 * NX * NX + NX + NY * NX, O = 2 * NX * NX + NX + NY * NX + NY,
                       size = 2 * NX * NX + NX + NY * NX + NY + NY * NY;
};

// ---------------------------------------------------------------------------
// Step 1: direct cotangents of the smoother output of one state row from
// its factor L = N^s and the cotangent lam = (m-bar, lower N-bar).
// ---------------------------------------------------------------------------
template <typename T, int NX>
SQSM_DEV void direct_row(const T* L, const T* lam, T* __restrict__ o) {
  T Lb[NX * NX];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) Lb[i * NX + j] = j <= i ? lam[NX + i * NX + j] : T(0);
  T M[NX * NX];
  mtm<T, NX, NX, NX>(L, Lb, M);                    // L^T Lbar
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) M[i * NX + j] = j < i ? M[i * NX + j] : (j == i ? T(0.5) * M[i * NX + j] : T(0));
  T Li[NX * NX];
  inv_lower<T, NX>(L, Li);
  T A[NX * NX], P[NX * NX];
  mtm<T, NX, NX, NX>(Li, M, A);                    // L^{-T} Phi
  mm<T, NX, NX, NX>(A, Li, P);                     // ... L^{-1}
#pragma unroll
  for (int i = 0; i < NX; ++i) o[i] = lam[i];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) o[NX + i * NX + j] = T(0.5) * (P[i * NX + j] + P[j * NX + i]);
}

// ---------------------------------------------------------------------------
// Maps of one time step from its tables (state rows e = s + b (k - 1) and
// e + 1 (k) of step s in sequence b).
// ---------------------------------------------------------------------------

// Forward-recurrence map of step s: x(row e) -> x(row e + 1),
// B = G_{k-1}, r = 0, s = direct_m(e+1), S = direct_P(e+1).
template <typename T, int NX>
SQSM_DEV void smoother_adj_map(const T* G, const T* dnext, T* mp) {
  using R = MapRec<NX>;
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) {
    mp[R::B + i] = G[i];
    mp[R::S + i] = dnext[NX + i];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    mp[R::r + i] = T(0);
    mp[R::s + i] = dnext[i];
  }
}

// Backward-recurrence map of Kalman step k: x(row e + 1) -> x(row e),
// B = A, r = w, s = lbar w + dfilt_m(e), S = -lbar/2 C + dfilt_P(e), from
// the head of the step's KfTab record.
template <typename T, int NX, int NY>
SQSM_DEV void filter_adj_map(const T* kt, T lbar, const T* dprev, T* mp) {
  using R = MapRec<NX>;
  using KT = KfTab<NX, NY>;
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) {
    mp[R::B + i] = kt[KT::A + i];
    mp[R::S + i] = T(-0.5) * lbar * kt[KT::C + i] + dprev[NX + i];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    mp[R::r + i] = kt[KT::w + i];
    mp[R::s + i] = lbar * kt[KT::w + i] + dprev[i];
  }
}

// ---------------------------------------------------------------------------
// Local VJPs
// ---------------------------------------------------------------------------

// RTS step at row e (k < n) with total cotangent x = (mt, Pt), its RtsTab
// record rt, transition matrix F and filter mean mf of row e: writes the
// direct filter cotangents of row e and the smoother part of the
// linearised-model cotangents of step t (F, c, Lambda).
template <typename T, int NX, int NY>
SQSM_DEV void rts_vjp(const T* rt, const T* F, const T* mf, const T* x, T* dfilt, T* gbar) {
  using GR = GRec<NX, NY>;
  using RT = RtsTab<NX>;
  const T* mt = x;
  const T* Pt = x + NX;
  const T* G = rt + RT::G;
  const T* Wp = rt + RT::Wp;
  const T* Pf = rt + RT::Pf;
  const T* dm_ = rt + RT::dm;
  const T* D = rt + RT::D;
  // Gb = mt dm^T + 2 Pt G D
  T PtG[NX * NX], Gb[NX * NX], tmp[NX * NX];
  mm<T, NX, NX, NX>(Pt, G, PtG);
  mm<T, NX, NX, NX>(PtG, D, tmp);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) Gb[i * NX + j] = mt[i] * dm_[j] + T(2) * tmp[i * NX + j];
  // dmp = -G^T mt ; dPp = -G^T Pt G - sym(G^T Gb Wp)
  T dmp[NX];
  mtv<T, NX, NX>(G, mt, dmp);
#pragma unroll
  for (int i = 0; i < NX; ++i) dmp[i] = -dmp[i];
  T dPp[NX * NX], GtPtG[NX * NX], GtGb[NX * NX], GtGbW[NX * NX];
  mtm<T, NX, NX, NX>(G, PtG, GtPtG);
  mtm<T, NX, NX, NX>(G, Gb, GtGb);
  mm<T, NX, NX, NX>(GtGb, Wp, GtGbW);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j)
      dPp[i * NX + j] = -GtPtG[i * NX + j] - T(0.5) * (GtGbW[i * NX + j] + GtGbW[j * NX + i]);
  // direct filter cotangents: dmf = mt + F^T dmp ; dPf = Pt + sym(Gb Wp F) + F^T dPp F
  T Ftd[NX];
  mtv<T, NX, NX>(F, dmp, Ftd);
  T GbW[NX * NX], GbWF[NX * NX], FtdPp[NX * NX], FtdPpF[NX * NX];
  mm<T, NX, NX, NX>(Gb, Wp, GbW);
  mm<T, NX, NX, NX>(GbW, F, GbWF);
  mtm<T, NX, NX, NX>(F, dPp, FtdPp);
  mm<T, NX, NX, NX>(FtdPp, F, FtdPpF);
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    dfilt[i] = mt[i] + Ftd[i];
#pragma unroll
    for (int j = 0; j < NX; ++j)
      dfilt[NX + i * NX + j] = Pt[i * NX + j] + T(0.5) * (GbWF[i * NX + j] + GbWF[j * NX + i]) +
                               FtdPpF[i * NX + j];
  }
  // gF = Wp Gb^T Pf + dmp mf^T + 2 dPp F Pf ; gc = dmp ; gL = dPp
  T WGbt[NX * NX], A1[NX * NX], FPf[NX * NX], A2[NX * NX];
  mmt<T, NX, NX, NX>(Wp, Gb, WGbt);
  mm<T, NX, NX, NX>(WGbt, Pf, A1);
  mm<T, NX, NX, NX>(F, Pf, FPf);
  mm<T, NX, NX, NX>(dPp, FPf, A2);
#pragma unroll
  for (int i = 0; i < NX; ++i) {
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      gbar[GR::F + i * NX + j] = A1[i * NX + j] + dmp[i] * mf[j] + T(2) * A2[i * NX + j];
      gbar[GR::L + i * NX + j] = dPp[i * NX + j];
    }
    gbar[GR::c + i] = dmp[i];
  }
}

// Kalman step k (t = k - 1) with total cotangent x = (ym, yP) of its output
// and lbar of l_k: adds the filter part of the linearised-model cotangents
// of step t to gbar (F, c, Lambda: +=; H, d, Omega: =).
template <typename T, int NX, int NY>
SQSM_DEV void kf_vjp(const KfQ<T, NX, NY>& q, const Gamma<T, NX, NY>& g, const T* mprev, T lbar,
                     const T* x, T* gbar) {
  using GR = GRec<NX, NY>;
  const T* ym = x;
  const T* yP = x + NX;
  T al[NY];
  mv<T, NY, NY>(q.W, q.v, al);
  T vb[NY], Sb[NY * NY];
#pragma unroll
  for (int i = 0; i < NY; ++i) vb[i] = -lbar * al[i];
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NY; ++j) Sb[i * NY + j] = T(-0.5) * lbar * (q.W[i * NY + j] - al[i] * al[j]);
  // m' = m^- + K v
  T mpb[NX];
#pragma unroll
  for (int i = 0; i < NX; ++i) mpb[i] = ym[i];
  T Ktym[NY];
  mtv<T, NX, NY>(q.K, ym, Ktym);
#pragma unroll
  for (int i = 0; i < NY; ++i) vb[i] += Ktym[i];
  // Kb = ym v^T ; Ub = -2 yP K + Kb W ; Wb = -U^T yP U + U^T Kb
  T Ub[NX * NY], yPK[NX * NY];
  mm<T, NX, NX, NY>(yP, q.K, yPK);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      T kw = T(0);
#pragma unroll
      for (int k = 0; k < NY; ++k) kw += q.v[k] * q.W[k * NY + j];
      Ub[i * NY + j] = T(-2) * yPK[i * NY + j] + ym[i] * kw;
    }
  T yPU[NX * NY], Wb[NY * NY];
  mm<T, NX, NX, NY>(yP, q.U, yPU);
  T Utym[NY];
  mtv<T, NX, NY>(q.U, ym, Utym);
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NY; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) s += q.U[k * NY + i] * yPU[k * NY + j];
      Wb[i * NY + j] = -s + Utym[i] * q.v[j];
    }
  // Sb -= sym(W Wb W)
  T WWb[NY * NY], WWbW[NY * NY];
  mm<T, NY, NY, NY>(q.W, Wb, WWb);
  mm<T, NY, NY, NY>(WWb, q.W, WWbW);
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NY; ++j) Sb[i * NY + j] -= T(0.5) * (WWbW[i * NY + j] + WWbW[j * NY + i]);
  // v = y - H m^- - d
  T gH[NY * NX];
#pragma unroll
  for (int i = 0; i < NY; ++i) {
    gbar[GR::d + i] = -vb[i];
#pragma unroll
    for (int j = 0; j < NX; ++j) gH[i * NX + j] = -vb[i] * q.mp[j];
  }
  T Htvb[NX];
  mtv<T, NY, NX>(g.H, vb, Htvb);
#pragma unroll
  for (int i = 0; i < NX; ++i) mpb[i] -= Htvb[i];
  // U = P^- H^T: Ppb += sym(Ub H); gH += Ub^T P^-
  // S = H P^- H^T + Omega: Ppb += H^T Sb H; gH += 2 Sb H P^-; gO = Sb
  T Ppb[NX * NX], UbH[NX * NX];
  mm<T, NX, NY, NX>(Ub, g.H, UbH);
  T SbH[NY * NX], HtSbH[NX * NX];
  mm<T, NY, NY, NX>(Sb, g.H, SbH);
  mtm<T, NX, NY, NX>(g.H, SbH, HtSbH);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j)
      Ppb[i * NX + j] = yP[i * NX + j] + T(0.5) * (UbH[i * NX + j] + UbH[j * NX + i]) + HtSbH[i * NX + j];
  T UbtPp[NY * NX], SbHPp[NY * NX];
  mtm<T, NY, NX, NX>(Ub, q.Pp, UbtPp);
  mm<T, NY, NX, NX>(SbH, q.Pp, SbHPp);
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) gbar[GR::H + i * NX + j] = gH[i * NX + j] + UbtPp[i * NX + j] + T(2) * SbHPp[i * NX + j];
#pragma unroll
  for (int i = 0; i < NY * NY; ++i) gbar[GR::O + i] = Sb[i];
  // m^- = F m + c ; P^- = F P F^T + Lambda
  T FPprev[NX * NX], PpbFP[NX * NX];
  mm<T, NX, NX, NX>(g.F, q.Pprev, FPprev);
  mm<T, NX, NX, NX>(Ppb, FPprev, PpbFP);
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    gbar[GR::c + i] += mpb[i];
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      gbar[GR::F + i * NX + j] += mpb[i] * mprev[j] + T(2) * PpbFP[i * NX + j];
      gbar[GR::L + i * NX + j] += Ppb[i * NX + j];
    }
  }
}

// VJP of the cubature regression of one function about (m, N) (Sec. 4.3 in
// the form of the forward kernel): given cotangents Gb of the regression
// matrix, ob of the offset (absolute form z_bar - G m) and Lb of the noise
// covariance, accumulate into mb, Nb.  JAC(x, J) writes the Jacobian of
// the regressed function at x; G, s (residual columns) are recomputed.
template <typename T, int NO, typename JAC>
SQSM_DEV void cubature_vjp(const T* m, const T* N, const T* G, const T* sres, const T* Gb,
                           const T* ob, const T* Lb, JAC jac, T* mb, T* Nb) {
  constexpr int NX = 5;
  const T sq = sq_sqrt(T(NX));
  // m-part of the offset: off = z_bar - G m
  T Fp[NO * NX];
#pragma unroll
  for (int r = 0; r < NO; ++r)
#pragma unroll
    for (int j = 0; j < NX; ++j) Fp[r * NX + j] = Gb[r * NX + j] - ob[r] * m[j];
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    T s = T(0);
#pragma unroll
    for (int r = 0; r < NO; ++r) s += G[r * NX + j] * ob[r];
    mb[j] -= s;
  }
  // G = D N^{-1}: Db = Fp N^{-T}; Nb -= G^T Fp N^{-T}
  T Db[NO * NX];
#pragma unroll
  for (int i = 0; i < NO * NX; ++i) Db[i] = Fp[i];
  rsolve_t<T, NO, NX>(Db, N);
  T GtDb[NX * NX];
  mtm<T, NX, NO, NX>(G, Db, GtDb);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) Nb[i] -= GtDb[i];
  // residual columns: sb_i = (2/NX) Lb s_i ; common = (ob - sum sb_i) / (2 NX)
  T sb[NO * NX], sum[NO];
#pragma unroll
  for (int r = 0; r < NO; ++r) sum[r] = T(0);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < NO; ++k) s += Lb[r * NO + k] * sres[k * NX + i];
      sb[r * NX + i] = T(2) / T(NX) * s;
      sum[r] += sb[r * NX + i];
    }
  T common[NO];
#pragma unroll
  for (int r = 0; r < NO; ++r) common[r] = (ob[r] - sum[r]) / T(2 * NX);
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    T X[NX], J[NO * NX], zp[NO], zn[NO], xp[NX], xn[NX];
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      zp[r] = Db[r * NX + i] / (T(2) * sq) + T(0.5) * sb[r * NX + i] + common[r];
      zn[r] = -Db[r * NX + i] / (T(2) * sq) + T(0.5) * sb[r * NX + i] + common[r];
    }
#pragma unroll
    for (int j = 0; j < NX; ++j) X[j] = m[j] + sq * N[j * NX + i];
    jac(X, J);
    mtv<T, NO, NX>(J, zp, xp);
#pragma unroll
    for (int j = 0; j < NX; ++j) X[j] = m[j] - sq * N[j * NX + i];
    jac(X, J);
    mtv<T, NO, NX>(J, zn, xn);
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      mb[j] += xp[j] + xn[j];
      Nb[j * NX + i] += sq * (xp[j] - xn[j]);
    }
  }
}

// VJP of a sigma-point regression with points X_p = m + N xi_p and weights
// w_p (sum w = 1, sum w xi = 0, sum w xi xi^T = I): the unscented rule
// (RULE 1: centre weight 1/6, pairs +-sqrt(6) e_i of weight 1/12) or the
// tensor-product three-point Gauss-Hermite rule (RULE 2: 243 points).  With
// the forward quantities D = sum w Dl_p xi_p^T (G = D N^{-1}, + I with
// ADD_I), residuals r_p = Dl_p - Dl_bar - D xi_p (Dl_p the point differences
// of DG, as in the forward kernel) and Lambda = Sc Sc^T + sum w r_p r_p^T,
// the cotangent of Z_p = f(X_p) is
//   Zb_p = w_p (Db xi_p + 2 Lb r_p + ob),  Db = (Gb - ob m^T) N^{-T},
// (the G and z_bar dependence of Lambda has zero derivative: sum w r = 0
// and sum w r xi^T = 0 at the regression), and it reaches (m, N) through
// X_p (J = JAC at X_p) and through G = D N^{-1} (Nb -= G^T Db) and the
// offset z_bar - G m (mb -= G^T ob).  Two passes over the points: the first
// rebuilds D and Dl_bar, the second the residuals and cotangents.
template <typename T, int NO, int RULE, bool ADD_I, typename DG, typename JAC>
SQSM_DEV void sigma_vjp(const T* m, const T* N, DG dg, JAC jac, const T* Gb, const T* ob,
                        const T* Lb, T* mb, T* Nb) {
  constexpr int NX = 5;
  constexpr int NP = RULE == 1 ? 2 * NX + 1 : 243;
  // point p: unit point xi and weight
  auto point = [&](int p, T* xi) -> T {
    if constexpr (RULE == 1) {
#pragma unroll
      for (int k = 0; k < NX; ++k) xi[k] = T(0);
      if (p == 0) return T(1.0 / 6.0);
      const int i = (p - 1) % NX;
      xi[i] = (p <= NX ? T(1) : T(-1)) * sq_sqrt(T(6));
      return T(1.0 / 12.0);
    } else {
      const T r3 = sq_sqrt(T(3));
      T w = T(1);
      int q = p;
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        const int dgt = q % 3;
        q /= 3;
        xi[k] = dgt == 0 ? T(0) : (dgt == 1 ? r3 : -r3);
        w *= dgt == 0 ? T(2.0 / 3.0) : T(1.0 / 6.0);
      }
      return w;
    }
  };
  auto delta = [&](const T* xi, T* dl) {
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      T a = T(0);
#pragma unroll
      for (int k = 0; k <= r; ++k) a += N[r * NX + k] * xi[k];
      dl[r] = a;
    }
  };
  T D[NO * NX], dbar[NO];
#pragma unroll
  for (int i = 0; i < NO * NX; ++i) D[i] = T(0);
#pragma unroll
  for (int r = 0; r < NO; ++r) dbar[r] = T(0);
#pragma unroll 1
  for (int p = 0; p < NP; ++p) {
    T xi[NX], dl[NX], z[NO];
    const T w = point(p, xi);
    delta(xi, dl);
    dg(m, dl, z);
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      dbar[r] += w * z[r];
#pragma unroll
      for (int k = 0; k < NX; ++k) D[r * NX + k] += w * z[r] * xi[k];
    }
  }
  T G[NO * NX];
#pragma unroll
  for (int i = 0; i < NO * NX; ++i) G[i] = D[i];
  rsolve<T, NO, NX>(G, N);
  if constexpr (ADD_I) {
#pragma unroll
    for (int r = 0; r < NO; ++r) G[r * NX + r] += T(1);
  }
  // offset and regression-matrix parts
  T Db[NO * NX];
#pragma unroll
  for (int r = 0; r < NO; ++r)
#pragma unroll
    for (int j = 0; j < NX; ++j) Db[r * NX + j] = Gb[r * NX + j] - ob[r] * m[j];
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    T a = T(0);
#pragma unroll
    for (int r = 0; r < NO; ++r) a += G[r * NX + j] * ob[r];
    mb[j] -= a;
  }
  rsolve_t<T, NO, NX>(Db, N);
  T GtDb[NX * NX];
  mtm<T, NX, NO, NX>(G, Db, GtDb);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) Nb[i] -= GtDb[i];
#pragma unroll 1
  for (int p = 0; p < NP; ++p) {
    T xi[NX], dl[NX], z[NO], zb[NO], X[NX], J[NO * NX], xb[NX];
    const T w = point(p, xi);
    delta(xi, dl);
    dg(m, dl, z);
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      T res = z[r] - dbar[r];
#pragma unroll
      for (int k = 0; k < NX; ++k) res -= D[r * NX + k] * xi[k];
      z[r] = res;
    }
#pragma unroll
    for (int r = 0; r < NO; ++r) {
      T a = ob[r];
#pragma unroll
      for (int k = 0; k < NX; ++k) a += Db[r * NX + k] * xi[k];
#pragma unroll
      for (int k = 0; k < NO; ++k) a += T(2) * Lb[r * NO + k] * z[k];
      zb[r] = w * a;
    }
#pragma unroll
    for (int j = 0; j < NX; ++j) X[j] = m[j] + dl[j];
    jac(X, J);
    mtv<T, NO, NX>(J, zb, xb);
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      mb[j] += xb[j];
#pragma unroll
      for (int k = 0; k < NX; ++k) Nb[j * NX + k] += xb[j] * xi[k];
    }
  }
}

// VJP of the Taylor linearisation (Sec. 4.2) of one function about m:
// G = J(m), offset z(m) - J(m) m (absolute form), noise factor independent
// of m.  The offset's z(m) and -J m parts cancel in m, leaving
//   mb += sum_ij (Gb - ob m^T)_ij dJ_ij/dm  (HJVP: the second derivatives
// of the function contracted with a Jacobian cotangent).
template <typename T, int NO, typename HJVP>
SQSM_DEV void taylor_vjp(const T* m, const T* Gb, const T* ob, HJVP hjvp, T* mb) {
  constexpr int NX = 5;
  T Jb[NO * NX];
#pragma unroll
  for (int r = 0; r < NO; ++r)
#pragma unroll
    for (int j = 0; j < NX; ++j) Jb[r * NX + j] = Gb[r * NX + j] - ob[r] * m[j];
  hjvp(m, Jb, mb);
}

// Forward quantities of the cubature regression needed by its VJP: G and
// the residual columns s_i, from the same difference formulas as the
// forward kernel.
template <typename T, int NO, bool ADD_I, typename DG>
SQSM_DEV void cubature_fwd(const T* m, const T* N, DG dg, T* G, T* sres) {
  constexpr int NX = 5;
  const T sq = sq_sqrt(T(NX));
  T Hs[NO * NX], dsum[NO];
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
      G[r * NX + i] = (zp[r] - zn[r]) / (T(2) * sq);
      Hs[r * NX + i] = T(0.5) * (zp[r] + zn[r]);
      dsum[r] += zp[r] + zn[r];
    }
  }
  rsolve<T, NO, NX>(G, N);
  if constexpr (ADD_I) {
#pragma unroll
    for (int r = 0; r < NO; ++r) G[r * NX + r] += T(1);
  }
#pragma unroll
  for (int r = 0; r < NO; ++r)
#pragma unroll
    for (int i = 0; i < NX; ++i) sres[r * NX + i] = Hs[r * NX + i] - dsum[r] / T(2 * NX);
}

}  // namespace sqsm
