// Scan elements and associative operators of the square-root parallel
// Kalman filter and RTS smoother (Sec. 3: Lemmas 1-4, Tables 1-5), one thread
// per element or combine, operands in registers.
//
// Filter element record (Pi^f_k of eq. pi-f), NX x NX matrices row-major:
//   A | b | U (lower) | eta | Z (lower, square)    -> FREC = 3 NX^2 + 2 NX
// Smoother element record (Pi^s_k = {E, g, D}):
//   E | g | D (lower)                               -> SREC = 2 NX^2 + NX
#pragma once

#include "linalg.cuh"

namespace sqsm {

// Per-step view of a linear(ised) model.  Row t holds the transition
// (F_t, c_t, S_Lambda_t) of x_{t+1} = F_t x_t + c_t + q_t and the
// observation (H_{t+1}, d_{t+1}, S_Omega_{t+1}) of y_{t+1}
// (eq. linear-model); strides are in elements, 0 = time-invariant.
template <typename T>
struct GammaView {
  const T *F, *c, *SQ, *H, *d, *SR;
  int64_t sF, sc, sSQ, sH, sd, sSR;
};

// Packed per-step record of the linearised model, the layout the iterated
// smoother keeps internally: 16-byte aligned, transition part first so that
// the smoother reads only that part,
//   F (NX x NX) | c | S_Lambda (lower, row-packed) | pad |
//   H (NY x NX) | d | S_Omega (lower, row-packed) | pad.
template <int NX, int NY> struct PRec {
  static constexpr int F = 0, c = NX * NX, SQ = NX * NX + NX;
  static constexpr int H = (SQ + NX * (NX + 1) / 2 + 3) / 4 * 4;   // also the transition size
  static constexpr int d = H + NY * NX, SR = d + NY;
  static constexpr int size = (SR + NY * (NY + 1) / 2 + 3) / 4 * 4;
};

template <typename T>
struct GammaPacked {
  T* rec;   // PRec records, one per step
};

// State rows (m_k, N_k) of a trajectory, rows k = 0..n of each sequence.
// RowsSplit is the API layout: m as NX values and N as a full NX x NX lower
// factor (zeros above the diagonal) per row; a null array is not written.
// RowsPacked is the iterated smoother's own layout: one 16-byte-aligned
// record per row, m | N (lower, row-packed) | pad.
template <int NX> struct XRow {
  static constexpr int size = (NX + NX * (NX + 1) / 2 + 3) / 4 * 4;
  static constexpr int mvec = (NX + 3) / 4 * 4;   // leading words that hold m
};

// E_k of Table 4 for one state row, 16-byte aligned (the 25 values padded):
// written by a full smoother pass, read by the mean-only refinement passes.
template <int NX> struct ETab {
  static constexpr int size = (NX * NX + 3) / 4 * 4;
};

template <typename T, int NX>
struct RowsSplit {
  T* m;
  T* N;
  SQSM_DEV void load(int64_t e, T* mo, T* No) const {
    sqsm::load<T, NX>(m + e * NX, mo);
    load_lower<T, NX>(N + e * NX * NX, No);
  }
  SQSM_DEV void load_mean(int64_t e, T* mo) const { sqsm::load<T, NX>(m + e * NX, mo); }
  SQSM_DEV void store(int64_t e, const T* mi, const T* Ni) const {
    if (m) sqsm::store<T, NX>(m + e * NX, mi);
    if (N) store_lower<T, NX>(N + e * NX * NX, Ni);
  }
};

template <typename T, int NX>
struct RowsPacked {
  T* rec;
  SQSM_DEV void load(int64_t e, T* mo, T* No) const {
    using R = XRow<NX>;
    T v[R::size];
    vload<T, R::size>(rec + e * R::size, v);
#pragma unroll
    for (int i = 0; i < NX; ++i) mo[i] = v[i];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j < NX; ++j) No[i * NX + j] = j <= i ? v[NX + i * (i + 1) / 2 + j] : T(0);
  }
  SQSM_DEV void load_mean(int64_t e, T* mo) const {
    using R = XRow<NX>;
    T v[R::mvec];
    vload<T, R::mvec>(rec + e * R::size, v);
#pragma unroll
    for (int i = 0; i < NX; ++i) mo[i] = v[i];
  }
  SQSM_DEV void store(int64_t e, const T* mi, const T* Ni) const {
    using R = XRow<NX>;
    T v[R::size];
#pragma unroll
    for (int i = 0; i < R::size; ++i) v[i] = T(0);
#pragma unroll
    for (int i = 0; i < NX; ++i) v[i] = mi[i];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) v[NX + i * (i + 1) / 2 + j] = Ni[i * NX + j];
    vstore<T, R::size>(rec + e * R::size, v);
  }
};

template <typename T, int NX, int NY>
struct Gamma {
  T F[NX * NX], c[NX], SQ[NX * NX], H[NY * NX], d[NY], SR[NY * NY];

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
      for (int j = 0; j < NX; ++j) SQ[i * NX + j] = j <= i ? v[P::SQ + i * (i + 1) / 2 + j] : T(0);
  }
  SQSM_DEV void load_observation(const GammaPacked<T>& g, int64_t t) {
    using P = PRec<NX, NY>;
    T v[P::size - P::H];
    vload<T, P::size - P::H>(g.rec + t * P::size + P::H, v);
#pragma unroll
    for (int i = 0; i < NY * NX; ++i) H[i] = v[i];
#pragma unroll
    for (int i = 0; i < NY; ++i) d[i] = v[P::d - P::H + i];
#pragma unroll
    for (int i = 0; i < NY; ++i)
#pragma unroll
      for (int j = 0; j < NY; ++j) SR[i * NY + j] = j <= i ? v[P::SR - P::H + i * (i + 1) / 2 + j] : T(0);
  }
  SQSM_DEV void load_all(const GammaPacked<T>& g, int64_t t) {
    load_transition(g, t);
    load_observation(g, t);
  }
  // Write this step's record (lower triangles of S_Lambda, S_Omega).
  SQSM_DEV void store_transition(const GammaPacked<T>& g, int64_t t) const {
    using P = PRec<NX, NY>;
    T v[P::H];
#pragma unroll
    for (int i = 0; i < P::H; ++i) v[i] = T(0);
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) v[P::F + i] = F[i];
#pragma unroll
    for (int i = 0; i < NX; ++i) v[P::c + i] = c[i];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) v[P::SQ + i * (i + 1) / 2 + j] = SQ[i * NX + j];
    vstore<T, P::H>(g.rec + t * P::size, v);
  }
  SQSM_DEV void store_observation(const GammaPacked<T>& g, int64_t t) const {
    using P = PRec<NX, NY>;
    T v[P::size - P::H];
#pragma unroll
    for (int i = 0; i < P::size - P::H; ++i) v[i] = T(0);
#pragma unroll
    for (int i = 0; i < NY * NX; ++i) v[i] = H[i];
#pragma unroll
    for (int i = 0; i < NY; ++i) v[P::d - P::H + i] = d[i];
#pragma unroll
    for (int i = 0; i < NY; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) v[P::SR - P::H + i * (i + 1) / 2 + j] = SR[i * NY + j];
    vstore<T, P::size - P::H>(g.rec + t * P::size + P::H, v);
  }

  SQSM_DEV void load_transition(const GammaView<T>& g, int64_t t) {
    load<T, NX * NX>(g.F + t * g.sF, F);
    load<T, NX>(g.c + t * g.sc, c);
    load_lower<T, NX>(g.SQ + t * g.sSQ, SQ);
  }
  SQSM_DEV void load_observation(const GammaView<T>& g, int64_t t) {
    load<T, NY * NX>(g.H + t * g.sH, H);
    load<T, NY>(g.d + t * g.sd, d);
    load_lower<T, NY>(g.SR + t * g.sSR, SR);
  }
  SQSM_DEV void load_all(const GammaView<T>& g, int64_t t) {
    load_transition(g, t);
    load_observation(g, t);
  }
};

// Record sizes are padded to whole 16-byte words (4 elements) so that
// records move with vector accesses.
template <int NX> struct FRec {
  static constexpr int A = 0, b = NX * NX, U = NX * NX + NX, eta = 2 * NX * NX + NX,
                       Z = 2 * NX * NX + 2 * NX, size = (3 * NX * NX + 2 * NX + 3) / 4 * 4;
};
template <int NX> struct SRec {
  static constexpr int E = 0, g = NX * NX, D = NX * NX + NX,
                       size = (2 * NX * NX + NX + 3) / 4 * 4;
};
// A Table 3 combine's gain G and A_j (I - U_i G^T), as the full filter pass
// stores them for the mean-only refinement passes (padded to 16 bytes).
template <int NX> struct FGm {
  static constexpr int G = 0, M = NX * NX, size = (2 * NX * NX + 3) / 4 * 4;
};
inline int frec_size(int nx) { return (3 * nx * nx + 2 * nx + 3) / 4 * 4; }
inline int srec_size(int nx) { return (2 * nx * nx + nx + 3) / 4 * 4; }
inline int fgm_size(int nx) { return (2 * nx * nx + 3) / 4 * 4; }
// Run-time sizes of PRec<nx, ny> and XRow<nx> (same formulas).
inline int prec_size(int nx, int ny) {
  const int h = (nx * nx + nx + nx * (nx + 1) / 2 + 3) / 4 * 4;
  return (h + ny * nx + ny + ny * (ny + 1) / 2 + 3) / 4 * 4;
}
inline int xrow_size(int nx) { return (nx + nx * (nx + 1) / 2 + 3) / 4 * 4; }

// Clear the padding words of a record after its fields are written.
template <typename T, int USED, int SIZE>
SQSM_DEV void zero_pad(T* rec) {
#pragma unroll
  for (int i = USED; i < SIZE; ++i) rec[i] = T(0);
}

constexpr double kLog2Pi = 1.8378770664093454835606594728112;

// Square-root Kalman predict + update from (m, N) at step k-1 to step k.
// This is the k = 1 construction of Lemma 1 / Table 1 with (m_0, N_0)
// replaced by (m, N): it is also the filter operator of Table 3 applied to a
// left operand that is a filtering distribution (A = 0), which is how the
// scan's carry is applied to the elements of a chunk.
//   m^- = F m + c, N^- = Tria([F N, S_Lambda]),
//   Psi = Tria([[H N^-, S_Omega], [N^-, 0]]),
//   m <- m^- + Psi_21 Psi_11^{-1} (y - H m^- - d),  N <- Psi_22,
// and returns l_k = log N(y; H m^- + d, Psi_11 Psi_11^T) (Sec. 5.1).
template <typename T, int NX, int NY>
SQSM_DEV T kf_step(const Gamma<T, NX, NY>& g, const T* y, T* m, T* N) {
  T mp[NX];
  mv<T, NX, NX>(g.F, m, mp);
#pragma unroll
  for (int i = 0; i < NX; ++i) mp[i] += g.c[i];
  T P[NX * 2 * NX];
#pragma unroll
  for (int i = 0; i < NX; ++i) {
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < NX; ++k) s += g.F[i * NX + k] * N[k * NX + j];
      P[i * 2 * NX + j] = s;                       // F N  (N lower)
      P[i * 2 * NX + NX + j] = g.SQ[i * NX + j];   // S_Lambda
    }
  }
  tria<T, NX, 2 * NX>(P);
  constexpr int W = NX + NY;
  T Psi[W * W];
#pragma unroll
  for (int i = 0; i < NY; ++i) {
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < NX; ++k) s += g.H[i * NX + k] * P[k * 2 * NX + j];
      Psi[i * W + j] = s;                          // H N^-
    }
#pragma unroll
    for (int j = 0; j < NY; ++j) Psi[i * W + NX + j] = g.SR[i * NY + j];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) {
#pragma unroll
    for (int j = 0; j < NX; ++j) Psi[(NY + i) * W + j] = j <= i ? P[i * 2 * NX + j] : T(0);
#pragma unroll
    for (int j = 0; j < NY; ++j) Psi[(NY + i) * W + NX + j] = T(0);
  }
  tria<T, W, W>(Psi);
  T e[NY], Y[NY * NY];
#pragma unroll
  for (int i = 0; i < NY; ++i) {
    T s = y[i] - g.d[i];
#pragma unroll
    for (int k = 0; k < NX; ++k) s -= g.H[i * NX + k] * mp[k];
    e[i] = s;
#pragma unroll
    for (int j = 0; j < NY; ++j) Y[i * NY + j] = j <= i ? Psi[i * W + j] : T(0);
  }
  lsolve<T, NY>(Y, e);                             // e = Y^{-1} v
  T ll = T(0);
#pragma unroll
  for (int i = 0; i < NY; ++i) ll += T(2) * sq_log(Y[i * NY + i]) + e[i] * e[i];
  ll = T(-0.5) * (T(NY) * T(kLog2Pi) + ll);
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    T s = mp[i];
#pragma unroll
    for (int k = 0; k < NY; ++k) s += Psi[(NY + i) * W + k] * e[k];  // K v = Psi21 e
    m[i] = s;
#pragma unroll
    for (int j = 0; j < NX; ++j) N[i * NX + j] = j <= i ? Psi[(NY + i) * W + NY + j] : T(0);
  }
  return ll;
}

// Z_k made square as in the proof of Lemma 1: zero columns when NX > NY,
// Tria(Z_k) when NX < NY.  Zr is NX x NY.
template <typename T, int NX, int NY>
SQSM_DEV void square_Z(T* Zr, T* Z) {
  if constexpr (NX >= NY) {
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j < NX; ++j) Z[i * NX + j] = j < NY ? Zr[i * NY + j] : T(0);
  } else {
    tria<T, NX, NY>(Zr);
    take_lower<T, NX, NY>(Zr, Z);
  }
}

// Filter element of Lemma 1.  first = true: Table 1 (k = 1, uses m0, N0);
// otherwise Table 2 (1 < k <= n) with Psi of eq. sqrt-filter-init-2.
// b_k uses d_k (the printed d_{k-1} is read as d_k).
template <typename T, int NX, int NY>
SQSM_DEV void filter_element(const Gamma<T, NX, NY>& g, const T* y, bool first, const T* m0,
                             const T* N0, T* e) {
  using R = FRec<NX>;
  constexpr int W = NX + NY;
  T Psi[W * W];
  T Bm[NX * NX];       // S_Lambda (k > 1) or N^- (k = 1)
  T mp[NX];            // c (k > 1) or m^- (k = 1)
  if (first) {
    mv<T, NX, NX>(g.F, m0, mp);
#pragma unroll
    for (int i = 0; i < NX; ++i) mp[i] += g.c[i];
    T P[NX * 2 * NX];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        T s = T(0);
#pragma unroll
        for (int k = j; k < NX; ++k) s += g.F[i * NX + k] * N0[k * NX + j];
        P[i * 2 * NX + j] = s;
        P[i * 2 * NX + NX + j] = g.SQ[i * NX + j];
      }
    tria<T, NX, 2 * NX>(P);
    take_lower<T, NX, 2 * NX>(P, Bm);
  } else {
#pragma unroll
    for (int i = 0; i < NX; ++i) mp[i] = g.c[i];
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) Bm[i] = g.SQ[i];
  }
#pragma unroll
  for (int i = 0; i < NY; ++i) {
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < NX; ++k) s += g.H[i * NX + k] * Bm[k * NX + j];
      Psi[i * W + j] = s;
    }
#pragma unroll
    for (int j = 0; j < NY; ++j) Psi[i * W + NX + j] = g.SR[i * NY + j];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) {
#pragma unroll
    for (int j = 0; j < NX; ++j) Psi[(NY + i) * W + j] = Bm[i * NX + j];
#pragma unroll
    for (int j = 0; j < NY; ++j) Psi[(NY + i) * W + NX + j] = T(0);
  }
  tria<T, W, W>(Psi);
  T Y[NY * NY];
#pragma unroll
  for (int i = 0; i < NY; ++i)
#pragma unroll
    for (int j = 0; j < NY; ++j) Y[i * NY + j] = j <= i ? Psi[i * W + j] : T(0);
  // residual for b: y - H m^- - d (k = 1) or y - H c - d (k > 1)
  T v[NY], r[NY];
#pragma unroll
  for (int i = 0; i < NY; ++i) {
    T s = y[i] - g.d[i], s2 = y[i] - g.d[i];
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      s -= g.H[i * NX + k] * mp[k];
      s2 -= g.H[i * NX + k] * g.c[k];
    }
    v[i] = s;
    r[i] = s2;
  }
  lsolve<T, NY>(Y, v);
  lsolve<T, NY>(Y, r);
  // b = m^- (or c) + Psi21 Y^{-1} v
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    T s = mp[i];
#pragma unroll
    for (int k = 0; k < NY; ++k) s += Psi[(NY + i) * W + k] * v[k];
    e[R::b + i] = s;
  }
  // Wm = Y^{-1} H F (NY x NX); Z = Wm^T; eta = Wm^T Y^{-1} (y - H c - d)
  T Wm[NY * NX];
  mm<T, NY, NX, NX>(g.H, g.F, Wm);
  {
    T inv[NY];
#pragma unroll
    for (int i = 0; i < NY; ++i) inv[i] = T(1) / Y[i * NY + i];
#pragma unroll
    for (int j = 0; j < NX; ++j) {
#pragma unroll
      for (int i = 0; i < NY; ++i) {
        T sacc = Wm[i * NX + j];
#pragma unroll
        for (int k = 0; k < i; ++k) sacc -= Y[i * NY + k] * Wm[k * NX + j];
        Wm[i * NX + j] = sacc * inv[i];
      }
    }
  }
  // A = (I - K H) F = F - Psi21 Wm  (k > 1);  A = 0 (k = 1)
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = g.F[i * NX + j];
#pragma unroll
      for (int k = 0; k < NY; ++k) s -= Psi[(NY + i) * W + k] * Wm[k * NX + j];
      e[R::A + i * NX + j] = first ? T(0) : s;
    }
#pragma unroll
  for (int i = 0; i < NX; ++i) {
#pragma unroll
    for (int j = 0; j < NX; ++j)
      e[R::U + i * NX + j] = j <= i ? Psi[(NY + i) * W + NY + j] : T(0);
    T s = T(0);
#pragma unroll
    for (int k = 0; k < NY; ++k) s += Wm[k * NX + i] * r[k];
    e[R::eta + i] = s;
  }
  T Zr[NX * NY];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NY; ++j) Zr[i * NY + j] = Wm[j * NX + i];
  square_Z<T, NX, NY>(Zr, e + R::Z);
  zero_pad<T, R::Z + NX * NX, R::size>(e);
}

// The blocks of Xi (eq. sqrt-filter-com-2), Xi = Tria([[M, I], [Z_j, 0]])
// with M = U_i^T Z_j, from two NX x 2NX Trias instead of one 2NX x 2NX one.
// Multiplying out Xi Xi^T = [[I + M M^T, M Z_j^T], [Z_j M^T, Z_j Z_j^T]]:
//   Xi_11 = Tria([M, I]),
//   Xi_21 = Z_j M^T Xi_11^{-T},
//   Xi_22 Xi_22^T = Z_j Z_j^T - Xi_21 Xi_21^T = Z_j (I + M^T M)^{-1} Z_j^T
//                 = W W^T  with  W = Z_j L^{-T},  L = Tria([M^T, I]),
// (the push-through identity); Xi_22 enters the operator only through
// Tria([A_i^T Xi_22, Z_i]), which W gives the same product.  Xi_11 and L
// are >= I, so the triangular solves are well conditioned.
template <typename T, int NX>
SQSM_DEV void xi_m(const T* Ui, const T* Zj, T* Mx) {
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = i; k < NX; ++k) s += Ui[k * NX + i] * Zj[k * NX + j];   // U_i lower
      Mx[i * NX + j] = s;
    }
}

// Tria([A, I]) for A (NX x NX), or Tria([A^T, I]) with TRANS.
template <typename T, int NX, bool TRANS>
SQSM_DEV void tria_with_identity(const T* A, T* L) {
  constexpr int C2 = 2 * NX;
  T B[NX * C2];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      B[i * C2 + j] = TRANS ? A[j * NX + i] : A[i * NX + j];
      B[i * C2 + NX + j] = i == j ? T(1) : T(0);
    }
  tria<T, NX, C2>(B);
  take_lower<T, NX, C2>(B, L);
}

// G = Xi_21 Xi_11^{-1} = Z_j M^T Xi_11^{-T} Xi_11^{-1}.
template <typename T, int NX>
SQSM_DEV void xi_gain(const T* Zj, const T* Mx, const T* X11, T* G) {
  mmt<T, NX, NX, NX>(Zj, Mx, G);
  rsolve_t<T, NX, NX>(G, X11);
  rsolve<T, NX, NX>(G, X11);
}

// b_ij and eta_ij of Table 3 from the combine's factors: A_i, U_i, Z_j, the
// gain G and A_j (I - U_i G^T) (see filter_combine).  The full operator and
// the mean-only refinement passes (which read the factors back from a
// table) both take this path, so the two give the same values bit for bit.
template <typename T, int NX>
SQSM_DEV void filter_combine_means(const T* Ai, const T* Ui, const T* Zj, const T* G,
                                   const T* AjM, const T* bi, const T* etai, const T* bj,
                                   const T* etaj, T* bo, T* etao) {
  // b_ij
  T t[NX], u[NX];
  mtv<T, NX, NX>(Ui, etaj, t);
  mv<T, NX, NX>(Ui, t, u);
#pragma unroll
  for (int i = 0; i < NX; ++i) u[i] += bi[i];
  mv<T, NX, NX>(AjM, u, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) bo[i] = t[i] + bj[i];
  // eta_ij
  T sv[NX], r[NX];
  mtv<T, NX, NX>(Zj, bi, sv);
  mv<T, NX, NX>(Zj, sv, r);
#pragma unroll
  for (int i = 0; i < NX; ++i) r[i] = etaj[i] - r[i];
  mtv<T, NX, NX>(Ui, r, t);
  mv<T, NX, NX>(G, t, sv);
#pragma unroll
  for (int i = 0; i < NX; ++i) r[i] -= sv[i];
  mtv<T, NX, NX>(Ai, r, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) etao[i] = t[i] + etai[i];
}

// Filter operator of Lemma 2 / Table 3 (right column) on full elements:
// out = e_i (x) e_j.  out must not alias the inputs.
//   G = Xi_21 Xi_11^{-1} (so that Xi_11^{-T} Xi_21^T = G^T),
//   (I + C_i J_j)^{-1} = I - U_i G^T                   (eq. sqrt-filter-com-3),
//   A_ij = A_j (I - U_i G^T) A_i,
//   b_ij = A_j (I - U_i G^T)(b_i + U_i U_i^T eta_j) + b_j,
//   U_ij = Tria([A_j U_i Xi_11^{-T}, U_j]),
//   eta_ij = A_i^T (I - G U_i^T)(eta_j - Z_j Z_j^T b_i) + eta_i,
//   Z_ij = Tria([A_i^T Xi_22, Z_i])  (with Xi_22 -> W, see above).
// PARTS selects the fields computed (bit 0: A, b, eta; bit 1: U; bit 2: Z),
// so that three threads can each take one part of a combine, each forming
// only the factors its part needs.  With gm (part 0) the combine's G and
// A_j (I - U_i G^T) are also stored there (FGm layout), for the mean-only
// passes that replay b_ij and eta_ij.
template <typename T, int NX, int PARTS = 7>
SQSM_DEV void filter_combine(const T* ei, const T* ej, T* out, T* gm = nullptr) {
  using R = FRec<NX>;
  constexpr int C2 = 2 * NX;
  constexpr bool ABE = PARTS & 1, UU = PARTS & 2, ZZ = PARTS & 4;
  const T* Ui = ei + R::U;
  const T* Zj = ej + R::Z;
  T Mx[NX * NX];
  xi_m<T, NX>(Ui, Zj, Mx);
  T X11[NX * NX];
  if constexpr (ABE || UU) tria_with_identity<T, NX, false>(Mx, X11);
  if constexpr (ABE) {
    T G[NX * NX];
    xi_gain<T, NX>(Zj, Mx, X11, G);
    // Minv = I - U_i G^T
    T Mi[NX * NX];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        T a = i == j ? T(1) : T(0);
#pragma unroll
        for (int k = 0; k <= i; ++k) a -= Ui[i * NX + k] * G[j * NX + k];
        Mi[i * NX + j] = a;
      }
    T AjM[NX * NX];
    mm<T, NX, NX, NX>(ej + R::A, Mi, AjM);
    mm<T, NX, NX, NX>(AjM, ei + R::A, out + R::A);
    filter_combine_means<T, NX>(ei + R::A, Ui, Zj, G, AjM, ei + R::b, ei + R::eta, ej + R::b,
                                ej + R::eta, out + R::b, out + R::eta);
    if (gm) {
      T v[FGm<NX>::size];
#pragma unroll
      for (int i = 0; i < NX * NX; ++i) {
        v[FGm<NX>::G + i] = G[i];
        v[FGm<NX>::M + i] = AjM[i];
      }
#pragma unroll
      for (int i = 2 * NX * NX; i < FGm<NX>::size; ++i) v[i] = T(0);
      vstore<T, FGm<NX>::size>(gm, v);
    }
  }
  if constexpr (UU) {
    // U_ij = Tria([A_j U_i Xi11^{-T}, U_j])
    T V[NX * NX];
    mm<T, NX, NX, NX>(ej + R::A, Ui, V);
    rsolve_t<T, NX, NX>(V, X11);
    T B[NX * C2];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        B[i * C2 + j] = V[i * NX + j];
        B[i * C2 + NX + j] = ej[R::U + i * NX + j];
      }
    tria<T, NX, C2>(B);
    take_lower<T, NX, C2>(B, out + R::U);
  }
  if constexpr (ZZ) {
    // Z_ij = Tria([A_i^T W, Z_i]),  W = Z_j L^{-T},  L = Tria([M^T, I])
    T L[NX * NX], W[NX * NX];
    tria_with_identity<T, NX, true>(Mx, L);
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) W[i] = Zj[i];
    rsolve_t<T, NX, NX>(W, L);
    T B[NX * C2];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j < NX; ++j) {
        T a = T(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) a += ei[R::A + k * NX + i] * W[k * NX + j];
        B[i * C2 + j] = a;
        B[i * C2 + NX + j] = ei[R::Z + i * NX + j];
      }
    tria<T, NX, C2>(B);
    take_lower<T, NX, C2>(B, out + R::Z);
  }
  if constexpr (PARTS == 7) zero_pad<T, R::Z + NX * NX, R::size>(out);
}

// Table 3 with a left operand that is a filtering distribution (A_i = 0):
// only b_ij and U_ij are needed (Xi_11 and G), so Xi_22, eta_ij and Z_ij are
// skipped.  (bi, Ui) -> (bo, Uo).
template <typename T, int NX>
SQSM_DEV void filter_apply(const T* bi, const T* Ui, const T* ej, T* bo, T* Uo) {
  using R = FRec<NX>;
  constexpr int C2 = 2 * NX;
  T Mx[NX * NX], X11[NX * NX], G[NX * NX];
  xi_m<T, NX>(Ui, ej + R::Z, Mx);
  tria_with_identity<T, NX, false>(Mx, X11);
  xi_gain<T, NX>(ej + R::Z, Mx, X11, G);
  T t[NX], u[NX], w[NX];
  mtv<T, NX, NX>(Ui, ej + R::eta, t);
  mv<T, NX, NX>(Ui, t, u);
#pragma unroll
  for (int i = 0; i < NX; ++i) u[i] += bi[i];
  // (I - U_i G^T) u
  // t = G^T u
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < NX; ++k) s += G[k * NX + i] * u[k];
    t[i] = s;
  }
  mv<T, NX, NX>(Ui, t, w);
#pragma unroll
  for (int i = 0; i < NX; ++i) w[i] = u[i] - w[i];
  mv<T, NX, NX>(ej + R::A, w, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) bo[i] = t[i] + ej[R::b + i];
  T V[NX * NX];
  mm<T, NX, NX, NX>(ej + R::A, Ui, V);
  rsolve_t<T, NX, NX>(V, X11);
  T B[NX * C2];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      B[i * C2 + j] = V[i * NX + j];
      B[i * C2 + NX + j] = ej[R::U + i * NX + j];
    }
  tria<T, NX, C2>(B);
  take_lower<T, NX, C2>(B, Uo);
}

// Smoother element of Lemma 3 / Table 4 (right column), 0 <= k < n, with Phi
// of eq. smooth-init-2:  E = Phi_21 Phi_11^{-1}, g = m^f - E (F m^f + c),
// D = Phi_22.  Uses only the transition part of g.
// The mean parts of Table 4, Table 5 and the RTS step, shared by the full
// kernels and by the mean-only kernels of the refinement passes (which must
// repeat the full kernels' operations exactly):
//   g_k = m^f_k - E_k (F m^f_k + c)                         (element),
//   E_ij = E_i E_j, g_ij = E_i g_j + g_i                    (combine),
//   g <- E_i g + g_i                                        (RTS step).
template <typename T, int NX>
SQSM_DEV void smoother_element_g(const T* E, const T* F, const T* c, const T* mf, T* g) {
  T fm[NX];
  mv<T, NX, NX>(F, mf, fm);
#pragma unroll
  for (int i = 0; i < NX; ++i) fm[i] += c[i];
#pragma unroll
  for (int i = 0; i < NX; ++i) {
    T s = mf[i];
#pragma unroll
    for (int k = 0; k < NX; ++k) s -= E[i * NX + k] * fm[k];
    g[i] = s;
  }
}

template <typename T, int NX>
SQSM_DEV void smoother_combine_g(const T* Ei, const T* gi, const T* Ej, const T* gj, T* Eo,
                                 T* go) {
  mm<T, NX, NX, NX>(Ei, Ej, Eo);
  T t[NX];
  mv<T, NX, NX>(Ei, gj, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) go[i] = t[i] + gi[i];
}

template <typename T, int NX>
SQSM_DEV void smoother_apply_g(const T* Ei, const T* gi, T* gm) {
  T t[NX];
  mv<T, NX, NX>(Ei, gm, t);
#pragma unroll
  for (int i = 0; i < NX; ++i) gm[i] = t[i] + gi[i];
}

template <typename T, int NX, int NY>
SQSM_DEV void smoother_element(const Gamma<T, NX, NY>& g, const T* mf, const T* Nf, T* e) {
  using R = SRec<NX>;
  constexpr int C2 = 2 * NX;
  T Phi[C2 * C2];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < NX; ++k) s += g.F[i * NX + k] * Nf[k * NX + j];
      Phi[i * C2 + j] = s;
      Phi[i * C2 + NX + j] = g.SQ[i * NX + j];
      Phi[(NX + i) * C2 + j] = Nf[i * NX + j];
      Phi[(NX + i) * C2 + NX + j] = T(0);
    }
  tria<T, C2, C2>(Phi);
  T P11[NX * NX];
  take_lower<T, NX, C2>(Phi, P11);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) e[R::E + i * NX + j] = Phi[(NX + i) * C2 + j];
  rsolve<T, NX, NX>(e + R::E, P11);
  smoother_element_g<T, NX>(e + R::E, g.F, g.c, mf, e + R::g);
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j)
      e[R::D + i * NX + j] = j <= i ? Phi[(NX + i) * C2 + NX + j] : T(0);
  zero_pad<T, R::D + NX * NX, R::size>(e);
}

// Caption of Table 4: E_n = 0, g_n = m^f_n, D_n = N^f_n.
template <typename T, int NX>
SQSM_DEV void smoother_element_last(const T* mf, const T* Nf, T* e) {
  using R = SRec<NX>;
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) {
    e[R::E + i] = T(0);
    e[R::D + i] = Nf[i];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) e[R::g + i] = mf[i];
  zero_pad<T, R::D + NX * NX, R::size>(e);
}

// Smoother operator of Lemma 4 / Table 5 (right column): out = e_i (x) e_j,
//   E_ij = E_i E_j, g_ij = E_i g_j + g_i, D_ij = Tria([E_i D_j, D_i]).
template <typename T, int NX>
SQSM_DEV void smoother_combine(const T* ei, const T* ej, T* out) {
  using R = SRec<NX>;
  constexpr int C2 = 2 * NX;
  smoother_combine_g<T, NX>(ei + R::E, ei + R::g, ej + R::E, ej + R::g, out + R::E, out + R::g);
  T B[NX * C2];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < NX; ++k) s += ei[R::E + i * NX + k] * ej[R::D + k * NX + j];
      B[i * C2 + j] = s;
      B[i * C2 + NX + j] = ei[R::D + i * NX + j];
    }
  tria<T, NX, C2>(B);
  take_lower<T, NX, C2>(B, out + R::D);
  zero_pad<T, R::D + NX * NX, R::size>(out);
}

// Table 5 with a right operand whose E is 0 (a smoothing distribution
// (g, D) = (m^s_{k+1}, N^s_{k+1})): this is the RTS step
//   m <- E_i m + g_i,  N <- Tria([E_i N, D_i]).   (gm, Dm) updated in place.
template <typename T, int NX>
SQSM_DEV void smoother_apply(const T* ei, T* gm, T* Dm) {
  using R = SRec<NX>;
  constexpr int C2 = 2 * NX;
  T B[NX * C2];
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = j; k < NX; ++k) s += ei[R::E + i * NX + k] * Dm[k * NX + j];
      B[i * C2 + j] = s;
      B[i * C2 + NX + j] = ei[R::D + i * NX + j];
    }
  tria<T, NX, C2>(B);
  smoother_apply_g<T, NX>(ei + R::E, ei + R::g, gm);
  take_lower<T, NX, C2>(B, Dm);
}

}  // namespace sqsm
