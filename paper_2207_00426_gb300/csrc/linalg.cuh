// Small dense linear algebra held in registers (one thread per matrix).
//
// Matrices are row-major arrays with compile-time shapes; every loop is fully
// unrolled so that the arrays stay in registers.  Tria (Sec. 2.2) is an LQ
// factorisation by Householder reflections applied from the right.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define SQSM_DEV __device__ __forceinline__

namespace sqsm {

template <typename T> struct Tiny;
template <> struct Tiny<float> { static constexpr float value = 1e-30f; };
template <> struct Tiny<double> { static constexpr double value = 1e-280; };

SQSM_DEV float sq_sqrt(float x) { return sqrtf(x); }
SQSM_DEV double sq_sqrt(double x) { return sqrt(x); }
SQSM_DEV float sq_log(float x) { return logf(x); }
SQSM_DEV double sq_log(double x) { return log(x); }

// Square root and reciprocal for the reflector of one Householder step and
// the diagonal of triangular solves (normal x > 0).  FP32 starts from the hardware reciprocal square root and
// reciprocal estimates and takes one Newton step each (on y^2 = x from
// y = x rsqrt(x), and on 1/x, as in Markstein's refinements), which keeps
// them within about an ulp without the slow-path branch of the IEEE
// operations, so that a whole Tria is one branch-free block the compiler can
// schedule across reflections.  FP64 keeps the correctly rounded operations.
SQSM_DEV float hh_sqrt(float x) {
  const float r = rsqrtf(x);
  const float y = x * r;
  return fmaf(fmaf(-y, y, x), 0.5f * r, y);
}
SQSM_DEV double hh_sqrt(double x) { return sqrt(x); }
SQSM_DEV float hh_rcp(float x) {
  const float r = __fdividef(1.0f, x);
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}
SQSM_DEV double hh_rcp(double x) { return 1.0 / x; }

// Tria(A) for an R x C matrix `a` (Sec. 2.2): on return columns 0..R-1 of
// `a` hold the lower-triangular L with L L^T = A A^T and diag(L) >= 0 (the
// strictly upper part of those columns and columns R..C-1 are left as
// scratch).  Step i reflects row i onto its pivot: v = x + sign(x0)|x| e_0,
// applied to rows i+1.., after which column i of L is final; its sign is
// flipped so that L_ii = |x|.  A row whose remaining part is zero (rank
// deficiency) takes the identity reflector.  With NREF < R only the first
// NREF reflections are applied: rows 0..NREF-1 of L and columns 0..NREF-1 of
// the remaining rows are then final (used where only the leading block
// columns of the factor are needed).
template <typename T, int R, int C, int NREF = R>
SQSM_DEV void tria(T* a) {
  static_assert(R <= C, "tria is only used on R x C blocks with R <= C");
  static_assert(NREF <= R, "at most R reflections");
  // Branch-free: a zero row selects the identity reflector (tau = 0, column
  // left as is).  Dot products use two partial sums to halve their chains.
#pragma unroll
  for (int i = 0; i < NREF; ++i) {
    T s2a = T(0), s2b = T(0);
#pragma unroll
    for (int j = i; j < C; j += 2) {
      s2a += a[i * C + j] * a[i * C + j];
      if (j + 1 < C) s2b += a[i * C + j + 1] * a[i * C + j + 1];
    }
    const T s2 = s2a + s2b;
    const T x0 = a[i * C + i];
    const bool nz = s2 > Tiny<T>::value;
    const T alpha = hh_sqrt(nz ? s2 : T(1));
    const T sgn = x0 >= T(0) ? T(1) : T(-1);
    const T v0 = x0 + sgn * alpha;
    const T tau = nz ? hh_rcp(alpha * (alpha + (x0 >= T(0) ? x0 : -x0))) : T(0);
#pragma unroll
    for (int r = i + 1; r < R; ++r) {
      T wa = a[r * C + i] * v0, wb = T(0);
#pragma unroll
      for (int j = i + 1; j < C; j += 2) {
        wa += a[r * C + j] * a[i * C + j];
        if (j + 1 < C) wb += a[r * C + j + 1] * a[i * C + j + 1];
      }
      const T w = (wa + wb) * tau;
      // column i of L, with the sign flip that makes L_ii = alpha > 0
      const T ci = -sgn * (a[r * C + i] - w * v0);
      a[r * C + i] = nz ? ci : a[r * C + i];
#pragma unroll
      for (int j = i + 1; j < C; ++j) a[r * C + j] -= w * a[i * C + j];
    }
    a[i * C + i] = nz ? alpha : T(0);
  }
}

// Copy the R x R lower factor out of the first R columns of an R x C array.
template <typename T, int R, int C>
SQSM_DEV void take_lower(const T* a, T* L) {
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int j = 0; j < R; ++j) L[r * R + j] = (j <= r && j < C) ? a[r * C + j] : T(0);
}

// C[M][N] = A[M][K] B[K][N]
template <typename T, int M, int K, int N>
SQSM_DEV void mm(const T* A, const T* B, T* Cm) {
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) s += A[i * K + k] * B[k * N + j];
      Cm[i * N + j] = s;
    }
}

// C[M][N] = A[K][M]^T B[K][N]
template <typename T, int M, int K, int N>
SQSM_DEV void mtm(const T* A, const T* B, T* Cm) {
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) s += A[k * M + i] * B[k * N + j];
      Cm[i * N + j] = s;
    }
}

// C[M][N] = A[M][K] B[N][K]^T
template <typename T, int M, int K, int N>
SQSM_DEV void mmt(const T* A, const T* B, T* Cm) {
#pragma unroll
  for (int i = 0; i < M; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < K; ++k) s += A[i * K + k] * B[j * K + k];
      Cm[i * N + j] = s;
    }
}

// y[M] = A[M][N] x[N]
template <typename T, int M, int N>
SQSM_DEV void mv(const T* A, const T* x, T* y) {
#pragma unroll
  for (int i = 0; i < M; ++i) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < N; ++k) s += A[i * N + k] * x[k];
    y[i] = s;
  }
}

// y[N] = A[M][N]^T x[M]
template <typename T, int M, int N>
SQSM_DEV void mtv(const T* A, const T* x, T* y) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < M; ++k) s += A[k * N + i] * x[k];
    y[i] = s;
  }
}

// Lower Cholesky factor in place (upper part cleared).  A non-positive pivot
// gives NaN, as the standard form does when a covariance loses definiteness.
template <typename T, int N>
SQSM_DEV void chol_inplace(T* A) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T s = A[j * N + j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= A[j * N + k] * A[j * N + k];
    const T d = sq_sqrt(s);
    const T inv = T(1) / d;
    A[j * N + j] = d;
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      T t = A[i * N + j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= A[i * N + k] * A[j * N + k];
      A[i * N + j] = t * inv;
    }
#pragma unroll
    for (int i = 0; i < j; ++i) A[i * N + j] = T(0);
  }
}

// Triangular solves divide once per diagonal entry and multiply by the
// reciprocal elsewhere.

// x = L^{-1} b for lower L (N x N); in place on b.
template <typename T, int N>
SQSM_DEV void lsolve(const T* L, T* b) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T s = b[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s -= L[i * N + k] * b[k];
    b[i] = s / L[i * N + i];
  }
}

// x = L^{-T} b for lower L (N x N); in place on b.
template <typename T, int N>
SQSM_DEV void ltsolve(const T* L, T* b) {
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    T s = b[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) s -= L[k * N + i] * b[k];
    b[i] = s / L[i * N + i];
  }
}

// X <- X L^{-1} for X (M x N), lower L (N x N): each row x solves z L = x.
template <typename T, int M, int N>
SQSM_DEV void rsolve(T* X, const T* L) {
  T inv[N];
#pragma unroll
  for (int i = 0; i < N; ++i) inv[i] = hh_rcp(L[i * N + i]);
#pragma unroll
  for (int r = 0; r < M; ++r) {
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      T s = X[r * N + i];
#pragma unroll
      for (int k = i + 1; k < N; ++k) s -= X[r * N + k] * L[k * N + i];
      X[r * N + i] = s * inv[i];
    }
  }
}

// X <- X L^{-T} for X (M x N), lower L (N x N): each row x solves z L^T = x.
template <typename T, int M, int N>
SQSM_DEV void rsolve_t(T* X, const T* L) {
  T inv[N];
#pragma unroll
  for (int i = 0; i < N; ++i) inv[i] = hh_rcp(L[i * N + i]);
#pragma unroll
  for (int r = 0; r < M; ++r) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s = X[r * N + i];
#pragma unroll
      for (int k = 0; k < i; ++k) s -= X[r * N + k] * L[i * N + k];
      X[r * N + i] = s * inv[i];
    }
  }
}

template <typename T, int N>
SQSM_DEV void load(const T* __restrict__ g, T* r) {
#pragma unroll
  for (int i = 0; i < N; ++i) r[i] = g[i];
}

template <typename T, int N>
SQSM_DEV void store(T* __restrict__ g, const T* r) {
#pragma unroll
  for (int i = 0; i < N; ++i) g[i] = r[i];
}

// Load an N x N lower factor, zeroing the strictly upper part.
template <typename T, int N>
SQSM_DEV void load_lower(const T* __restrict__ g, T* r) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) r[i * N + j] = j <= i ? g[i * N + j] : T(0);
}

// N consecutive elements through 16-byte vector accesses (g 16-byte aligned,
// N * sizeof(T) a multiple of 16).
template <typename T, int N>
SQSM_DEV void vload(const T* __restrict__ g, T* r) {
  static_assert((N * sizeof(T)) % 16 == 0, "vector access of whole 16-byte words");
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 v = reinterpret_cast<const float4*>(g)[i];
      r[4 * i] = v.x; r[4 * i + 1] = v.y; r[4 * i + 2] = v.z; r[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N / 2; ++i) {
      const double2 v = reinterpret_cast<const double2*>(g)[i];
      r[2 * i] = v.x; r[2 * i + 1] = v.y;
    }
  }
}

template <typename T, int N>
SQSM_DEV void vstore(T* __restrict__ g, const T* r) {
  static_assert((N * sizeof(T)) % 16 == 0, "vector access of whole 16-byte words");
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
      reinterpret_cast<float4*>(g)[i] = make_float4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < N / 2; ++i)
      reinterpret_cast<double2*>(g)[i] = make_double2(r[2 * i], r[2 * i + 1]);
  }
}

// Store an N x N lower factor with explicit zeros above the diagonal.
template <typename T, int N>
SQSM_DEV void store_lower(T* __restrict__ g, const T* r) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) g[i * N + j] = j <= i ? r[i * N + j] : T(0);
}

template <typename T> SQSM_DEV bool finite(T x) { return isfinite(x); }

}  // namespace sqsm
