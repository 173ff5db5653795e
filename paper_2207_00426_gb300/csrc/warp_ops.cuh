// Warp-cooperative forms of the scan operators, for the upper scan levels
// where few chunks are left and one thread per combine would leave the GPU
// idle: one warp per combine, operands in warp-private shared memory, each
// lane computing some rows or entries.  Same arithmetic as elements.cuh
// (Tables 3 and 5 and their restrictions to a distribution operand).
#pragma once

#include "elements.cuh"

namespace sqsm {

constexpr int kWarp = 32;

// Tria (Sec. 2.2) of an R x C block `a` (shared, row-major), rows
// distributed one per lane: lane `row` (0 <= row < R, `own` true) holds its
// row in registers; for each reflector the pivot lane publishes v, tau and
// the sign in `vb` (C + 2 values) and every lower row applies it.  Lanes
// that hold no row still take part in the __syncwarp()s.  On return columns
// 0..R-1 of `a` hold L (lower, diagonal >= 0) as in tria().
template <typename T, int R, int C, int NREF = R>
SQSM_DEV void wtria_rows(T* a, T* vb, int row, bool own) {
  static_assert(R <= C && NREF <= R && R <= kWarp, "shape");
  T x[C];
  if (own) {
#pragma unroll
    for (int j = 0; j < C; ++j) x[j] = a[row * C + j];
  }
#pragma unroll
  for (int i = 0; i < NREF; ++i) {
    if (own && row == i) {
      T s2 = T(0);
#pragma unroll
      for (int j = i; j < C; ++j) s2 += x[j] * x[j];
      const T x0 = x[i];
      if (s2 > Tiny<T>::value) {
        const T alpha = sq_sqrt(s2);
        const T sgn = x0 >= T(0) ? T(1) : T(-1);
        vb[i] = x0 + sgn * alpha;
#pragma unroll
        for (int j = i + 1; j < C; ++j) vb[j] = x[j];
        vb[C] = T(1) / (alpha * (alpha + (x0 >= T(0) ? x0 : -x0)));
        vb[C + 1] = sgn;
        x[i] = alpha;
      } else {
        vb[C] = T(0);
        x[i] = T(0);
      }
    }
    __syncwarp();
    if (own && row > i) {
      const T tau = vb[C];
      if (tau != T(0)) {
        const T sgn = vb[C + 1];
        T w = x[i] * vb[i];
#pragma unroll
        for (int j = i + 1; j < C; ++j) w += x[j] * vb[j];
        w *= tau;
        x[i] = -sgn * (x[i] - w * vb[i]);
#pragma unroll
        for (int j = i + 1; j < C; ++j) x[j] -= w * vb[j];
      }
    }
    __syncwarp();
  }
  if (own) {
#pragma unroll
    for (int j = 0; j < C; ++j) a[row * C + j] = x[j];
  }
  __syncwarp();
}

template <typename T, int N>
SQSM_DEV void wcopy(const T* src, T* dst, int lane) {
  for (int i = lane; i < N; i += kWarp) dst[i] = src[i];
}

// Warp-private workspace of the filter combine.
template <typename T, int NX> struct WFilterWs {
  static constexpr int C2 = 2 * NX;
  T X[C2 * C2], G[NX * NX], Mi[NX * NX], AjM[NX * NX], Bu[NX * C2], Bz[NX * C2];
  T vb0[C2 + 2], vb1[C2 + 2], t[NX], u[NX], r[NX], q[NX];
};

// Xi of eq. sqrt-filter-com-2, G = Xi21 Xi11^{-1} and (I + C_i J_j)^{-1}.
template <typename T, int NX, int NREF>
SQSM_DEV void wxi(const T* Ui, const T* Zj, WFilterWs<T, NX>& w, int lane) {
  constexpr int C2 = 2 * NX;
  for (int o = lane; o < C2 * C2; o += kWarp) {
    const int r = o / C2, c = o % C2;
    T v;
    if (r < NX && c < NX) {
      v = T(0);
      // U_i is lower; Z_j need not be (a single element's Z is zero-padded)
      for (int k = r; k < NX; ++k) v += Ui[k * NX + r] * Zj[k * NX + c];
    } else if (r < NX) {
      v = (c - NX == r) ? T(1) : T(0);
    } else if (c < NX) {
      v = Zj[(r - NX) * NX + c];
    } else {
      v = T(0);
    }
    w.X[o] = v;
  }
  __syncwarp();
  wtria_rows<T, C2, C2, NREF>(w.X, w.vb0, lane, lane < C2);
  // G = Xi21 Xi11^{-1}: lane r solves row r
  if (lane < NX) {
    T g[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) g[i] = w.X[(NX + lane) * C2 + i];
#pragma unroll
    for (int i = NX - 1; i >= 0; --i) {
      T s = g[i];
#pragma unroll
      for (int k = i + 1; k < NX; ++k) s -= g[k] * w.X[k * C2 + i];
      g[i] = s * (T(1) / w.X[i * C2 + i]);
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) w.G[lane * NX + i] = g[i];
  }
  __syncwarp();
  // Mi = I - U_i G^T
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    T s = i == j ? T(1) : T(0);
    for (int k = 0; k <= i; ++k) s -= Ui[i * NX + k] * w.G[j * NX + k];
    w.Mi[o] = s;
  }
  __syncwarp();
}

// b_ij and the first block of U_ij's Tria input (A_j U_i Xi11^{-T} | U_j).
template <typename T, int NX>
SQSM_DEV void wfilter_bU(const T* bi, const T* Ui, const T* Aj, const T* bj, const T* etaj,
                         const T* Uj, WFilterWs<T, NX>& w, T* bo, int lane) {
  constexpr int C2 = 2 * NX;
  // AjM = A_j Mi ; t = U_i^T eta_j ; V = A_j U_i (into Bu)
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    T s = T(0), v = T(0);
    for (int k = 0; k < NX; ++k) s += Aj[i * NX + k] * w.Mi[k * NX + j];
    for (int k = j; k < NX; ++k) v += Aj[i * NX + k] * Ui[k * NX + j];
    w.AjM[o] = s;
    w.Bu[i * C2 + j] = v;
    w.Bu[i * C2 + NX + j] = Uj[o];
  }
  if (lane < NX) {
    T s = T(0);
    for (int k = lane; k < NX; ++k) s += Ui[k * NX + lane] * etaj[k];
    w.t[lane] = s;
  }
  __syncwarp();
  if (lane < NX) {
    // u = b_i + U_i t
    T s = bi[lane];
    for (int k = 0; k <= lane; ++k) s += Ui[lane * NX + k] * w.t[k];
    w.u[lane] = s;
    // V row <- V row Xi11^{-T}
    T v[NX];
#pragma unroll
    for (int i = 0; i < NX; ++i) v[i] = w.Bu[lane * C2 + i];
#pragma unroll
    for (int i = 0; i < NX; ++i) {
      T s2 = v[i];
#pragma unroll
      for (int k = 0; k < i; ++k) s2 -= v[k] * w.X[i * C2 + k];
      v[i] = s2 * (T(1) / w.X[i * C2 + i]);
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) w.Bu[lane * C2 + i] = v[i];
  }
  __syncwarp();
  if (lane < NX) {
    T s = bj[lane];
    for (int k = 0; k < NX; ++k) s += w.AjM[lane * NX + k] * w.u[k];
    bo[lane] = s;
  }
  __syncwarp();
}

// Table 3 (right column) on full elements, one warp: out = ei (x) ej.
template <typename T, int NX>
SQSM_DEV void wfilter_combine(const T* ei, const T* ej, T* out, WFilterWs<T, NX>& w, int lane) {
  using R = FRec<NX>;
  constexpr int C2 = 2 * NX;
  const T* Ai = ei + R::A;
  const T* Ui = ei + R::U;
  const T* Aj = ej + R::A;
  const T* Zj = ej + R::Z;
  wxi<T, NX, C2>(Ui, Zj, w, lane);
  wfilter_bU<T, NX>(ei + R::b, Ui, Aj, ej + R::b, ej + R::eta, ej + R::U, w, out + R::b, lane);
  // A_ij = AjM A_i ; Bz = [A_i^T Xi22 | Z_i] ; s = Z_j^T b_i
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    T s = T(0), z = T(0);
    for (int k = 0; k < NX; ++k) s += w.AjM[i * NX + k] * Ai[k * NX + j];
    for (int k = j; k < NX; ++k) z += Ai[k * NX + i] * w.X[(NX + k) * C2 + NX + j];
    out[R::A + o] = s;
    w.Bz[i * C2 + j] = z;
    w.Bz[i * C2 + NX + j] = ei[R::Z + o];
  }
  if (lane < NX) {
    T s = T(0);
    for (int k = 0; k < NX; ++k) s += Zj[k * NX + lane] * ei[R::b + k];
    w.t[lane] = s;
  }
  __syncwarp();
  // eta_ij = A_i^T (r - G U_i^T r) + eta_i, r = eta_j - Z_j (Z_j^T b_i)
  if (lane < NX) {
    T s = ej[R::eta + lane];
    for (int k = 0; k < NX; ++k) s -= Zj[lane * NX + k] * w.t[k];
    w.r[lane] = s;
  }
  __syncwarp();
  if (lane < NX) {
    T s = T(0);
    for (int k = lane; k < NX; ++k) s += Ui[k * NX + lane] * w.r[k];
    w.q[lane] = s;
  }
  __syncwarp();
  if (lane < NX) {
    T s = w.r[lane];
    for (int k = 0; k < NX; ++k) s -= w.G[lane * NX + k] * w.q[k];
    w.u[lane] = s;
  }
  __syncwarp();
  if (lane < NX) {
    T s = ei[R::eta + lane];
    for (int k = 0; k < NX; ++k) s += Ai[k * NX + lane] * w.u[k];
    out[R::eta + lane] = s;
  }
  // U_ij = Tria(Bu) on lanes 0..NX-1, Z_ij = Tria(Bz) on lanes 16..16+NX-1
  {
    const bool gz = lane >= 16;
    const int row = gz ? lane - 16 : lane;
    T* Bm = gz ? w.Bz : w.Bu;
    T* vb = gz ? w.vb1 : w.vb0;
    wtria_rows<T, NX, C2>(Bm, vb, row, row < NX);
  }
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    out[R::U + o] = j <= i ? w.Bu[i * C2 + j] : T(0);
    out[R::Z + o] = j <= i ? w.Bz[i * C2 + j] : T(0);
  }
  __syncwarp();
}

// Table 3 with a distribution as left operand (A_i = 0): (bi, Ui) -> (bo, Uo).
template <typename T, int NX>
SQSM_DEV void wfilter_apply(const T* bi, const T* Ui, const T* ej, T* bo, T* Uo,
                            WFilterWs<T, NX>& w, int lane) {
  using R = FRec<NX>;
  constexpr int C2 = 2 * NX;
  wxi<T, NX, NX>(Ui, ej + R::Z, w, lane);
  wfilter_bU<T, NX>(bi, Ui, ej + R::A, ej + R::b, ej + R::eta, ej + R::U, w, bo, lane);
  wtria_rows<T, NX, C2>(w.Bu, w.vb0, lane, lane < NX);
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    Uo[o] = j <= i ? w.Bu[i * C2 + j] : T(0);
  }
  __syncwarp();
}

template <typename T, int NX> struct WSmootherWs {
  T B[NX * 2 * NX], vb[2 * NX + 2], g[NX];
};

// Table 5 (right column), one warp: out = ei (x) ej.
template <typename T, int NX>
SQSM_DEV void wsmoother_combine(const T* ei, const T* ej, T* out, WSmootherWs<T, NX>& w,
                                int lane) {
  using R = SRec<NX>;
  constexpr int C2 = 2 * NX;
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    T e = T(0), b = T(0);
    for (int k = 0; k < NX; ++k) e += ei[R::E + i * NX + k] * ej[R::E + k * NX + j];
    for (int k = j; k < NX; ++k) b += ei[R::E + i * NX + k] * ej[R::D + k * NX + j];
    out[R::E + o] = e;
    w.B[i * C2 + j] = b;
    w.B[i * C2 + NX + j] = ei[R::D + o];
  }
  if (lane < NX) {
    T s = ei[R::g + lane];
    for (int k = 0; k < NX; ++k) s += ei[R::E + lane * NX + k] * ej[R::g + k];
    out[R::g + lane] = s;
  }
  __syncwarp();
  wtria_rows<T, NX, C2>(w.B, w.vb, lane, lane < NX);
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    out[R::D + o] = j <= i ? w.B[i * C2 + j] : T(0);
  }
  __syncwarp();
}

// Table 5 with a distribution (E = 0) as right operand: the RTS step,
// (gm, Dm) <- (E_i gm + g_i, Tria([E_i Dm, D_i])), in place (shared).
template <typename T, int NX>
SQSM_DEV void wsmoother_apply(const T* ei, T* gm, T* Dm, WSmootherWs<T, NX>& w, int lane) {
  using R = SRec<NX>;
  constexpr int C2 = 2 * NX;
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    T b = T(0);
    for (int k = j; k < NX; ++k) b += ei[R::E + i * NX + k] * Dm[k * NX + j];
    w.B[i * C2 + j] = b;
    w.B[i * C2 + NX + j] = ei[R::D + o];
  }
  if (lane < NX) {
    T s = ei[R::g + lane];
    for (int k = 0; k < NX; ++k) s += ei[R::E + lane * NX + k] * gm[k];
    w.g[lane] = s;
  }
  __syncwarp();
  wtria_rows<T, NX, C2>(w.B, w.vb, lane, lane < NX);
  for (int o = lane; o < NX * NX; o += kWarp) {
    const int i = o / NX, j = o % NX;
    Dm[o] = j <= i ? w.B[i * C2 + j] : T(0);
  }
  if (lane < NX) gm[lane] = w.g[lane];
  __syncwarp();
}

}  // namespace sqsm
