// Record layouts of the per-step tables of the reverse pass (host and
// device code both size buffers from them).
#pragma once

namespace sqsm {

// Per-step quantities of the reverse pass that depend on the linearisation
// and on the forward filter / smoother output only, and so stay fixed over
// the fixed-point iterations: one record per time step, written once per
// evaluation.  Every block starts on a 16-byte boundary.
//
// Kalman step k (t = k - 1), from the filter output at k - 1:
// m^- = F m + c, P^- = N^- N^-^T, S = H P^- H^T + Omega, W = S^{-1},
// U = P^- H^T, K = U W, v = y - H m^- - d, P_prev = N N^T; and the parts of
// its backward map that do not depend on the iterate: A = (I - K H) F,
// w = F^T H^T W v, C = F^T H^T W H F - w w^T (the map is B = A, r = w,
// s = lbar w + dfilt_m, S = -lbar/2 C + dfilt_P).  The map comes first, so
// that the up-sweep reads only the head.
template <int NX, int NY> struct KfTab {
  static constexpr int A = 0, w = NX * NX, C = NX * NX + NX, head = (2 * NX * NX + NX + 3) / 4 * 4,
                       W = head, v = W + NY * NY, K = v + NY, U = K + NX * NY, mp = U + NX * NY,
                       Pp = mp + NX, Pprev = Pp + NX * NX,
                       size = (Pprev + NX * NX + 3) / 4 * 4;
};

// RTS step at row e = k: gain G = P^f F^T (P^-_{k+1})^{-1} first (all the
// forward map needs), then W^- = (P^-_{k+1})^{-1}, P^f, and the differences
// dm = m^s_{k+1} - m^-_{k+1}, D = P^s_{k+1} - P^-_{k+1} used by its VJP.
template <int NX> struct RtsTab {
  static constexpr int G = 0, head = (NX * NX + 3) / 4 * 4, Wp = head, Pf = Wp + NX * NX,
                       dm = Pf + NX * NX, D = dm + NX, size = (D + NX * NX + 3) / 4 * 4;
};

// Cubature regressions of step s (Sec. 4.3), forward quantities of their
// VJP: regression matrix G and residual columns s_i of the transition at the
// nominal row e = s + b, and of the observation at row e + 1.
template <int NX, int NY> struct SlrTab {
  static constexpr int Gf = 0, sf = NX * NX, obs = (2 * NX * NX + 3) / 4 * 4, Gh = obs,
                       sh = Gh + NY * NX, size = (sh + NY * NX + 3) / 4 * 4;
};

// The kernels move records with 16-byte vector accesses from 256-byte
// aligned buffers, but only from three kinds of offset: the start of a
// record, its head (KfTab/RtsTab::head, SlrTab::obs) and the record size.
// Those are multiples of four elements (16 bytes in FP32, 32 in FP64); the
// inner block offsets (KfTab K, mp, ...; RtsTab Pf, ...) are not, and those
// blocks are read element by element.
static_assert(KfTab<5, 2>::head % 4 == 0 && KfTab<5, 2>::size % 4 == 0, "KfTab alignment");
static_assert(RtsTab<5>::head % 4 == 0 && RtsTab<5>::size % 4 == 0, "RtsTab alignment");
static_assert(SlrTab<5, 2>::obs % 4 == 0 && SlrTab<5, 2>::size % 4 == 0, "SlrTab alignment");

}  // namespace sqsm
