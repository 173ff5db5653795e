// Stochastic Ricker population model with Poisson counts (Sec. 6.1), the
// paper's general (non-additive) state-space model:
//   x_k = log a + x_{k-1} - exp(x_{k-1}) + q_k,  q_k ~ N(0, Q),
//   y_k | x_k ~ Poisson(b exp(x_k)),  E[y | x] = Var[y | x] = b exp(x),
// so the observation SLR takes the conditional factor sqrt(b exp(X_i)) of
// each sigma point (GSLR of Sec. 4.3).  n_x = n_y = 1; theta =
// (log a, log b, log Q).  A zero state factor (the known initial state)
// takes the SLR's limit, the Taylor linearisation.
#pragma once

#include "ct_model.cuh"

namespace sqsm {

template <typename T>
struct PopParams {
  T log_a, b, sq;   // log a, b, sqrt(Q)
};

template <typename T>
__global__ void pop_params_kernel(double th0, double th1, double th2, PopParams<T>* P) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  PopParams<T> p;
  p.log_a = (T)th0;
  p.b = (T)exp(th1);
  p.sq = (T)sqrt(exp(th2));
  *P = p;
}

SQSM_DEV float sq_exp(float x) { return expf(x); }
SQSM_DEV double sq_exp(double x) { return exp(x); }
SQSM_DEV float sq_expm1(float x) { return expm1f(x); }
SQSM_DEV double sq_expm1(double x) { return expm1(x); }

// One thread per step s: transition from state row s + b, observation at
// row s + b + 1 of the nominal trajectory; LIN 0: cubature (points m +- N),
// 1: Taylor; centered as in ct_slr_kernel_lin.  Records are PRec<1, 1>.
template <typename T, typename NO, int LIN>
__global__ void __launch_bounds__(kBlock)
pop_slr_kernel(DevLevel lv, int leaf, DevSeqs sq, const PopParams<T>* __restrict__ Pp, int centered,
               NO nom, const T* __restrict__ y, T* __restrict__ gam) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ch = tid / leaf;
  if (ch >= lv.n_chunks) return;
  const int j = (int)(tid - ch * leaf);
  if (j >= lv.count[ch]) return;
  const PopParams<T> P = *Pp;
  const int b = lv.seq[ch];
  const int64_t s = lv.first[ch] + j;
  const int64_t rp = s + b, rk = s + b + 1;
  Gamma<T, 1, 1> out;
  {
    // transition: f(x) = log a + x - e^x; differences f(m + d) - f(m) =
    // d - e^m expm1(d) without cancellation
    T m[1], N[1];
    nom.load(rp, m, N);
    const T em = sq_exp(m[0]);
    T fm;   // f(m) (absolute) or f(m) - m_k (deviation form)
    if (centered) {
      T mk[1];
      nom.load_mean(rk, mk);
      fm = P.log_a - em + (m[0] - mk[0]);
    } else {
      fm = P.log_a + m[0] - em;
    }
    T F, dbar = T(0);
    if (LIN == 0 && fabs(N[0]) > Tiny<T>::value) {
      const T dp = N[0];   // points m +- N (n_x = 1)
      const T zp = dp - em * sq_expm1(dp), zn = -dp - em * sq_expm1(-dp);
      F = (zp - zn) / (T(2) * dp);
      dbar = T(0.5) * (zp + zn);
      // one pair: its residual (zp + zn)/2 - dbar is 0, so Lambda = Q
    } else {
      F = T(1) - em;
    }
    out.F[0] = F;
    out.c[0] = fm + dbar - (centered ? T(0) : F * m[0]);
    out.SQ[0] = P.sq;
    out.store_transition(GammaPacked<T>{gam}, s);
  }
  {
    // observation: E[y | x] = b e^x, conditional factor sqrt(b e^x)
    T m[1], N[1];
    nom.load(rk, m, N);
    const T hm = P.b * sq_exp(m[0]);
    T H, dbar = T(0), S;
    if (LIN == 0 && fabs(N[0]) > Tiny<T>::value) {
      const T dp = N[0];
      const T zp = hm * sq_expm1(dp), zn = hm * sq_expm1(-dp);
      H = (zp - zn) / (T(2) * dp);
      dbar = T(0.5) * (zp + zn);
      // Omega = w (S+^2 + S-^2) (the pair's residual is 0), w = 1/2
      S = sq_sqrt(T(0.5) * (hm * sq_exp(dp) + hm * sq_exp(-dp)));
    } else {
      H = hm;
      S = sq_sqrt(hm);
    }
    out.H[0] = H;
    out.d[0] = hm + dbar - (centered ? T(0) : H * m[0]);
    out.SR[0] = S;
    out.store_observation(GammaPacked<T>{gam}, s);
  }
  (void)y;
}

template <typename T, typename NO>
void launch_pop_slr(unsigned grid, cudaStream_t s, int linearization, DevLevel lv, int leaf,
                    DevSeqs sq, const PopParams<T>* Pp, int centered, NO nom, const T* y, T* gam) {
  if (linearization == 0)
    pop_slr_kernel<T, NO, 0><<<grid, kBlock, 0, s>>>(lv, leaf, sq, Pp, centered, nom, y, gam);
  else
    pop_slr_kernel<T, NO, 1><<<grid, kBlock, 0, s>>>(lv, leaf, sq, Pp, centered, nom, y, gam);
}

}  // namespace sqsm
