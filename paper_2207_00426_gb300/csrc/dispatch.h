// Interface between the host API (api.cu) and the kernel translation units
// (one per dtype and path, compiled in parallel).
#pragma once

#include <cuda_runtime.h>

#include "adj_tables.h"
#include "engine.cuh"

namespace sqsm {

struct LgssmArgs {
  int nx, ny;
  const void *F, *c, *SQ, *H, *d, *SR;
  int64_t sF, sc, sSQ, sH, sd, sSR;
  const void *m0, *N0, *y;
  void *mf, *Nf, *ms, *Ns;
  Prof* prof;
};

// Returns 0 if (nx, ny) is compiled in and the launches were enqueued,
// SQSM_ERR_UNSUPPORTED otherwise.  mf/Nf must be valid device buffers
// (the caller substitutes workspace for NULL outputs).
int lgssm_enqueue_f32(const LgssmArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s);
int lgssm_enqueue_f64(const LgssmArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s);
bool lgssm_shape_supported(int nx, int ny);

struct IplsArgs {
  int linearization, M;
  int leaf;            // leaf chunk length of the plan
  double theta[4], dt, sensors[4];   // theta[3]: CT second sensor log sigma
  const void *y, *m0, *N0, *init_ms, *init_Ns;
  void *ms, *Ns;
  double* loglik;
  // workspace
  void *mf, *Nf, *F, *c, *SQ, *H, *d, *SR, *params, *dm0;
  void *frows, *nrows;   // packed filter output and nominal trajectory (RowsPacked)
  Prof* prof;   // optional per-kernel events
  int centered = 1;   // 1: deviation coordinates, 0: printed absolute coordinates
  int textbook = 0;   // 1: cubature SLR with the printed (naive) differences
  // mixed-precision refinement of each iteration's linear smoother (deviation
  // coordinates only): passes, the nominal rows before the last smoother
  // pass (RowsPacked) and the refinement passes' log-likelihood partials
  int refine = 0;
  void* prevrows = nullptr;
  double* partial2 = nullptr;
  void* etab = nullptr;   // E_k per state row for the mean-only passes (null: full passes)
  void* ftab = nullptr;   // factors of the filter's latency-bound combines (FMeansTab;
                          // null: full filter passes)
};

// Everything of Alg. 3 after the parameter kernel; capturable.
void ipls_enqueue_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s);
void ipls_enqueue_f64(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s);
// Alg. 3 in the standard (covariance) form on a fold-only plan (radix 4);
// a.N0 holds prior covariances P0, a.Ns receives full covariances.
void std_ipls_enqueue_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                          const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                          int* status, cudaStream_t s);
void std_ipls_enqueue_f64(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                          const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                          int* status, cudaStream_t s);

// Phases of Alg. 3 for the tolerance mode (see ipls_phase).
enum { IPLS_PRE = 0, IPLS_ITER = 1, IPLS_POST = 2 };
void ipls_phase_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                    const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                    int* status, cudaStream_t s, int phase, unsigned* dmax);
void ipls_phase_f64(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                    const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                    int* status, cudaStream_t s, int phase, unsigned* dmax);
// The Ricker population model (n_x = n_y = 1): parameters and phases.
void pop_params_f32(const IplsArgs& a, cudaStream_t s);
void pop_params_f64(const IplsArgs& a, cudaStream_t s);
void pop_phase_f32(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                   const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                   int* status, cudaStream_t s, int phase, unsigned* dmax);
void pop_phase_f64(const IplsArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                   const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                   int* status, cudaStream_t s, int phase, unsigned* dmax);

// After one iteration of the tolerance mode: counts it in *iters, compares
// the largest change *dmax (float bits) with tol, clears *dmax, and sets
// whether the loop continues (change >= tol and fewer than max_iters
// iterations): into the conditional handle when use_handle, into *go when
// go is set.
void enqueue_tol_check(unsigned* dmax, int* iters, int max_iters, float tol,
                       cudaGraphConditionalHandle handle, int use_handle, int* go, cudaStream_t s);

// The parameter kernel (theta -> model constants), launched before each
// replay so that theta is not baked into a captured graph.
void ipls_params_f32(const IplsArgs& a, cudaStream_t s);
void ipls_params_f64(const IplsArgs& a, cudaStream_t s);

// Buffers of the NLL + gradient evaluation (all device).
struct AdjArgs {
  int iters;                          // adjoint fixed-point iterations
  int n_theta;                        // 3: one CT noise level, 4: one per sensor
  void *nom_m, *nom_N, *ms2, *Ns2;    // linearisation point, its smoother output
  void *dir, *dfilt, *gbar, *lam_a, *lam_b;
  void *ktab, *rtab, *stab;           // per-step KfTab / RtsTab / SlrTab records
  double *th_partial, *ll, *nll, *grad, *change;
  double* ichange;                    // relative change of the trajectory in one more iteration
  double tol;                         // fixed-point tolerance of the status check (<= 0: none)
  void* change_words;                 // four words: the adjoint's and the trajectory's change
};
void adj_enqueue_f32(const IplsArgs& a, const AdjArgs& g, const LevelSet& Lf,
                     const ScanBuffers& Wf, const LevelSet& Ls, const ScanBuffers& Ws,
                     const ScanBuffers& Wa, DevSeqs sq, double* partial, int* status,
                     cudaStream_t s);
void adj_enqueue_f64(const IplsArgs& a, const AdjArgs& g, const LevelSet& Lf,
                     const ScanBuffers& Wf, const LevelSet& Ls, const ScanBuffers& Ws,
                     const ScanBuffers& Wa, DevSeqs sq, double* partial, int* status,
                     cudaStream_t s);

// One SLR pass (Sec. 4.2 / 4.3) of the CT model into caller arrays.
void ct_linearize_f32(const IplsArgs& a, const LevelSet& Lf, DevSeqs sq, cudaStream_t s);
void ct_linearize_f64(const IplsArgs& a, const LevelSet& Lf, DevSeqs sq, cudaStream_t s);

void enqueue_loglik_reduce(DevSeqs sq, const double* partial, double* loglik, int* status,
                           cudaStream_t s, Prof* P = nullptr);

// Largest state dimension of the prior Cholesky kernel.
constexpr int kMaxPriorNx = 8;
// N0[b] = chol(P0[b]) in FP64 for b < batch (nx x nx, row-major, element
// type double if dtype_f64 else float); a P0 that is not positive definite
// gives a NaN factor and sets SQSM_ERR_NOT_PD in *status.
// Adds one group's {nll, grad[n_theta], adj_change, ipls_change} (device
// doubles, grad at g + 1, the changes at g + 5 and g + 6) into the caller's
// outputs (first group: copies).
void enqueue_nll_grad_group_add(int first, int n_theta, const double* g, double* nll, double* grad,
                                double* adj_change, double* ipls_change, cudaStream_t s);
void enqueue_prior_cholesky(int dtype_f64, int64_t batch, int nx, const void* P0, void* N0,
                            int* status, cudaStream_t s);

}  // namespace sqsm

// (nx, ny) pairs compiled into the linear smoother.
#define SQSM_LGSSM_SHAPES(X) X(1, 1) X(1, 2) X(2, 2) X(3, 2) X(2, 3) X(4, 2) X(5, 2) X(6, 3)
