// Linear-Gaussian parallel square-root filter + smoother, float.
#include "dispatch.h"

namespace sqsm {
namespace {

template <int NX, int NY>
void run(const LgssmArgs& a, const LevelSet& Lf, const ScanBuffers& Wf, const LevelSet& Ls,
         const ScanBuffers& Ws, DevSeqs sq, double* partial, int* status, cudaStream_t s) {
  using T = float;
  GammaView<T> gv{(const T*)a.F, (const T*)a.c, (const T*)a.SQ, (const T*)a.H,
                  (const T*)a.d, (const T*)a.SR, a.sF, a.sc, a.sSQ, a.sH, a.sd, a.sSR};
  const RowsSplit<T, NX> fo{(T*)a.mf, (T*)a.Nf}, so{(T*)a.ms, (T*)a.Ns};
  enqueue_filter<T, NX, NY>(Lf, Wf, sq, gv, (const T*)a.y, (const T*)a.m0, (const T*)a.N0, fo,
                            partial, status, s, a.prof);
  enqueue_smoother<T, NX, NY>(Ls, Ws, sq, gv, fo, so, status, s, a.prof);
}

}  // namespace

int lgssm_enqueue_f32(const LgssmArgs& a, const LevelSet& Lf, const ScanBuffers& Wf,
                      const LevelSet& Ls, const ScanBuffers& Ws, DevSeqs sq, double* partial,
                      int* status, cudaStream_t s) {
#define SQSM_CASE(X, Y) \
  if (a.nx == X && a.ny == Y) { run<X, Y>(a, Lf, Wf, Ls, Ws, sq, partial, status, s); return 0; }
  SQSM_LGSSM_SHAPES(SQSM_CASE)
#undef SQSM_CASE
  return 2;
}

}  // namespace sqsm
