// Segmented reduce-then-scan of the square-root filter (Alg. 1) and smoother
// (Alg. 2) over a batch of independent sequences.
//
// Level 0 items are the time steps (filter, k = 1..n_b) or the smoothing
// elements (smoother, k = 0..n_b) of each sequence; a level-l chunk is a run
// of consecutive items of one sequence, folded by one thread into one item of
// level l+1, until every sequence has a single item.  The down-sweep then
// gives every item the exclusive prefix (filter) or suffix (smoother) of its
// sequence -- a filtering (resp. smoothing) distribution, i.e. an element
// with A = 0 (resp. E = 0) -- and the leaves apply it to their own steps.
// Applying a distribution to an element is Table 3 (resp. Table 5) with that
// zero block, which is the sequential square-root Kalman (resp. RTS) step.
//
// No thread waits on another: levels are separate launches.
#pragma once

#include "elements.cuh"

namespace sqsm {

// One level of the plan (device arrays).
struct DevLevel {
  int64_t n_chunks;
  const int64_t* first;   // first item of each chunk (global item index)
  const int32_t* count;   // items in each chunk
  const int32_t* seq;     // sequence of each chunk
};

// Sequence bookkeeping: offsets[b] = first observation of sequence b
// (observations of b are rows offsets[b]..offsets[b+1]-1; its state rows are
// offsets[b]+b .. offsets[b+1]+b).
struct DevSeqs {
  int32_t B;
  const int64_t* offsets;        // B+1
  const int64_t* leaf_chunk_off; // B+1: leaf chunks of sequence b
};

constexpr int kBlock = 128;

template <typename T, int N>
SQSM_DEV void copy(const T* a, T* b) {
#pragma unroll
  for (int i = 0; i < N; ++i) b[i] = a[i];
}

SQSM_DEV void flag_status(int* status, int code) {
  if (status) atomicOr(status, code);
}

// ---------------------------------------------------------------------------
// Filter
// ---------------------------------------------------------------------------

// Leaf up-sweep: build the elements of Lemma 1 for the steps of a chunk and
// fold them left to right with Table 3.
template <typename T, int NX, int NY, typename GV>
__global__ void __launch_bounds__(kBlock)
filter_leaf_up(DevLevel lv, DevSeqs sq, GV gv, const T* __restrict__ y,
               const T* __restrict__ m0, const T* __restrict__ N0, T* __restrict__ items) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = FRec<NX>::size;
  const int b = lv.seq[c];
  const int64_t s0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t off = sq.offsets[b];
  T agg[REC], el[REC], tmp[REC];
  T m0b[NX], N0b[NX * NX];
  load<T, NX>(m0 + (int64_t)b * NX, m0b);
  load_lower<T, NX>(N0 + (int64_t)b * NX * NX, N0b);
  for (int j = 0; j < cnt; ++j) {
    const int64_t s = s0 + j;
    Gamma<T, NX, NY> g;
    g.load_all(gv, s);
    T ys[NY];
    load<T, NY>(y + s * NY, ys);
    if (j == 0) {
      filter_element<T, NX, NY>(g, ys, s == off, m0b, N0b, agg);
    } else {
      filter_element<T, NX, NY>(g, ys, s == off, m0b, N0b, el);
      filter_combine<T, NX>(agg, el, tmp);
      copy<T, REC>(tmp, agg);
    }
  }
  vstore<T, REC>(items + c * REC, agg);
}

// Upper up-sweep: fold `count` consecutive items left to right.
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
filter_up(DevLevel lv, const T* __restrict__ items_in, T* __restrict__ items_out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = FRec<NX>::size;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T agg[REC], el[REC], tmp[REC];
  vload<T, REC>(items_in + i0 * REC, agg);
  for (int j = 1; j < cnt; ++j) {
    vload<T, REC>(items_in + (i0 + j) * REC, el);
    filter_combine<T, NX>(agg, el, tmp);
    copy<T, REC>(tmp, agg);
  }
  vstore<T, REC>(items_out + c * REC, agg);
}

// Upper down-sweep: item c of level l+1 carries the filtering distribution
// (b, U) just before its chunk (flag 0: none, the chunk starts the
// sequence).  Give each item of the chunk its own exclusive prefix.
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
filter_down(DevLevel lv, const T* __restrict__ items, const T* __restrict__ carry_in,
            const int* __restrict__ flag_in, T* __restrict__ carry_out, int* __restrict__ flag_out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = FRec<NX>::size;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  int flag = flag_in[c];
  const RowsPacked<T, NX> cin{(T*)carry_in}, cout{carry_out};
  T cb[NX], cU[NX * NX];
  cin.load(c, cb, cU);
  for (int j = 0; j < cnt; ++j) {
    const int64_t i = i0 + j;
    cout.store(i, cb, cU);
    flag_out[i] = flag;
    if (j + 1 < cnt) {
      const T* it = items + i * REC;
      if (flag) {
        T el[REC], nb[NX], nU[NX * NX];
        vload<T, REC>(it, el);
        filter_apply<T, NX>(cb, cU, el, nb, nU);
        copy<T, NX>(nb, cb);
        copy<T, NX * NX>(nU, cU);
      } else {
        load<T, NX>(it + FRec<NX>::b, cb);
        load<T, NX * NX>(it + FRec<NX>::U, cU);
        flag = 1;
      }
    }
  }
}

// Leaf down-sweep: sequential square-root Kalman steps from the chunk's
// carry (or from the prior (m0, N0) for the first chunk of a sequence),
// writing m^f, N^f and the chunk's partial log-likelihood (FP64 sum).
template <typename T, int NX, int NY, typename GV, typename FO>
__global__ void __launch_bounds__(kBlock)
filter_leaf_down(DevLevel lv, DevSeqs sq, GV gv, const T* __restrict__ y,
                 const T* __restrict__ m0, const T* __restrict__ N0,
                 const T* __restrict__ carry, const int* __restrict__ flag,
                 FO fo, double* __restrict__ partial, int* status) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  const int b = lv.seq[c];
  const int64_t s0 = lv.first[c];
  const int cnt = lv.count[c];
  T m[NX], N[NX * NX];
  if (flag[c]) {
    RowsPacked<T, NX>{(T*)carry}.load(c, m, N);
  } else {
    load<T, NX>(m0 + (int64_t)b * NX, m);
    load_lower<T, NX>(N0 + (int64_t)b * NX * NX, N);
    fo.store(sq.offsets[b] + b, m, N);   // k = 0
  }
  double acc = 0.0;
  bool ok = true;
  for (int j = 0; j < cnt; ++j) {
    const int64_t s = s0 + j;
    Gamma<T, NX, NY> g;
    g.load_all(gv, s);
    T ys[NY];
    load<T, NY>(y + s * NY, ys);
    const T ll = kf_step<T, NX, NY>(g, ys, m, N);
    acc += (double)ll;
    fo.store(s + b + 1, m, N);
#pragma unroll
    for (int i = 0; i < NX; ++i) ok = ok && finite(m[i]);
  }
  if (partial) partial[c] = acc;
  if (!ok) flag_status(status, 8);
}

// ---------------------------------------------------------------------------
// Smoother (reverse scan)
// ---------------------------------------------------------------------------

// Leaf up-sweep: build the elements of Lemma 3 for the chunk's k (state
// rows) and fold them right to left with Table 5.
template <typename T, int NX, int NY, typename GV, typename FO>
__global__ void __launch_bounds__(kBlock)
smoother_leaf_up(DevLevel lv, DevSeqs sq, GV gv, FO fo, T* __restrict__ items,
                 T* __restrict__ etab) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = SRec<NX>::size;
  const int b = lv.seq[c];
  const int64_t e0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t so = sq.offsets[b] + b;
  const int64_t nb = sq.offsets[b + 1] - sq.offsets[b];
  T agg[REC], el[REC], tmp[REC];
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t e = e0 + j;
    const int64_t k = e - so;
    T m[NX], N[NX * NX];
    fo.load(e, m, N);
    T* dst = (j == cnt - 1) ? agg : el;
    if (k == nb) {
      smoother_element_last<T, NX>(m, N, dst);
    } else {
      Gamma<T, NX, NY> g;
      g.load_transition(gv, sq.offsets[b] + k);
      smoother_element<T, NX, NY>(g, m, N, dst);
      // E_k for the mean-only refinement passes (with the first words of g
      // in the padding)
      if (etab) vstore<T, ETab<NX>::size>(etab + e * ETab<NX>::size, dst + SRec<NX>::E);
    }
    if (j != cnt - 1) {
      smoother_combine<T, NX>(el, agg, tmp);
      copy<T, REC>(tmp, agg);
    }
  }
  vstore<T, REC>(items + c * REC, agg);
}

// Upper up-sweep: fold `count` items right to left.
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
smoother_up(DevLevel lv, const T* __restrict__ items_in, T* __restrict__ items_out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = SRec<NX>::size;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T agg[REC], el[REC], tmp[REC];
  vload<T, REC>(items_in + (i0 + cnt - 1) * REC, agg);
  for (int j = cnt - 2; j >= 0; --j) {
    vload<T, REC>(items_in + (i0 + j) * REC, el);
    smoother_combine<T, NX>(el, agg, tmp);
    copy<T, REC>(tmp, agg);
  }
  vstore<T, REC>(items_out + c * REC, agg);
}

// Upper down-sweep: item c of level l+1 carries the smoothing distribution
// (g, D) just after its chunk (flag 0: none, the chunk ends the sequence).
template <typename T, int NX>
__global__ void __launch_bounds__(kBlock)
smoother_down(DevLevel lv, const T* __restrict__ items, const T* __restrict__ carry_in,
              const int* __restrict__ flag_in, T* __restrict__ carry_out, int* __restrict__ flag_out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = SRec<NX>::size;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  int flag = flag_in[c];
  const RowsPacked<T, NX> cin{(T*)carry_in}, cout{carry_out};
  T cg[NX], cD[NX * NX];
  cin.load(c, cg, cD);
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t i = i0 + j;
    cout.store(i, cg, cD);
    flag_out[i] = flag;
    if (j > 0) {
      const T* it = items + i * REC;
      if (flag) {
        T el[REC];
        vload<T, REC>(it, el);
        smoother_apply<T, NX>(el, cg, cD);
      } else {
        load<T, NX>(it + SRec<NX>::g, cg);
        load<T, NX * NX>(it + SRec<NX>::D, cD);
        flag = 1;
      }
    }
  }
}

// Leaf down-sweep: sequential square-root RTS steps from the chunk's carry
// (m^s, N^s just after the chunk), writing m^s, N^s to `out_rows`.  With
// add_nominal the scan runs on deviations from a nominal trajectory held in
// `out_rows` itself, and the written mean is nominal + deviation (each row is
// read, then written, by the same thread); with dmax set, the largest
// change of a mean from the one held in `out_rows` (the deviation, with
// add_nominal) is max-reduced over all rows into *dmax (float bits).
template <typename T, int NX, int NY, typename GV, typename FO, typename SO>
__global__ void __launch_bounds__(kBlock)
smoother_leaf_down(DevLevel lv, DevSeqs sq, GV gv, FO fo, const T* __restrict__ carry,
                   const int* __restrict__ flag, SO out_rows, int* status, bool add_nominal,
                   unsigned* dmax) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = SRec<NX>::size;
  const int b = lv.seq[c];
  const int64_t e0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t r0 = sq.offsets[b] + b;
  const int64_t nb = sq.offsets[b + 1] - sq.offsets[b];
  float change = 0.f;
  T gm[NX], Dm[NX * NX];
  if (flag[c]) RowsPacked<T, NX>{(T*)carry}.load(c, gm, Dm);
  bool ok = true;
  // The inputs of a step (filter row, transition record, the mean held in
  // out_rows) do not depend on the steps after it, so each iteration issues
  // the loads of the next step before computing its own: their latency
  // overlaps this step's element and RTS step instead of stalling the chain
  // (the row it writes is never one it prefetches).
  const bool need_old = add_nominal || dmax != nullptr;
  auto fetch = [&](int j, T* m, T* N, Gamma<T, NX, NY>& g, T* old) {
    const int64_t e = e0 + j;
    fo.load(e, m, N);
    if (e - r0 != nb) g.load_transition(gv, sq.offsets[b] + (e - r0));
    if (need_old) out_rows.load_mean(e, old);
  };
  T m[NX], N[NX * NX], old[NX];
  Gamma<T, NX, NY> g;
  fetch(cnt - 1, m, N, g, old);
  for (int j = cnt - 1; j >= 0; --j) {
    const int64_t e = e0 + j;
    const int64_t k = e - r0;
    T pm[NX], pN[NX * NX], pold[NX];
    Gamma<T, NX, NY> pg;
    if (j > 0) fetch(j - 1, pm, pN, pg, pold);
    if (k == nb) {
      copy<T, NX>(m, gm);
      copy<T, NX * NX>(N, Dm);
    } else {
      T el[REC];
      smoother_element<T, NX, NY>(g, m, N, el);
      smoother_apply<T, NX>(el, gm, Dm);
    }
    if (add_nominal) {
      T out[NX];
#pragma unroll
      for (int i = 0; i < NX; ++i) out[i] = old[i] + gm[i];
      out_rows.store(e, out, Dm);
      if (dmax) {
#pragma unroll
        for (int i = 0; i < NX; ++i) change = fmaxf(change, fabsf((float)gm[i]));
      }
    } else {
      if (dmax) {   // the change from the previous mean held in out_rows
#pragma unroll
        for (int i = 0; i < NX; ++i) change = fmaxf(change, fabsf((float)(gm[i] - old[i])));
      }
      out_rows.store(e, gm, Dm);
    }
#pragma unroll
    for (int i = 0; i < NX; ++i) ok = ok && finite(gm[i]);
    if (j > 0) {
      copy<T, NX>(pm, m);
      copy<T, NX * NX>(pN, N);
      copy<T, NX>(pold, old);
      g = pg;
    }
  }
  if (!ok) flag_status(status, 8);
  if (dmax) {
    // max over the grid of |deviation| = |new - previous nominal mean|, as
    // the bits of a non-negative float (ordered like the values)
    unsigned bits = __float_as_uint(ok ? change : INFINITY);
    const unsigned mask = __activemask();
    bits = __reduce_max_sync(mask, bits);
    if ((int)(threadIdx.x & 31) == __ffs(mask) - 1) atomicMax(dmax, bits);
  }
}

// Per-sequence FP64 sum of the leaf partial log-likelihoods in a fixed
// order (deterministic).  One block per sequence.
__global__ void loglik_reduce(DevSeqs sq, const double* __restrict__ partial,
                              double* __restrict__ loglik, int* status);

}  // namespace sqsm
