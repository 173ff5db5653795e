// Kernels of the reverse pass (see adjoint.cuh) for the CT bearings model.
//
// Per time step s of sequence b: state rows e = s + b (k - 1) and e + 1 (k).
// Buffers (state layout unless noted):
//   nom      nominal trajectory (m, N) the linearisation was taken at,
//   gam      linearised model of the step (absolute form, PRec per step),
//   mf, Nf   filter output, ms, Ns smoother output of that linearisation,
//   dir      direct cotangents (m, P) of the smoother output,
//   dfilt    direct cotangents (m, P) of the filter output (from the RTS VJP),
//   gbar     cotangents of the linearised model (GRec, per step),
//   lam      cotangent of the nominal trajectory (m, lower N),
//   ktab, rtab, stab  per-step KfTab / RtsTab / SlrTab records (written
//            once per evaluation).
#pragma once

#include "adjoint.cuh"

namespace sqsm {

struct AdjBufs {
  const void *mf, *Nf, *ms, *Ns, *nom_m, *nom_N, *y;
  const void* gam;   // linearised model, PRec records
  void *dir, *dfilt, *gbar;
  void *ktab, *rtab, *stab;
};

template <typename T>
SQSM_DEV GammaPacked<T> gview(const AdjBufs& a) {
  return GammaPacked<T>{(T*)a.gam};
}

// --------------------------- per-step tables --------------------------------

// One thread per time step (leaf chunks of `leaf` steps): the KfTab, RtsTab
// and SlrTab records of the step from the final linearisation, its filter
// and smoother output, and the nominal trajectory.
template <typename T>
__global__ void __launch_bounds__(kBlock)
adj_tables_kernel(DevLevel lv, int leaf, const CTParams<T>* __restrict__ Pp, AdjBufs a,
                  bool slr_tab) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ch = tid / leaf;
  if (ch >= lv.n_chunks) return;
  const int j = (int)(tid - ch * leaf);
  if (j >= lv.count[ch]) return;
  constexpr int NX = 5, NY = 2;
  using KT = KfTab<NX, NY>;
  using RT = RtsTab<NX>;
  using ST = SlrTab<NX, NY>;
  const int64_t s = lv.first[ch] + j, e = s + lv.seq[ch];
  {
    Gamma<T, NX, NY> g;
    g.load_all(gview<T>(a), s);
    T ys[NY], mf[NX], Nf[NX * NX], msn[NX], Nsn[NX * NX];
    load<T, NY>((const T*)a.y + s * NY, ys);
    load<T, NX>((const T*)a.mf + e * NX, mf);
    load_lower<T, NX>((const T*)a.Nf + e * NX * NX, Nf);
    load<T, NX>((const T*)a.ms + (e + 1) * NX, msn);
    load_lower<T, NX>((const T*)a.Ns + (e + 1) * NX * NX, Nsn);
    T kt[KT::size], rt[RT::size];
    adj_step_tables<T, NX, NY>(g, ys, mf, Nf, msn, Nsn, kt, rt);
    vstore<T, KT::size>((T*)a.ktab + s * KT::size, kt);
    vstore<T, RT::size>((T*)a.rtab + s * RT::size, rt);
  }
  if (!slr_tab) return;   // the other rules' VJPs recompute their regressions
  const CTParams<T> P = *Pp;
  T st[ST::size];
#pragma unroll
  for (int i = 0; i < ST::size; ++i) st[i] = T(0);
  {
    T m[NX], N[NX * NX];
    load<T, NX>((const T*)a.nom_m + e * NX, m);
    load_lower<T, NX>((const T*)a.nom_N + e * NX * NX, N);
    const Turn<T> tm = turn(m[4], P.dt);
    cubature_fwd<T, NX, true>(m, N, [&](const T* mm_, const T* dl, T* o) { ct_g_delta(P, tm, mm_, dl, o); },
                              st + ST::Gf, st + ST::sf);
  }
  {
    T m[NX], N[NX * NX];
    load<T, NX>((const T*)a.nom_m + (e + 1) * NX, m);
    load_lower<T, NX>((const T*)a.nom_N + (e + 1) * NX * NX, N);
    cubature_fwd<T, NY, false>(m, N, [&](const T* mm_, const T* dl, T* o) { ct_h_delta(P, mm_, dl, o); },
                               st + ST::Gh, st + ST::sh);
  }
  vstore<T, ST::size>((T*)a.stab + s * ST::size, st);
}

// --------------------------- smoother adjoint (forward in time) -----------

template <typename T>
SQSM_DEV void build_smoother_map(const AdjBufs& a, int64_t s, int64_t e, bool first, T* mp) {
  constexpr int NX = 5, X = XRec<NX>::size;
  using RT = RtsTab<NX>;
  T G[RT::head];
  vload<T, RT::head>((const T*)a.rtab + s * RT::size, G);
  smoother_adj_map<T, NX>(G, (const T*)a.dir + (e + 1) * X, mp);
  if (first) {
    T x0[X];
    load<T, X>((const T*)a.dir + e * X, x0);
    map_make_constant<T, NX>(mp, x0);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
adj_smoother_leaf_up(DevLevel lv, DevSeqs sq, AdjBufs a, T* __restrict__ items) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = MapRec<5>::size;
  const int b = lv.seq[c];
  const int64_t s0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t off = sq.offsets[b];
  T agg[REC], mp[REC], tmp[REC];
  build_smoother_map<T>(a, s0, s0 + b, s0 == off, agg);
  for (int j = 1; j < cnt; ++j) {
    const int64_t s = s0 + j;
    build_smoother_map<T>(a, s, s + b, false, mp);
    map_compose<T, 5>(agg, mp, tmp);
    copy<T, REC>(tmp, agg);
  }
  vstore<T, REC>(items + c * REC, agg);
}

// Leaf chunks of `leaf` steps.  per_step: one thread per time step; the
// cotangent entering step j of a chunk is the chunk's carry (or the
// sequence's first direct cotangent) pushed through the maps of steps
// 0 .. j-1 of the chunk, then the RTS VJP of the step (short chunks: the
// replayed maps are cheap next to the VJP).  Otherwise one thread per chunk
// walks its steps in order (long chunks, e.g. one per sequence).
template <typename T>
__global__ void __launch_bounds__(kBlock)
adj_smoother_leaf_down(DevLevel lv, int leaf, bool per_step, DevSeqs sq, AdjBufs a,
                       const T* __restrict__ carry, const int* __restrict__ flag) {
  constexpr int NX = 5, NY = 2, X = XRec<NX>::size, REC = MapRec<NX>::size;
  using GR = GRec<NX, NY>;
  using RT = RtsTab<NX>;
  // FP32 writes the gbar records of a warp's steps through shared memory
  constexpr bool STAGE = sizeof(T) == 4;
  __shared__ T SG[STAGE ? kBlock * GR::size : 1];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = per_step ? tid / leaf : tid;
  const bool in = c < lv.n_chunks;
  const int cnt = in ? lv.count[c] : 0;
  const int jj = per_step ? (int)(tid - c * leaf) : 0;
  const bool active = in && jj < cnt;
  const int b = active ? lv.seq[c] : 0;
  const int64_t s0 = active ? lv.first[c] : 0;
  const int64_t last = active ? sq.offsets[b + 1] - 1 : -1;
  T x[X];
  if (active) {
    if (flag[c]) load<T, X>(carry + c * X, x);
    else load<T, X>((const T*)a.dir + (s0 + b) * X, x);
  }
  // The RTS VJP of step j (the expensive part), writing its record part
  // F | c | Lambda at go, and the map that carries the cotangent from step j
  // to j + 1.
  auto vjp = [&](int j, T* go) {
    const int64_t s = s0 + j, e = s + b;
    const T* rtg = (const T*)a.rtab + s * RT::size;
    Gamma<T, NX, NY> g;
    g.load_transition(gview<T>(a), s);
    T mf[NX];
    load<T, NX>((const T*)a.mf + e * NX, mf);
    T df[X], gb[GR::size];
    // FP32 holds the record in registers; FP64 reads it where it is used
    // (twice the registers per value would spill).
    T rtr[sizeof(T) == 4 ? RT::size : 4];
    if constexpr (sizeof(T) == 4) vload<T, RT::size>(rtg, rtr);
    const T* rt = sizeof(T) == 4 ? rtr : rtg;
    rts_vjp<T, NX, NY>(rt, g.F, mf, x, df, gb);
    store<T, X>((T*)a.dfilt + e * X, df);
    store<T, NX * NX>(go + GR::F, gb + GR::F);
    store<T, NX>(go + GR::c, gb + GR::c);
    store<T, NX * NX>(go + GR::L, gb + GR::L);
  };
  auto advance = [&](int j) {
    const int64_t s = s0 + j, e = s + b;
    T G[RT::head], mp[REC], xn[X];
    vload<T, RT::head>((const T*)a.rtab + s * RT::size, G);
    smoother_adj_map<T, NX>(G, (const T*)a.dir + (e + 1) * X, mp);
    map_apply<T, NX>(mp, x, xn);
    copy<T, X>(xn, x);
    if (s == last) store<T, X>((T*)a.dfilt + (e + 1) * X, x);   // k = n: dmf_n = x_n
  };
  T* gbar = (T*)a.gbar;
  if (!per_step) {   // one thread walks its whole chunk
    if (!active) return;
    for (int j = 0; j < cnt; ++j) {
      vjp(j, gbar + (s0 + j) * GR::size);
      if (j + 1 < cnt || s0 + j == last) advance(j);
    }
    return;
  }
  // One thread per step: every lane first walks the maps before its own
  // step, then all lanes take their VJP together (inside the walk each
  // lane's VJP would come at a different trip and the warp would run it once
  // per distinct step).
  if (active)
    for (int j = 0; j < jj; ++j) advance(j);
  const int64_t s = s0 + jj;
  if constexpr (STAGE) {
    // The steps of a warp's active lanes are consecutive and increase with
    // the lane: their records go out as one block.  The observation part
    // H | d | Omega is written as zeros here; the filter adjoint, which runs
    // next, assigns it.
    const unsigned mask = __ballot_sync(0xffffffffu, active);
    if (mask == 0) return;   // uniform per warp
    const int lane = threadIdx.x % kWarp;
    const int64_t s_lo = __shfl_sync(0xffffffffu, s, __ffs(mask) - 1);
    const int na = __popc(mask);
    T* sh = SG + (threadIdx.x / kWarp) * kWarp * GR::size;
    if (active) {
      T* rec = sh + (int)(s - s_lo) * GR::size;
      vjp(jj, rec);
#pragma unroll
      for (int k = GR::H; k < GR::size; ++k) rec[k] = T(0);
      if (s == last) advance(jj);
    }
    __syncwarp();
    T* gw = gbar + s_lo * GR::size;
    for (int k = lane; k < na * GR::size; k += kWarp) gw[k] = sh[k];
  } else {
    if (active) {
      vjp(jj, gbar + s * GR::size);
      if (s == last) advance(jj);
    }
  }
}

// --------------------------- filter adjoint (backward in time) ------------

template <typename T>
SQSM_DEV void build_filter_map(const AdjBufs& a, int64_t s, int64_t e, bool lastb, T lbar, T* mp) {
  constexpr int NX = 5, NY = 2, X = XRec<NX>::size;
  using KT = KfTab<NX, NY>;
  T h[KT::head];
  vload<T, KT::head>((const T*)a.ktab + s * KT::size, h);
  filter_adj_map<T, NX, NY>(h, lbar, (const T*)a.dfilt + e * X, mp);
  if (lastb) {
    T xn[X];
    load<T, X>((const T*)a.dfilt + (e + 1) * X, xn);
    map_make_constant<T, NX>(mp, xn);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
adj_filter_leaf_up(DevLevel lv, DevSeqs sq, AdjBufs a, T lbar, T* __restrict__ items) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = MapRec<5>::size;
  const int b = lv.seq[c];
  const int64_t s0 = lv.first[c];
  const int cnt = lv.count[c];
  const int64_t last = sq.offsets[b + 1] - 1;
  T agg[REC], mp[REC], tmp[REC];
  build_filter_map<T>(a, s0 + cnt - 1, s0 + cnt - 1 + b, s0 + cnt - 1 == last, lbar, agg);
  for (int j = cnt - 2; j >= 0; --j) {
    const int64_t s = s0 + j;
    build_filter_map<T>(a, s, s + b, false, lbar, mp);
    map_compose<T, 5>(agg, mp, tmp);
    copy<T, REC>(tmp, agg);
  }
  vstore<T, REC>(items + c * REC, agg);
}

// Leaf chunks of `leaf` steps, walked backward in time.  per_step: one
// thread per time step; the cotangent entering step j of a chunk (of its
// output row) is the chunk's carry (or the sequence's last filter
// cotangent) pushed back through the maps of steps cnt-1 .. j+1, then the
// Kalman-step VJP of the step.  Otherwise one thread per chunk walks its
// steps from the last.
template <typename T>
__global__ void __launch_bounds__(kBlock)
adj_filter_leaf_down(DevLevel lv, int leaf, bool per_step, DevSeqs sq, AdjBufs a, T lbar,
                     const T* __restrict__ carry, const int* __restrict__ flag) {
  constexpr int NX = 5, NY = 2, X = XRec<NX>::size, REC = MapRec<NX>::size;
  using GR = GRec<NX, NY>;
  using KT = KfTab<NX, NY>;
  // FP32 moves the gbar records of a warp's steps through shared memory
  // (FP64 records would not fit beside the block's other data)
  constexpr bool STAGE = sizeof(T) == 4;
  __shared__ T SG[STAGE ? kBlock * GR::size : 1];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = per_step ? tid / leaf : tid;
  const bool in = c < lv.n_chunks;
  const int cnt = in ? lv.count[c] : 0;
  const int jj = per_step ? (int)(tid - c * leaf) : 0;
  const bool active = in && jj < cnt;
  const int b = active ? lv.seq[c] : 0;
  const int64_t s0 = active ? lv.first[c] : 0;
  T x[X];
  if (active) {
    if (flag[c]) load<T, X>(carry + c * X, x);
    else load<T, X>((const T*)a.dfilt + (s0 + cnt - 1 + b + 1) * X, x);
  }
  // The Kalman-step VJP of step j on the record at go and the map that
  // carries the cotangent from step j to j - 1.
  auto vjp = [&](int j, T* go) {
    const int64_t s = s0 + j, e = s + b;
    Gamma<T, NX, NY> g;
    g.load_all(gview<T>(a), s);
    T kt[KT::size], mprev[NX];
    vload<T, KT::size>((const T*)a.ktab + s * KT::size, kt);
    load<T, NX>((const T*)a.mf + e * NX, mprev);
    KfQ<T, NX, NY> q;
    q.load(kt);
    T gb[GR::size];
    load<T, GR::size>(go, gb);
    kf_vjp<T, NX, NY>(q, g, mprev, lbar, x, gb);
    store<T, GR::size>(go, gb);
  };
  auto advance = [&](int j) {
    const int64_t s = s0 + j, e = s + b;
    T h[KT::head], mp[REC], xn[X];
    vload<T, KT::head>((const T*)a.ktab + s * KT::size, h);
    filter_adj_map<T, NX, NY>(h, lbar, (const T*)a.dfilt + e * X, mp);
    map_apply<T, NX>(mp, x, xn);
    copy<T, X>(xn, x);
  };
  T* gbar = (T*)a.gbar;
  if (!per_step) {   // one thread walks its whole chunk
    if (!active) return;
    for (int j = cnt - 1; j >= 0; --j) {
      vjp(j, gbar + (s0 + j) * GR::size);
      if (j > 0) advance(j);
    }
    return;
  }
  // One thread per step: the lanes walk their maps first and take their VJPs
  // together (as in adj_smoother_leaf_down).
  if (active)
    for (int j = cnt - 1; j > jj; --j) advance(j);
  const int64_t s = s0 + jj;
  if constexpr (STAGE) {
    // The steps of a warp's active lanes are consecutive and increase with
    // the lane (chunks of consecutive steps; only a sequence's last chunk is
    // short): their records are read and written as one block.
    const unsigned mask = __ballot_sync(0xffffffffu, active);
    if (mask == 0) return;   // uniform per warp
    const int lane = threadIdx.x % kWarp;
    const int64_t s_lo = __shfl_sync(0xffffffffu, s, __ffs(mask) - 1);
    const int na = __popc(mask);
    T* sh = SG + (threadIdx.x / kWarp) * kWarp * GR::size;
    T* gw = gbar + s_lo * GR::size;
    for (int k = lane; k < na * GR::size; k += kWarp) sh[k] = gw[k];
    __syncwarp();
    if (active) vjp(jj, sh + (int)(s - s_lo) * GR::size);
    __syncwarp();
    for (int k = lane; k < na * GR::size; k += kWarp) gw[k] = sh[k];
  } else {
    if (active) vjp(jj, gbar + s * GR::size);
  }
}

// --------------------------- upper levels (both directions) ---------------

template <typename T, bool FWD>
__global__ void __launch_bounds__(kBlock)
adj_up(DevLevel lv, const T* __restrict__ in, T* __restrict__ out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = MapRec<5>::size;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  T agg[REC], mp[REC], tmp[REC];
  vload<T, REC>(in + (FWD ? i0 : i0 + cnt - 1) * REC, agg);
  for (int j = 1; j < cnt; ++j) {
    vload<T, REC>(in + (FWD ? i0 + j : i0 + cnt - 1 - j) * REC, mp);
    map_compose<T, 5>(agg, mp, tmp);
    copy<T, REC>(tmp, agg);
  }
  vstore<T, REC>(out + c * REC, agg);
}

// carry = the cotangent vector entering the chunk (forward: before its
// first item; backward: after its last); flag 0: none, the chunk holds the
// constant boundary map.
template <typename T, bool FWD>
__global__ void __launch_bounds__(kBlock)
adj_down(DevLevel lv, const T* __restrict__ items, const T* __restrict__ cin,
         const int* __restrict__ fin, T* __restrict__ cout, int* __restrict__ fout) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= lv.n_chunks) return;
  constexpr int REC = MapRec<5>::size, X = XRec<5>::size;
  const int64_t i0 = lv.first[c];
  const int cnt = lv.count[c];
  int flag = fin[c];
  T x[X];
  load<T, X>(cin + c * X, x);
  if (!flag) {
#pragma unroll
    for (int i = 0; i < X; ++i) x[i] = T(0);
  }
  for (int j = 0; j < cnt; ++j) {
    const int64_t i = FWD ? i0 + j : i0 + cnt - 1 - j;
    store<T, X>(cout + i * X, x);
    fout[i] = flag;
    if (j + 1 < cnt) {
      T mp[REC], xn[X];
      vload<T, REC>(items + i * REC, mp);
      map_apply<T, 5>(mp, x, xn);
      copy<T, X>(xn, x);
      flag = 1;
    }
  }
}

// Chunk-scan variant of an upper level: one warp per chunk of at most 32
// maps computes, in place, the composition of the chunk's maps from its
// first (in scan order) through each item, and writes the chunk's total.
template <typename T, bool FWD>
__global__ void __launch_bounds__(kChunkScan)
adj_up_cs(DevLevel lv, T* __restrict__ items, T* __restrict__ out) {
  constexpr int REC = MapRec<5>::size;
  __shared__ __align__(16) T S[kChunkScan * REC];
  const int64_t c = blockIdx.x;
  const int t = threadIdx.x;   // position in scan order
  const int cnt = lv.count[c];
  const int64_t i = lv.first[c] + (FWD ? t : cnt - 1 - t);
  T mine[REC], tmp[REC];
  if (t < cnt) vload<T, REC>(items + i * REC, mine);
  for (int d = 1; d < cnt; d <<= 1) {
    if (t < cnt) vstore<T, REC>(S + t * REC, mine);
    __syncwarp();
    if (t < cnt && t >= d) {
      map_compose<T, 5>(S + (t - d) * REC, mine, tmp);
      copy<T, REC>(tmp, mine);
    }
    __syncwarp();
  }
  if (t < cnt) vstore<T, REC>(items + i * REC, mine);
  if (t == cnt - 1) vstore<T, REC>(out + c * REC, mine);
}

// One thread per item of a chunk-scanned level: the cotangent entering item
// i is the chunk's carry pushed through the composed maps of the items
// before i (in scan order).
template <typename T, bool FWD>
__global__ void __launch_bounds__(kBlock)
adj_down_cs(DevLevel lv, const T* __restrict__ items, const T* __restrict__ cin,
            const int* __restrict__ fin, T* __restrict__ cout, int* __restrict__ fout) {
  constexpr int REC = MapRec<5>::size, X = XRec<5>::size;
  static_assert(kChunkScan == kWarp && kBlock % kWarp == 0, "one chunk per warp");
  __shared__ T SO[kBlock / kWarp][kWarp * X];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = tid / kChunkScan;
  if (c >= lv.n_chunks) return;   // uniform per warp
  const int j = (int)(tid - c * kChunkScan);
  const int cnt = lv.count[c];
  const bool active = j < cnt;
  const int64_t i0 = lv.first[c];
  const int64_t i = i0 + j;
  const bool head = FWD ? j == 0 : j == cnt - 1;
  const int flag = fin[c];
  T x[X];
  load<T, X>(cin + c * X, x);
  if (!flag) {
#pragma unroll
    for (int k = 0; k < X; ++k) x[k] = T(0);
  }
  if (active && !head) {
    T mp[REC], xn[X];
    vload<T, REC>(items + (FWD ? i - 1 : i + 1) * REC, mp);
    map_apply<T, 5>(mp, x, xn);
    copy<T, X>(xn, x);
  }
  // the chunk's items are consecutive: their rows go out as one block
  warp_store_rows<T, X>(cout + i0 * X, SO[threadIdx.x / kWarp], x, j, cnt, active);
  if (active) fout[i] = head ? flag : 1;
}

// Top of an adjoint scan: one block per sequence scans the sequence's items
// of the level (at most KS of them, in scan order) with Kogge-Stone in
// shared memory.  The first item in scan order holds the constant boundary
// map (flag 0), so every prefix is a constant map and the cotangent
// entering item t is the constant part (s, S) of the composition of the
// items before it.
template <typename T, bool FWD>
__global__ void __launch_bounds__((KsMax<T, MapRec<5>::size>::value))
adj_top_ks(const int64_t* __restrict__ seq_item_off, const T* __restrict__ items,
           T* __restrict__ carry_out, int* __restrict__ flag_out) {
  constexpr int REC = MapRec<5>::size, KS = KsMax<T, REC>::value, X = XRec<5>::size;
  using R = MapRec<5>;
  __shared__ __align__(16) T S[KS * REC];
  const int b = blockIdx.x, t = threadIdx.x;
  const int64_t i0 = seq_item_off[b];
  const int c = (int)(seq_item_off[b + 1] - i0);
  const int64_t i = i0 + (FWD ? t : c - 1 - t);
  T mine[REC], tmp[REC];
  if (t < c) vload<T, REC>(items + i * REC, mine);
  for (int d = 1; d < c; d <<= 1) {
    if (t < c) vstore<T, REC>(S + t * REC, mine);
    __syncthreads();
    if (t < c && t >= d) {
      map_compose<T, 5>(S + (t - d) * REC, mine, tmp);
      copy<T, REC>(tmp, mine);
    }
    __syncthreads();
  }
  if (t < c) vstore<T, REC>(S + t * REC, mine);
  __syncthreads();
  if (t < c) {
    if (t > 0) {
      const T* p = S + (t - 1) * REC;
      T* co = carry_out + i * X;
#pragma unroll
      for (int k = 0; k < 5; ++k) co[k] = p[R::s + k];
#pragma unroll
      for (int k = 0; k < 25; ++k) co[5 + k] = p[R::S + k];
    }
    flag_out[i] = t > 0 ? 1 : 0;
  }
}

// --------------------------- SLR VJP and reductions ------------------------

// Nominal-trajectory cotangent lam of state row e of sequence b from the
// transition regression of step k (k < n) and the observation regression of
// step k - 1 (k >= 1), the row's theta partials added to th, and the direct
// cotangents of the row that the next iteration starts from (step 1 applied
// to lam); the regressions' forward quantities come from the SlrTab records.
// LIN: 0 cubature (forward quantities from the SlrTab records), 1 Taylor,
// 2 unscented, 3 Gauss-Hermite (recomputed from the nominal rows).
template <typename T, int LIN = 0>
SQSM_DEV void adj_slr_row(int64_t e, int b, const DevSeqs& sq, const CTParams<T>* __restrict__ Pp,
                          const AdjBufs& a, T* o, T* d, double* th) {
  constexpr int NX = 5, NY = 2;
  using GR = GRec<NX, NY>;
  using ST = SlrTab<NX, NY>;
  const CTParams<T> P = *Pp;
  const int64_t k = e - (sq.offsets[b] + b);
  const int64_t nb = sq.offsets[b + 1] - sq.offsets[b];
  T m[NX], N[NX * NX], mb[NX], Nb[NX * NX];
  load<T, NX>((const T*)a.nom_m + e * NX, m);
  load_lower<T, NX>((const T*)a.nom_N + e * NX * NX, N);
#pragma unroll
  for (int i = 0; i < NX; ++i) mb[i] = T(0);
#pragma unroll
  for (int i = 0; i < NX * NX; ++i) Nb[i] = T(0);
  if (k < nb) {
    const int64_t s = sq.offsets[b] + k;
    const T* gb = (const T*)a.gbar + s * GR::size;
    T Lb[NX * NX];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int q = 0; q < NX; ++q) Lb[i * NX + q] = T(0.5) * (gb[GR::L + i * NX + q] + gb[GR::L + q * NX + i]);
    auto jf = [&](const T* xx, T* J) { ct_jac_f(P, xx, J); };
    if constexpr (LIN == 0) {
      T t[ST::obs];
      vload<T, ST::obs>((const T*)a.stab + s * ST::size, t);
      cubature_vjp<T, NX>(m, N, t + ST::Gf, t + ST::sf, gb + GR::F, gb + GR::c, Lb, jf, mb, Nb);
    } else if constexpr (LIN == 1) {
      taylor_vjp<T, NX>(m, gb + GR::F, gb + GR::c,
                        [&](const T* xx, const T* Jb, T* o) { ct_jac_f_vjp(P, xx, Jb, o); }, mb);
    } else {
      const Turn<T> tm = turn(m[4], P.dt);
      sigma_vjp<T, NX, LIN == 2 ? 1 : 2, true>(
          m, N, [&](const T* mm_, const T* dl, T* o) { ct_g_delta(P, tm, mm_, dl, o); }, jf,
          gb + GR::F, gb + GR::c, Lb, mb, Nb);
    }
    // Q = q_c Q_c + q_w Q_w (Q_w only at (4, 4)): d/d log q_c = Lambda-bar :
    // (Q - Q_44 e_4 e_4^T), d/d log q_w = Lambda-bar_44 Q_44
    T Q[NX * NX];
    gram_lower<T, NX>(P.SQ, Q);
    double tq = 0.0;
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) tq += (double)Lb[i] * (double)Q[i];
    const double t44 = (double)Lb[24] * (double)Q[24];
    th[1] += tq - t44;
    th[2] += t44;
  }
  if (k >= 1) {
    const int64_t s = sq.offsets[b] + k - 1;
    const T* gb = (const T*)a.gbar + s * GR::size;
    T Lb[NY * NY];
#pragma unroll
    for (int i = 0; i < NY; ++i)
#pragma unroll
      for (int q = 0; q < NY; ++q) Lb[i * NY + q] = T(0.5) * (gb[GR::O + i * NY + q] + gb[GR::O + q * NY + i]);
    auto jh = [&](const T* xx, T* J) { ct_jac_h(P, xx, J); };
    if constexpr (LIN == 0) {
      T t[ST::size - ST::obs];
      vload<T, ST::size - ST::obs>((const T*)a.stab + s * ST::size + ST::obs, t);
      cubature_vjp<T, NY>(m, N, t + (ST::Gh - ST::obs), t + (ST::sh - ST::obs), gb + GR::H,
                          gb + GR::d, Lb, jh, mb, Nb);
    } else if constexpr (LIN == 1) {
      taylor_vjp<T, NY>(m, gb + GR::H, gb + GR::d,
                        [&](const T* xx, const T* Jb, T* o) { ct_jac_h_vjp(P, xx, Jb, o); }, mb);
    } else {
      sigma_vjp<T, NY, LIN == 2 ? 1 : 2, false>(
          m, N, [&](const T* mm_, const T* dl, T* o) { ct_h_delta(P, mm_, dl, o); }, jh,
          gb + GR::H, gb + GR::d, Lb, mb, Nb);
    }
    // Omega = diag(sigma_1^2, sigma_2^2): d/d log sigma_i = 2 sigma_i^2 Omega-bar_ii
    th[0] += 2.0 * (double)P.sigma[0] * (double)P.sigma[0] * (double)Lb[0];
    th[3] += 2.0 * (double)P.sigma[1] * (double)P.sigma[1] * (double)Lb[3];
  }
#pragma unroll
  for (int i = 0; i < NX; ++i) o[i] = mb[i];
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int q = 0; q < NX; ++q) o[NX + r * NX + q] = q <= r ? Nb[r * NX + q] : T(0);
  // the next iteration's direct cotangents of this row (step 1)
  T L[NX * NX];
  load_lower<T, NX>((const T*)a.Ns + e * NX * NX, L);
  direct_row<T, NX>(L, o, d);
}

// Sum of four values over the block (kBlock threads) in a fixed order,
// written by thread 0 to out[0..3].
SQSM_DEV void block_sum4(double* v, double* __restrict__ out) {
  __shared__ double part[kBlock / 32][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) part[w][j] = v[j];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < kBlock / 32; ++q) t += part[q][j];
      out[j] = t;
    }
}

// One thread per state row (smoother leaf chunks of `leaf` rows); every
// thread of the block takes part in the block's theta sums (rows past the
// end add zero), written to th_partial[4 * block]: log sigma_1, log q_c,
// log q_w, log sigma_2.
template <typename T, int LIN = 0>
__global__ void __launch_bounds__(kBlock)
adj_slr_kernel(DevLevel lv, int leaf, DevSeqs sq, const CTParams<T>* __restrict__ Pp, AdjBufs a,
               T* __restrict__ lam_out, double* __restrict__ th_partial) {
  constexpr int X = XRec<5>::size;
  __shared__ T SO[kBlock / kWarp][kWarp * X];
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ch = tid / leaf;
  const int jr = (int)(tid - ch * leaf);
  double th[4] = {0.0, 0.0, 0.0, 0.0};
  const bool active = ch < lv.n_chunks && jr < lv.count[ch];
  const int64_t e = active ? lv.first[ch] + jr : 0;
  T o[X], d[X];
  if (active) adj_slr_row<T, LIN>(e, lv.seq[ch], sq, Pp, a, o, d, th);
  // The rows of a warp's active lanes are consecutive and increase with the
  // lane (chunks of consecutive rows; only a sequence's last chunk is
  // short): the two rows of each lane go out as two blocks through shared
  // memory, every store instruction covering consecutive words.
  const unsigned mask = __ballot_sync(0xffffffffu, active);
  if (mask) {
    const int64_t e_lo = __shfl_sync(0xffffffffu, e, __ffs(mask) - 1);
    const int na = __popc(mask), r = active ? (int)(e - e_lo) : 0;
    T* sh = SO[threadIdx.x / kWarp];
    warp_store_rows<T, X>(lam_out + e_lo * X, sh, o, r, na, active);
    __syncwarp();
    warp_store_rows<T, X>((T*)a.dir + e_lo * X, sh, d, r, na, active);
  }
  block_sum4(th, th_partial + 4 * blockIdx.x);
}

// Fixed-order sums of the theta partials (one block over n four-entry
// partials): with n_theta = 4, out[j] = sign * sum of entry j; with 3 (one
// noise level for both sensors), out[0] sums entries 0 and 3.
static __global__ void adj_theta_reduce(int64_t n, const double* __restrict__ part, double sign,
                                        int n_theta, double* __restrict__ out) {
  __shared__ double buf[4][256];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
    for (int j = 0; j < 4; ++j) acc[j] += part[i * 4 + j];
  for (int j = 0; j < 4; ++j) buf[j][threadIdx.x] = acc[j];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int j = 0; j < 4; ++j) buf[j][threadIdx.x] += buf[j][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (n_theta == 4) {
      for (int j = 0; j < 4; ++j) out[j] = sign * buf[j][0];
    } else {
      out[0] = sign * (buf[0][0] + buf[3][0]);
      out[1] = sign * buf[1][0];
      out[2] = sign * buf[2][0];
    }
  }
}

// Relative max-norm change between two cotangent iterates, in two kernels:
// every block max-reduces |a - b| and |a| over a grid-stride slice and folds
// them into words[0], words[1] (bits of non-negative floats, ordered like
// the values; the caller clears them), then one thread forms the ratio.
template <typename T>
static __global__ void __launch_bounds__(256)
adj_change_partial(int64_t n, const T* __restrict__ a, const T* __restrict__ b,
                   unsigned* __restrict__ words) {
  float d = 0.f, m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    // a NaN counts as an infinite change (fmaxf alone would drop it)
    const float di = fabsf((float)(a[i] - b[i])), mi = fabsf((float)a[i]);
    d = di == di ? fmaxf(d, di) : INFINITY;
    m = mi == mi ? fmaxf(m, mi) : INFINITY;
  }
  unsigned bd = __float_as_uint(d), bm = __float_as_uint(m);
  bd = __reduce_max_sync(0xffffffffu, bd);
  bm = __reduce_max_sync(0xffffffffu, bm);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(words, bd);
    atomicMax(words + 1, bm);
  }
}

// Relative changes of lambda (words 0, 1; 0 without adjoint iterations) and
// of the trajectory (words 2, 3) into the optional outputs; with tol > 0 a
// change >= tol or not finite sets SQSM_ERR_NOT_CONVERGED (128).
static __global__ void adj_settle_check(const unsigned* __restrict__ words, int have_adj,
                                        double tol, double* __restrict__ adj_change,
                                        double* __restrict__ ipls_change, int* status) {
  const double da = __uint_as_float(words[0]), ma = __uint_as_float(words[1]);
  const double di = __uint_as_float(words[2]), mi = __uint_as_float(words[3]);
  const double ra = have_adj ? (ma > 0.0 ? da / ma : da) : 0.0;
  const double ri = mi > 0.0 ? di / mi : di;
  if (adj_change) adj_change[0] = ra;
  if (ipls_change) ipls_change[0] = ri;
  if (tol > 0.0 && status && !(ra < tol && ri < tol)) atomicOr(status, 128);
}

// Sum of the per-sequence log-likelihoods times sign (one thread, fixed order).
static __global__ void adj_nll_kernel(int B, const double* __restrict__ ll, double sign,
                                      double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += ll[b];
  out[0] = sign * s;
}

}  // namespace sqsm
