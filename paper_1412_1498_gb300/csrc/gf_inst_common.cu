// gf_inst_common.cu -- the finishing reduction and the element kernels (all storages).
#include "gf_kernels.cuh"

namespace gf {

// One block per unit adds the unit's tile partials, kept as pairs (hi, lo) of floats,
// with FP32 instructions only (FP64 issues at ~1/64 of the FP32 rate here): each thread
// sums a fixed stride of tiles, then a fixed binary tree in shared memory.  Thread 0
// finishes the unit; the loop state is updated by the block itself when there is one
// unit, else by the last block to take a ticket.  Every addition has a fixed order:
// deterministic.
//
// Modes.  MEASURE / RESET (outside the loop): F and theta of every unit from the two
// parity passes; RESET also sets the masks.  In the loop a check sweep runs ODD after
// the odd half-sweep, which measured F and the odd-site part of theta: theta >= the
// odd part (every Tr[Delta Delta^+] >= 0), so a unit whose odd part is already >= eps
// continues, exactly as the full theta would decide; the others (and every unit on the
// last sweep of the budget) are pending.  With nothing pending ODD also does the
// sweep's bookkeeping and closes it; otherwise the even-site pass runs for the pending
// units and LOOP completes their theta and masks, counts the sweep and updates the
// loop state.  OPEN is the opening check of a phase in the same manner: after the
// odd-site pass alone it starts every unit whose odd part is >= its threshold; if some
// unit is undecided it leaves the loop state open (hold, need_exact = 2), and the gated
// even-site pass and a gated RESET then measure every unit as RESET does.
//
// One history record: the sweep number, then F and theta of every lattice (lattice totals
// already written); by one thread.
__device__ __forceinline__ void history_record(const FinishArgs& a, int sweep_no) {
  const int n = a.st->hist_n;
  if (n >= a.hist_cap) return;
  double* r = a.hist + (size_t)n * (1 + 2 * a.n_lat);
  r[0] = (double)sweep_no;
  for (int l = 0; l < a.n_lat; ++l) {
    r[1 + 2 * l] = __ldcg(a.lat_F + l);
    r[2 + 2 * l] = __ldcg(a.lat_theta + l);
  }
  a.st->hist_n = n + 1;
}

__global__ void __launch_bounds__(kFinishThreads) k_finish(FinishArgs a) {
  __shared__ float2 red[3][kFinishThreads];
  __shared__ int s_last;
  __shared__ int s_cnt[kFinishThreads / 32];
  grid_dep_wait();
  grid_dep_launch();
  const int tid = (int)threadIdx.x;
  const int u = (int)blockIdx.x;
  const bool loop = a.mode == FINISH_LOOP || a.mode == FINISH_ODD;
  // Every load that does not depend on another one is issued here, together: the
  // kernel is short and its time is mostly dependent round trips to memory.
  const int n_active = a.st->n_active, sweep = a.st->sweep, limit = a.st->limit;
  const int ci = a.st->check_interval, closed = a.st->sweep_closed, hold = a.st->hold;
  const int need_in = a.st->need_exact;
  const double eps = a.st->eps, eps_mid = a.st->eps_mid;
  const int final_level = a.st->final_level;
  const int lvl_in = a.active[u];  // > 0: sweeping at that precision level
  const bool was_active = lvl_in > 0;
  const bool pend_in = a.pending[u] != 0;
  const int tb = a.n_units == 1 ? 0 : a.unit_tiles[u];
  const int te = a.n_units == 1 ? (a.mode == FINISH_ODD ? a.n_odd_parts : a.n_tiles) : a.unit_tiles[u + 1];
  // The first pass of tile partials: with one unit its range is a kernel argument, so
  // these loads wait for nothing and travel with the ones above.  (FINISH_LOOP, which
  // mostly has nothing to add, loads inside the reduction.)
  const bool outside = a.mode == FINISH_MEASURE || a.mode == FINISH_RESET || a.mode == FINISH_ENTER;
  const bool early = a.mode != FINISH_LOOP;
  const float2* p1 = (a.mode == FINISH_ODD || a.mode == FINISH_OPEN) ? a.part_th_odd : a.part_th_even;
  float2 x0[kFinishUnroll], x1[kFinishUnroll], x2[kFinishUnroll];
#pragma unroll
  for (int j = 0; j < kFinishUnroll; ++j) {
    const int i = tb + tid + j * kFinishThreads;
    const bool in = early && i < te;
    x0[j] = in ? a.part_F[i] : make_float2(0.f, 0.f);
    x1[j] = in ? p1[i] : make_float2(0.f, 0.f);
    x2[j] = in && outside ? a.part_th_odd[i] : make_float2(0.f, 0.f);
  }
  // what thread 0 needs after the reduction
  double invF = 0.0, invT = 0.0, uF_old = 0.0, uT_old = 0.0, uTo = 0.0;
  if (tid == 0) {
    invF = a.unit_norm[2 * u];
    invT = a.unit_norm[2 * u + 1];
    uF_old = a.unit_sumF[u];
    uT_old = a.unit_sumTh[u];
    uTo = a.unit_sumTh_odd[u];
  }
  bool check = true;
  if (loop) {
    if (!(n_active > 0 && sweep < limit)) return;  // uniform over the grid: no ticket taken
    if (a.mode == FINISH_ODD && hold) return;        // the previous sweep is still open
    check = ((sweep + 1) % ci) == 0 || sweep + 1 == limit;  // state_check_sweep
    // the loop finish serves an open sweep only (written by the odd-part finish), so a
    // second one after the sweep was resolved does nothing
    if (a.mode == FINISH_LOOP && (closed || !hold)) return;
  }
  if (a.gated && !(hold && need_in == 2)) return;  // the opening check decided every unit
  bool reduce;
  // a sweep without a check is closed by the odd-part finish (counts, no sums)
  if (a.mode == FINISH_ODD) reduce = was_active && check;
  else if (a.mode == FINISH_LOOP) reduce = check && was_active && pend_in;
  else if (a.mode == FINISH_ENTER) reduce = pend_in;
  else reduce = true;
  if (reduce) {
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0, acc2 = acc0;
    // kFinishUnroll tiles per thread and pass, all loads of a pass in flight together,
    // added as a fixed binary tree
    for (int i0 = tb + tid; i0 < te; i0 += kFinishUnroll * kFinishThreads) {
      if (i0 != tb + tid || !early) {
#pragma unroll
        for (int j = 0; j < kFinishUnroll; ++j) {
          const int i = i0 + j * kFinishThreads;
          const bool in = i < te;
          x0[j] = in && a.mode != FINISH_LOOP ? a.part_F[i] : make_float2(0.f, 0.f);
          x1[j] = in ? p1[i] : make_float2(0.f, 0.f);
          x2[j] = in && outside ? a.part_th_odd[i] : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int w = kFinishUnroll / 2; w > 0; w >>= 1)
#pragma unroll
        for (int j = 0; j < w; ++j) {
          x0[j] = pair_add(x0[j], x0[j + w]);
          x1[j] = pair_add(x1[j], x1[j + w]);
          x2[j] = pair_add(x2[j], x2[j + w]);
        }
      acc0 = pair_add(acc0, x0[0]);
      acc1 = pair_add(acc1, x1[0]);
      acc2 = pair_add(acc2, x2[0]);
    }
    red[0][tid] = acc0;
    red[1][tid] = acc1;
    red[2][tid] = acc2;
    __syncthreads();
#pragma unroll
    for (int w = kFinishThreads / 2; w > 0; w >>= 1) {
      if (tid < w) {
        red[0][tid] = pair_add(red[0][tid], red[0][tid + w]);
        red[1][tid] = pair_add(red[1][tid], red[1][tid + w]);
        red[2][tid] = pair_add(red[2][tid], red[2][tid + w]);
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    const bool forced = loop && sweep + 1 == limit;  // last sweep of the budget: measure exactly
    const double s0 = reduce ? pair_value(red[0][0]) : 0.0;
    const double s1 = reduce ? pair_value(red[1][0]) : 0.0;
    const double s2 = reduce ? pair_value(red[2][0]) : 0.0;
    double uF = uF_old, uT = uT_old;
    int pend = 0;
    bool act = was_active;
    // the unit's precision level (a reset starts every unit at level 1) and its threshold
    const int lvl = (a.mode == FINISH_RESET || a.mode == FINISH_OPEN) ? 1 : lvl_in;
    const double thr = (lvl == 1 && final_level > 1) ? eps_mid : eps;
    if (a.mode == FINISH_OPEN) {
      // F and the odd-site part of theta (kept until a check replaces them); the unit
      // sweeps if that part alone reaches the threshold, otherwise it is undecided
      a.unit_sumF[u] = s0;
      a.unit_F[u] = s0 * invF;
      a.unit_sumTh[u] = s1;
      a.unit_theta[u] = s1 * invT;
      pend = a.hist != nullptr || !(s1 * invT >= thr);  // a history wants the opening theta
      a.pending[u] = pend ? 1 : 0;
      if (!pend) a.active[u] = 1;
    } else if (a.mode == FINISH_ODD) {
      if (reduce) {
        uF = s0;
        a.unit_sumF[u] = s0;
        a.unit_F[u] = s0 * invF;
        a.unit_sumTh_odd[u] = s1;
        pend = forced || a.hist != nullptr || !(s1 * invT >= thr);  // a history wants every theta
      }
      a.pending[u] = pend ? lvl : 0;  // the even-site pass of this level serves the unit
    } else {
      if (reduce) {
        uT = a.mode == FINISH_LOOP ? s1 + uTo : s1 + s2;
        a.unit_sumTh[u] = uT;
        a.unit_theta[u] = uT * invT;
        if (a.mode != FINISH_LOOP) {
          uF = s0;
          a.unit_sumF[u] = s0;
          a.unit_F[u] = s0 * invF;
        }
        if (a.mode != FINISH_MEASURE) {
          act = uT * invT >= thr;
          a.active[u] = act ? lvl : (lvl >= final_level ? 0 : -lvl);
        }
        if (a.mode == FINISH_ENTER) a.pending[u] = 0;
      }
      if (a.mode == FINISH_LOOP && was_active) a.iters[u] += 1;
    }
    if (a.n_units == 1) {
      // one unit is one Landau lattice: the loop state follows from this thread's values
      // (the same totals and counts as the general path below, without re-reading them)
      if (a.mode == FINISH_ODD && pend) {
        a.st->need_exact = 1;
        a.st->sweep_closed = 0;
        a.st->hold = 1;
      } else if (a.mode == FINISH_OPEN) {
        if (pend) {
          a.st->need_exact = 2;
          a.st->hold = 1;
        } else {
          a.st->n_active = 1;
        }
      } else {
        if (a.mode == FINISH_ODD && was_active) a.iters[u] += 1;
        if (!loop || check) {
          a.lat_F[0] = uF * invF;
          a.lat_theta[0] = uT * invT;
        }
        if (a.mode == FINISH_ODD) {
          a.st->need_exact = 0;
          a.st->sweep_closed = 1;
        } else if (a.mode != FINISH_MEASURE) {
          a.st->n_active = act ? 1 : 0;
        }
        if (a.mode == FINISH_LOOP) a.st->hold = 0;
        if (a.gated) {
          a.st->hold = 0;
          a.st->need_exact = 0;
        }
        if (loop) a.st->sweep = sweep + 1;
        if (a.hist && ((a.mode == FINISH_LOOP && check) || (a.mode == FINISH_RESET && a.st->hist_n == 0)))
          history_record(a, a.mode == FINISH_LOOP ? a.st->hist_base + sweep + 1 : 0);
      }
      a.st->ticket = 0u;
      s_last = 0;
    } else {
      __threadfence();
      s_last = atomicAdd(&a.st->ticket, 1u) == (unsigned int)(a.n_units - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the loop state: counts, lattice totals in a fixed order
  int cnt = 0;  // ODD, OPEN: pending units; otherwise: active units
  for (int v = tid; v < a.n_units; v += blockDim.x)
    cnt += (a.mode == FINISH_ODD || a.mode == FINISH_OPEN) ? (__ldcg(a.pending + v) != 0)
                                                           : (__ldcg(a.active + v) > 0);
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((tid & 31) == 0) s_cnt[tid >> 5] = cnt;
  __syncthreads();
  int n = 0;
  for (int w = 0; w < kFinishThreads / 32; ++w) n += s_cnt[w];
  if (a.mode == FINISH_ODD && n > 0) {
    if (tid == 0) {
      a.st->need_exact = 1;
      a.st->sweep_closed = 0;
      a.st->hold = 1;
      a.st->ticket = 0u;
    }
    return;
  }
  if (a.mode == FINISH_OPEN) {  // undecided units wait for the gated reset; else all sweep
    if (tid == 0) {
      if (n > 0) {
        a.st->need_exact = 2;
        a.st->hold = 1;
      } else {
        a.st->n_active = a.n_units;
      }
      a.st->ticket = 0u;
    }
    return;
  }
  if (a.mode == FINISH_ODD)  // nothing pending: every active unit continues; close the sweep
    for (int v = tid; v < a.n_units; v += blockDim.x)
      if (__ldcg(a.active + v) > 0) a.iters[v] += 1;
  if (!loop || check) {
    for (int l = tid; l < a.n_lat; l += blockDim.x) {
      const LatDev lat = a.lats[l];
      double sF = 0.0, sTh = 0.0;
      for (int k = 0; k < lat.n_units; ++k) {
        sF += __ldcg(a.unit_sumF + lat.unit0 + k);
        sTh += __ldcg(a.unit_sumTh + lat.unit0 + k);
      }
      // the reciprocals as the host forms the per-unit ones (same bits for one-unit lattices)
      a.lat_F[l] = sF * (1.0 / ((double)a.nd * 3.0 * (double)lat.V));
      a.lat_theta[l] = sTh * (1.0 / (3.0 * (double)lat.V));
    }
  }
  __syncthreads();  // lattice totals written by other threads of this block
  if (tid == 0) {
    if (a.mode == FINISH_ODD) {
      a.st->need_exact = 0;
      a.st->sweep_closed = 1;
    } else if (a.mode != FINISH_MEASURE) {
      a.st->n_active = n;
    }
    if (a.mode == FINISH_LOOP) a.st->hold = 0;
    if (a.gated) {
      a.st->hold = 0;
      a.st->need_exact = 0;
    }
    if (a.hist && ((a.mode == FINISH_LOOP && check) || (a.mode == FINISH_RESET && a.st->hist_n == 0)))
      history_record(a, a.mode == FINISH_LOOP ? a.st->hist_base + sweep + 1 : 0);
    if (loop) a.st->sweep += 1;
    a.st->ticket = 0u;
  }
}

// FINISH_ODD of a one-unit loop (the odd half-sweep's per-CTA partials, a few hundred)
// by one warp: each lane adds every 32nd partial in order, then a fixed shuffle tree, no
// block barrier; thread 0 then does exactly what k_finish's one-unit FINISH_ODD does.
// This finish runs after every odd half-sweep, between it and the next even one.
__global__ void __launch_bounds__(32) k_finish_odd1(FinishArgs a) {
  grid_dep_wait();
  grid_dep_launch();
  const int lane = (int)threadIdx.x;
  // Every load is issued before anything depends on it (the partials too, although they
  // are used only on check sweeps): the kernel is one round trip to L2, the tree and
  // thread 0's stores.
  const int n_active = a.st->n_active, sweep = a.st->sweep, limit = a.st->limit;
  const int ci = a.st->check_interval, hold = a.st->hold, final_level = a.st->final_level;
  const double eps = a.st->eps, eps_mid = a.st->eps_mid;
  const int lvl = a.active[0];
  const double invF = a.unit_norm[0], invT = a.unit_norm[1];
  const double uF_old = a.unit_sumF[0], uT_old = a.unit_sumTh[0];
  float2 aF = make_float2(0.f, 0.f), aT = aF;
#pragma unroll 8
  for (int i = lane; i < a.n_odd_parts; i += 32) {
    aF = pair_add(aF, a.part_F[i]);
    aT = pair_add(aT, a.part_th_odd[i]);
  }
  if (!(n_active > 0 && sweep < limit) || hold) return;  // stopped, or the sweep is open
  const bool check = ((sweep + 1) % ci) == 0 || sweep + 1 == limit;  // state_check_sweep
  const bool was_active = lvl > 0;
  const bool reduce = was_active && check;
  if (reduce) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float2 bF, bT;
      bF.x = __shfl_down_sync(0xffffffffu, aF.x, o);
      bF.y = __shfl_down_sync(0xffffffffu, aF.y, o);
      bT.x = __shfl_down_sync(0xffffffffu, aT.x, o);
      bT.y = __shfl_down_sync(0xffffffffu, aT.y, o);
      aF = pair_add(aF, bF);
      aT = pair_add(aT, bT);
    }
  }
  if (lane != 0) return;
  const double thr = (lvl == 1 && final_level > 1) ? eps_mid : eps;
  const bool forced = sweep + 1 == limit;  // the budget's last sweep is measured exactly
  double uF = uF_old;
  bool pend = false;
  if (reduce) {
    const double s0 = pair_value(aF), s1 = pair_value(aT);
    uF = s0;
    a.unit_sumF[0] = s0;
    a.unit_F[0] = s0 * invF;
    a.unit_sumTh_odd[0] = s1;
    pend = forced || a.hist != nullptr || !(s1 * invT >= thr);  // a history wants every theta
  }
  a.pending[0] = pend ? lvl : 0;
  if (pend) {
    a.st->need_exact = 1;
    a.st->sweep_closed = 0;
    a.st->hold = 1;
  } else {
    if (was_active) a.iters[0] += 1;
    if (check) {
      a.lat_F[0] = uF * invF;
      a.lat_theta[0] = uT_old * invT;
    }
    a.st->need_exact = 0;
    a.st->sweep_closed = 1;
    a.st->sweep = sweep + 1;
  }
  a.st->ticket = 0u;
}

void launch_finish(const FinishArgs& a, cudaStream_t s) {
  if (a.mode == FINISH_ODD && a.n_units == 1 && a.n_odd_parts <= 1024)
    launch_dep(a.dep != 0, k_finish_odd1, dim3(1), dim3(32), 0, s, a);
  else
    launch_dep(a.dep != 0, k_finish, dim3(a.n_units), dim3(kFinishThreads), 0, s, a);
}

// ---------------------------------------------------------------------------------
// element kernels
// ---------------------------------------------------------------------------------
// Canonical <-> storage.  A block takes kPackLinks consecutive canonical links (9
// complex128 each, site-major): the canonical side moves through shared memory with
// consecutive threads on consecutive 16-byte words (coalesced, also when the canonical
// buffer is pinned host memory read or written directly over the host link); each
// thread then converts one link.
constexpr int kPackLinks = 128;

__device__ __forceinline__ int storage_idx(const LatDev& lat, long long s) {
  const int sl = (int)s;  // V < 2^31 (checked at creation)
  const int x = sl % lat.L[0];
  int r = sl / lat.L[0];
  const int y = r % lat.L[1];
  r /= lat.L[1];
  const int z = r % lat.L[2];
  const int t = r / lat.L[2];
  return ((x + y + z + t) & 1) * lat.Vh + (sl >> 1);
}

template <int S>
__global__ void __launch_bounds__(kPackLinks) k_pack(char* links, LatDev lat, const double2* src,
                                                     long long s0, long long nsites) {
  using St = Store<S>;
  using T = typename St::T;
  __shared__ double2 sm[kPackLinks * 9];
  const long long l0 = (long long)blockIdx.x * kPackLinks;  // first link of the block
  const long long nl = nsites * 4;
  const int nb = (int)(nl - l0 < kPackLinks ? nl - l0 : kPackLinks);
  for (int w = threadIdx.x; w < nb * 9; w += kPackLinks) sm[w] = src[l0 * 9 + w];
  __syncthreads();
  if ((int)threadIdx.x >= nb) return;
  const long long i = l0 + threadIdx.x;
  const long long s = s0 + i / 4;
  const int mu = (int)(i % 4);
  cx<T> e[St::NE];
#pragma unroll
  for (int k = 0; k < St::NE; ++k) {
    const double2 v = sm[threadIdx.x * 9 + k];
    e[k] = {(T)v.x, (T)v.y};
  }
  St::store(links + lat.off_bytes, lat.V, mu, storage_idx(lat, s), e);
}

template <int S>
__global__ void __launch_bounds__(kPackLinks) k_unpack(const char* links, LatDev lat, double2* dst,
                                                       long long s0, long long nsites) {
  using St = Store<S>;
  using T = typename St::T;
  __shared__ double2 sm[kPackLinks * 9];
  const long long l0 = (long long)blockIdx.x * kPackLinks;
  const long long nl = nsites * 4;
  const int nb = (int)(nl - l0 < kPackLinks ? nl - l0 : kPackLinks);
  if ((int)threadIdx.x < nb) {
    const long long i = l0 + threadIdx.x;
    const long long s = s0 + i / 4;
    const int mu = (int)(i % 4);
    cx<T> e[St::NE];
    St::load(links + lat.off_bytes, lat.V, mu, storage_idx(lat, s), e);
    cx<double> m[9];
#pragma unroll
    for (int k = 0; k < St::NE; ++k) m[k] = {(double)e[k].re, (double)e[k].im};
    if constexpr (St::NE == 6) third_row(m, m + 6);
#pragma unroll
    for (int k = 0; k < 9; ++k) sm[threadIdx.x * 9 + k] = make_double2(m[k].re, m[k].im);
  }
  __syncthreads();
  for (int w = threadIdx.x; w < nb * 9; w += kPackLinks) dst[l0 * 9 + w] = sm[w];
}

template <int S>
__global__ void __launch_bounds__(256) k_reunit(char* links, LatDev lat) {
  using St = Store<S>;
  using T = typename St::T;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4 * lat.V) return;
  const int mu = (int)(i / lat.V), idx = (int)(i % lat.V);
  cx<T> e[St::NE];
  St::load(links + lat.off_bytes, lat.V, mu, idx, e);
  reunit(e);
  St::store(links + lat.off_bytes, lat.V, mu, idx, e);
}

template <int S>
__global__ void __launch_bounds__(256) k_to_fp64(const char* src, char* dst, LatDev ls, LatDev ld) {
  using St = Store<S>;
  using T = typename St::T;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4 * ls.V) return;
  const int mu = (int)(i / ls.V), idx = (int)(i % ls.V);
  cx<T> e[St::NE];
  St::load(src + ls.off_bytes, ls.V, mu, idx, e);
  cx<double> m[9];
#pragma unroll
  for (int k = 0; k < St::NE; ++k) m[k] = {(double)e[k].re, (double)e[k].im};
  if constexpr (St::NE == 6) third_row(m, m + 6);
  reunit(m);
  Store<GF_FP64_18>::store(dst + ld.off_bytes, ld.V, mu, idx, m);
}

__global__ void k_fill_int(int* p, int value, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = value;
}

void launch_fill_int(int* p, int value, int n, cudaStream_t s) {
  if (n > 0) k_fill_int<<<(n + 255) / 256, 256, 0, s>>>(p, value, n);
}

static unsigned int blocks_for(long long n, int threads) { return (unsigned int)((n + threads - 1) / threads); }

#define GF_ELEM_SWITCH(storage, CALL)                  \
  switch (storage) {                                   \
    case GF_FP64_18: CALL(GF_FP64_18); break;          \
    case GF_FP32_18: CALL(GF_FP32_18); break;          \
    case GF_FP64_12: CALL(GF_FP64_12); break;          \
    case GF_FP32_8: CALL(GF_FP32_8); break;            \
    case GF_FP64_8: CALL(GF_FP64_8); break;            \
    default: CALL(GF_FP32_12); break;                  \
  }

void launch_pack(int storage, char* links, const LatDev& lat, const double* src, long long s0,
                 long long nsites, cudaStream_t s) {
  if (nsites <= 0) return;
  const unsigned int nb = blocks_for(nsites * 4, kPackLinks);
  const double2* p = reinterpret_cast<const double2*>(src);
#define GF_CALL(S) k_pack<S><<<nb, kPackLinks, 0, s>>>(links, lat, p, s0, nsites)
  GF_ELEM_SWITCH(storage, GF_CALL)
#undef GF_CALL
}

void launch_unpack(int storage, const char* links, const LatDev& lat, double* dst, long long s0,
                   long long nsites, cudaStream_t s) {
  if (nsites <= 0) return;
  const unsigned int nb = blocks_for(nsites * 4, kPackLinks);
  double2* p = reinterpret_cast<double2*>(dst);
#define GF_CALL(S) k_unpack<S><<<nb, kPackLinks, 0, s>>>(links, lat, p, s0, nsites)
  GF_ELEM_SWITCH(storage, GF_CALL)
#undef GF_CALL
}

void launch_reunit(int storage, char* links, const LatDev& lat, cudaStream_t s) {
  const unsigned int nb = blocks_for(4 * lat.V, 256);
#define GF_CALL(S) k_reunit<S><<<nb, 256, 0, s>>>(links, lat)
  GF_ELEM_SWITCH(storage, GF_CALL)
#undef GF_CALL
}

void launch_to_fp64(int storage, const char* src, char* dst, const LatDev& ls, const LatDev& ld,
                    cudaStream_t s) {
  const unsigned int nb = blocks_for(4 * ls.V, 256);
#define GF_CALL(S) k_to_fp64<S><<<nb, 256, 0, s>>>(src, dst, ls, ld)
  GF_ELEM_SWITCH(storage, GF_CALL)
#undef GF_CALL
}

}  // namespace gf
