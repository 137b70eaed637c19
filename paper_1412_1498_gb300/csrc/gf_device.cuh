// gf_device.cuh -- device-side types and SU(3) arithmetic of libgf (sm_103a).
//
// Lattice layout in device memory (Section 2 of the paper: sites split by parity, each
// complex element of a link at a stride of 4 V), packed into 128-bit words:
//
//   site s = x + Lx (y + Ly (z + Lz t)),  parity p = (x+y+z+t) & 1,  h = s / 2
//   idx(s) = p * V/2 + h                      (0 <= idx < V)
//   word w of link (mu, s) at  plane[(w * 4 + mu) * V + idx]
//
//   GF_FP64_18: 9 double2 planes, one complex element per 16-byte word (row-major).
//   GF_FP32_12: 3 float4 planes, two complex elements per word: (U00,U01) (U02,U10)
//               (U11,U12); row 2 = conj(row0 x row1) is rebuilt on every load.
//   GF_FP32_18: 4 float4 planes (U00..U21) then one float2 plane (U22).
//
// Consecutive threads take consecutive h of one parity, so every forward link load is
// a contiguous run and every backward link U_mu(x - mu) a shifted contiguous run (mu >
// 0) or an interleave of two neighbouring words (mu = 0): all 128-bit coalesced.
//
// The arithmetic helpers below spell out every complex operation in a fixed order.
// Compiled with -fmad=false (the "reproducible" FP64 kernels) they perform exactly the
// IEEE operations of a plain C implementation written in the same order; compiled
// normally, nvcc contracts them into fused multiply-adds.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gf.h"

namespace gf {

// ----------------------------------------------------------------------------------
// Tables shared by host and device
// ----------------------------------------------------------------------------------
struct LatDev {
  int L[4];             // Lx, Ly, Lz, Lt
  int Vh;               // V / 2
  int V3h;              // Lx Ly Lz / 2
  long long V;          // sites
  long long off_bytes;  // start of this lattice's link region in the link buffer
  int unit0;            // first convergence unit of this lattice
  int n_units;          // 1 (Landau) or Lt (Coulomb)
};

// One block of sites of one lattice, one time slice: (lat, t, first h3, unit)
// (int4 tiles in device memory).

// Sweep-loop state kept in device memory so that a captured CUDA graph can run many
// sweeps with every decision (mask, reunitarisation, check, stop) taken on the device.
struct DevState {
  int sweep;            // sweeps done in the current phase
  int limit;            // sweep budget of the current phase
  int check_interval;   // F / theta every this many sweeps
  int reunit_interval;  // reunitarise after the odd half-sweep every this many sweeps
  int n_active;         // active units after the last check
  unsigned int ticket;  // last-block-done counter of the finishing kernel
  int stop;             // Fourier-accelerated loop: final field measured, nothing left to do
  double eps;           // stop threshold of the current phase
};

__host__ __device__ inline bool state_running(const DevState* st) {
  return st->n_active > 0 && st->sweep < st->limit;
}
__host__ __device__ inline bool state_check_sweep(const DevState* st) {
  return ((st->sweep + 1) % st->check_interval) == 0 || st->sweep + 1 == st->limit;
}
__host__ __device__ inline bool state_reunit_sweep(const DevState* st) {
  return st->reunit_interval > 0 && ((st->sweep + 1) % st->reunit_interval) == 0;
}

// ----------------------------------------------------------------------------------
// Complex arithmetic in a fixed order
// ----------------------------------------------------------------------------------
template <class T>
struct cx {
  T re, im;
};

template <class T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T>
__device__ __forceinline__ cx<T> cconj(cx<T> a) { return {a.re, -a.im}; }
template <class T>
__device__ __forceinline__ cx<T> cneg(cx<T> a) { return {-a.re, -a.im}; }
// (ac - bd) + i (ad + bc)
template <class T>
__device__ __forceinline__ cx<T> cmul(cx<T> x, cx<T> y) {
  return {x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re};
}
template <class T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <class T>
__device__ __forceinline__ T cnorm2(cx<T> a) { return a.re * a.re + a.im * a.im; }

template <class T>
__device__ __forceinline__ T gf_sqrt(T x);
template <>
__device__ __forceinline__ double gf_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float gf_sqrt<float>(float x) { return sqrtf(x); }

// ----------------------------------------------------------------------------------
// Storage formats: load / store the stored complex elements of one link
// ----------------------------------------------------------------------------------
template <int S>
struct Store;

template <>
struct Store<GF_FP64_18> {
  using T = double;
  static constexpr int NE = 9;           // stored complex elements
  static constexpr int LINK_BYTES = 144;
  __device__ static __forceinline__ void load(const char* base, long long V, int mu, int idx,
                                              cx<T> (&e)[NE]) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int w = 0; w < 9; ++w) {
      double2 v = p[(long long)(w * 4 + mu) * V + idx];
      e[w] = {v.x, v.y};
    }
  }
  __device__ static __forceinline__ void store(char* base, long long V, int mu, int idx,
                                               const cx<T> (&e)[NE]) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int w = 0; w < 9; ++w) p[(long long)(w * 4 + mu) * V + idx] = make_double2(e[w].re, e[w].im);
  }
};

template <>
struct Store<GF_FP32_12> {
  using T = float;
  static constexpr int NE = 6;
  static constexpr int LINK_BYTES = 48;
  __device__ static __forceinline__ void load(const char* base, long long V, int mu, int idx,
                                              cx<T> (&e)[NE]) {
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      float4 v = p[(long long)(w * 4 + mu) * V + idx];
      e[2 * w] = {v.x, v.y};
      e[2 * w + 1] = {v.z, v.w};
    }
  }
  __device__ static __forceinline__ void store(char* base, long long V, int mu, int idx,
                                               const cx<T> (&e)[NE]) {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int w = 0; w < 3; ++w)
      p[(long long)(w * 4 + mu) * V + idx] =
          make_float4(e[2 * w].re, e[2 * w].im, e[2 * w + 1].re, e[2 * w + 1].im);
  }
};

template <>
struct Store<GF_FP32_18> {
  using T = float;
  static constexpr int NE = 9;
  static constexpr int LINK_BYTES = 72;
  __device__ static __forceinline__ void load(const char* base, long long V, int mu, int idx,
                                              cx<T> (&e)[NE]) {
    const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      float4 v = p[(long long)(w * 4 + mu) * V + idx];
      e[2 * w] = {v.x, v.y};
      e[2 * w + 1] = {v.z, v.w};
    }
    const float2* q = reinterpret_cast<const float2*>(base + 256LL * V);
    float2 v = q[(long long)mu * V + idx];
    e[8] = {v.x, v.y};
  }
  __device__ static __forceinline__ void store(char* base, long long V, int mu, int idx,
                                               const cx<T> (&e)[NE]) {
    float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
    for (int w = 0; w < 4; ++w)
      p[(long long)(w * 4 + mu) * V + idx] =
          make_float4(e[2 * w].re, e[2 * w].im, e[2 * w + 1].re, e[2 * w + 1].im);
    float2* q = reinterpret_cast<float2*>(base + 256LL * V);
    q[(long long)mu * V + idx] = make_float2(e[8].re, e[8].im);
  }
};

// ----------------------------------------------------------------------------------
// SU(3) helpers on full matrices m[9] (row-major) and stored links e[NE]
// ----------------------------------------------------------------------------------

// row 2 of an SU(3) matrix from rows 0 and 1: conj(row0 x row1)
template <class T>
__device__ __forceinline__ void third_row(const cx<T>* r, cx<T>* out) {
  out[0] = cconj(csub(cmul(r[1], r[5]), cmul(r[2], r[4])));
  out[1] = cconj(csub(cmul(r[2], r[3]), cmul(r[0], r[5])));
  out[2] = cconj(csub(cmul(r[0], r[4]), cmul(r[1], r[3])));
}

template <class T, int NE>
__device__ __forceinline__ void to_full(const cx<T> (&e)[NE], cx<T> (&m)[9]) {
#pragma unroll
  for (int k = 0; k < NE; ++k) m[k] = e[k];
  if constexpr (NE == 6) third_row(e, m + 6);
}

// Re Tr of a stored link
template <class T, int NE>
__device__ __forceinline__ T re_trace(const cx<T> (&e)[NE]) {
  if constexpr (NE == 9) {
    return e[0].re + e[4].re + e[8].re;
  } else {
    cx<T> u22 = csub(cmul(e[0], e[4]), cmul(e[1], e[3]));  // conj() keeps the real part
    return e[0].re + e[4].re + u22.re;
  }
}

// out rows (NE/3 of them) = G * U, U given by its stored elements
template <class T, int NE>
__device__ __forceinline__ void left_mul(const cx<T> (&G)[9], cx<T> (&e)[NE]) {
  cx<T> u[9];
  to_full(e, u);
#pragma unroll
  for (int i = 0; i < NE / 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = {T(0), T(0)};
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cadd(acc, cmul(G[3 * i + k], u[3 * k + j]));
      e[3 * i + j] = acc;
    }
}

// stored rows = U * G^dagger (needs only the stored rows of U)
template <class T, int NE>
__device__ __forceinline__ void right_mul_dag(cx<T> (&e)[NE], const cx<T> (&G)[9]) {
#pragma unroll
  for (int i = 0; i < NE / 3; ++i) {
    cx<T> r0 = e[3 * i], r1 = e[3 * i + 1], r2 = e[3 * i + 2];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cx<T> acc = {T(0), T(0)};
      acc = cadd(acc, cmul(r0, cconj(G[3 * j + 0])));
      acc = cadd(acc, cmul(r1, cconj(G[3 * j + 1])));
      acc = cadd(acc, cmul(r2, cconj(G[3 * j + 2])));
      e[3 * i + j] = acc;
    }
  }
}

// Gram-Schmidt projection to SU(3): normalise row 0, orthogonalise and normalise row 1,
// row 2 = conj(row0 x row1) (stored only for 18-real links).
template <class T, int NE>
__device__ __forceinline__ void reunit(cx<T> (&u)[NE]) {
  T n0 = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) n0 = n0 + (u[k].re * u[k].re + u[k].im * u[k].im);
  n0 = T(1) / gf_sqrt(n0);
#pragma unroll
  for (int k = 0; k < 3; ++k) u[k] = cscale(u[k], n0);
  cx<T> p = {T(0), T(0)};
#pragma unroll
  for (int k = 0; k < 3; ++k) p = cadd(p, cmul(cconj(u[k]), u[3 + k]));
#pragma unroll
  for (int k = 0; k < 3; ++k) u[3 + k] = csub(u[3 + k], cmul(p, u[k]));
  T n1 = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) n1 = n1 + (u[3 + k].re * u[3 + k].re + u[3 + k].im * u[3 + k].im);
  n1 = T(1) / gf_sqrt(n1);
#pragma unroll
  for (int k = 0; k < 3; ++k) u[3 + k] = cscale(u[3 + k], n1);
  if constexpr (NE == 9) third_row(u, u + 6);
}

// ----------------------------------------------------------------------------------
// Lattice geometry for one thread: site of parity p with half-index h
// ----------------------------------------------------------------------------------
struct Site {
  int x, y, z, t;
  long long lexi;
};

__device__ __forceinline__ Site site_of(const LatDev& lat, int parity, int h) {
  long long s2 = 2LL * h;
  Site s;
  int x0 = (int)(s2 % lat.L[0]);
  long long r = s2 / lat.L[0];
  s.y = (int)(r % lat.L[1]);
  r /= lat.L[1];
  s.z = (int)(r % lat.L[2]);
  s.t = (int)(r / lat.L[2]);
  s.x = x0 + ((s.y + s.z + s.t + parity) & 1);
  s.lexi = s2 + (s.x - x0);
  return s;
}

// lexicographic index of x - mu_hat (periodic)
__device__ __forceinline__ long long back_lexi(const LatDev& lat, const Site& s, int mu) {
  const long long Lx = lat.L[0], LxLy = Lx * lat.L[1], V3 = LxLy * lat.L[2];
  switch (mu) {
    case 0: return s.x == 0 ? s.lexi + (Lx - 1) : s.lexi - 1;
    case 1: return s.y == 0 ? s.lexi + Lx * (lat.L[1] - 1) : s.lexi - Lx;
    case 2: return s.z == 0 ? s.lexi + LxLy * (lat.L[2] - 1) : s.lexi - LxLy;
    default: return s.t == 0 ? s.lexi + V3 * (lat.L[3] - 1) : s.lexi - V3;
  }
}

// parity-split index of the site with lexicographic index lexi
__device__ __forceinline__ int idx_from_lexi(const LatDev& lat, long long lexi) {
  long long r = lexi;
  const int x = (int)(r % lat.L[0]); r /= lat.L[0];
  const int y = (int)(r % lat.L[1]); r /= lat.L[1];
  const int z = (int)(r % lat.L[2]);
  const int t = (int)(r / lat.L[2]);
  return ((x + y + z + t) & 1) * lat.Vh + (int)(lexi >> 1);
}

// lexicographic index of lexi + dir * mu_hat (periodic), dir = +1 or -1
__device__ __forceinline__ long long lexi_step(const LatDev& lat, long long lexi, int mu, int dir) {
  long long stride = 1;
  for (int k = 0; k < mu; ++k) stride *= lat.L[k];
  const int c = (int)((lexi / stride) % lat.L[mu]);
  const int L = lat.L[mu];
  if (dir > 0) return c == L - 1 ? lexi - stride * (L - 1) : lexi + stride;
  return c == 0 ? lexi + stride * (L - 1) : lexi - stride;
}

// ----------------------------------------------------------------------------------
// Block reduction of doubles in a fixed order (deterministic for a given block size)
// ----------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* NV * 32 */) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[k * 32 + warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nw ? smem[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      v[k] = x;
    }
  }
}

// ----------------------------------------------------------------------------------
// Block reduction of FP32 values without FP64 arithmetic per thread (FP64 issues at a
// small fraction of the FP32 rate on this GPU): a compensated (TwoSum, Knuth) tree in
// FP32 keeps each partial as an unevaluated sum hi + lo, so the block total is exact to
// about 2^-44 relative; one conversion to FP64 per block.  Fixed order: deterministic.
// ----------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <int NV>
__device__ __forceinline__ void block_sum_f32(const float (&v)[NV], double (&out)[NV],
                                              float* smem /* 2 * NV * 32 */) {
  float hi[NV], lo[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    hi[k] = v[k];
    lo[k] = 0.f;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const float oh = __shfl_down_sync(0xffffffffu, hi[k], o);
      const float ol = __shfl_down_sync(0xffffffffu, lo[k], o);
      float s, e;
      two_sum(hi[k], oh, s, e);
      hi[k] = s;
      lo[k] = (lo[k] + ol) + e;
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      smem[(2 * k) * 32 + warp] = hi[k];
      smem[(2 * k + 1) * 32 + warp] = lo[k];
    }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float h = lane < nw ? smem[(2 * k) * 32 + lane] : 0.f;
      float l = lane < nw ? smem[(2 * k + 1) * 32 + lane] : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, h, o);
        const float ol = __shfl_down_sync(0xffffffffu, l, o);
        float s, e;
        two_sum(h, oh, s, e);
        h = s;
        l = (l + ol) + e;
      }
      out[k] = (double)h + (double)l;
    }
  }
}

}  // namespace gf
