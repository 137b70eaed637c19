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
//   GF_FP64_12: 6 double2 planes (U00..U12); row 2 rebuilt on every load.
//   GF_FP32_8:  2 float4 planes (U01,U02) (U10, arg U00, arg U20).
//   GF_FP64_8:  4 double2 planes U01, U02, U10, (arg U00, arg U20).
//               Rows 0 and 1 are rebuilt from the 8 reals on every load (Store8 below).
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
  unsigned int mx, my;  // ceil(2^32 / Lx), ceil(2^32 / Ly): n / L = umulhi(n, m) for n L < 2^32
};

// Number of sites of a lattice with extents d[0..3], or -1 when an extent is below 1
// or the product exceeds max_sites.  Every partial product is compared with max_sites
// before the next multiplication (by division), so no intermediate value can overflow
// whatever the extents are (host code: creation checks and the allocation-free call).
inline long long lattice_sites_checked(const int* d, long long max_sites) {
  long long v = 1;
  for (int k = 0; k < 4; ++k) {
    if (d[k] < 1) return -1;
    if ((long long)d[k] > max_sites / v) return -1;
    v *= d[k];
  }
  return v;
}

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
  int need_exact;       // this check sweep has units whose odd-site theta alone is below eps
                        // (2: the opening check of a phase has such units)
  int sweep_closed;     // the odd-part finish already counted this sweep (nothing pending)
  int hold;             // the odd-part finish left this sweep open: it waits for the even-site
                        // pass and the loop finish, and no sweep starts before they ran
  int hist_n;           // history records written in the current gf_fix
  int hist_base;        // sweep number of the record = hist_base + sweep (across phases)
  double eps;           // stop threshold (of the final precision level)
  double eps_mid;       // threshold of level 1 when it is not the final level (mixed runs)
  int final_level;      // 1, or 3 in a mixed run (1 FP32 storage, 2 double-float, 3 FP64)
};

// Stop threshold of a unit at precision level lvl (a mixed run leaves level 1 at the
// switch threshold, the polish levels at eps).
__host__ __device__ inline double state_threshold(const DevState* st, int lvl) {
  return (lvl == 1 && st->final_level > 1) ? st->eps_mid : st->eps;
}
// Mask entry of a unit at level lvl after a check that found it below its threshold:
// done (0) at the final level, otherwise waiting (-lvl) for the host to move its
// lattice to the next level.
__host__ __device__ inline int state_mask_below(const DevState* st, int lvl) {
  return lvl >= st->final_level ? 0 : -lvl;
}

__host__ __device__ inline bool state_running(const DevState* st) {
  return st->n_active > 0 && st->sweep < st->limit;
}
// a half-sweep (or the odd-part finish) may start: running, and no open sweep before it
__host__ __device__ inline bool state_sweeping(const DevState* st) {
  return state_running(st) && !st->hold;
}
__host__ __device__ inline bool state_check_sweep(const DevState* st) {
  return ((st->sweep + 1) % st->check_interval) == 0 || st->sweep + 1 == st->limit;
}
__host__ __device__ inline bool state_reunit_sweep(const DevState* st) {
  return st->reunit_interval > 0 && ((st->sweep + 1) % st->reunit_interval) == 0;
}
// the gated even-site theta pass runs: a check sweep of the loop, or the opening check of
// a phase, was left open for units that the odd-site part alone does not decide
__host__ __device__ inline bool state_even_pass(const DevState* st) {
  if (!st->hold) return false;
  if (st->need_exact == 2) return true;
  return st->need_exact && state_running(st) && state_check_sweep(st);
}

// ----------------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization (launch_dep) may be scheduled while the kernel before it in the stream
// is still running.  grid_dep_wait() returns once that kernel has completed and its
// memory operations are visible.  Every block of such a kernel calls it first, before
// any memory access and before any early return: a block that left without waiting
// could let the kernel complete ahead of its predecessor, and the next kernel's wait
// would then no longer cover the predecessor's writes.  grid_dep_launch() lets the next
// kernel of the stream be scheduled once every block of this one has started; its
// blocks take the resources this kernel's blocks free and wait in grid_dep_wait().
// Both are no-ops in a kernel launched without the attribute.
// ----------------------------------------------------------------------------------
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
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
__device__ __forceinline__ void gf_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void gf_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ double gf_atan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float gf_atan2(float y, float x) { return atan2f(y, x); }

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

template <>
struct Store<GF_FP64_12> {
  using T = double;
  static constexpr int NE = 6;
  static constexpr int LINK_BYTES = 96;
  __device__ static __forceinline__ void load(const char* base, long long V, int mu, int idx,
                                              cx<T> (&e)[NE]) {
    const double2* p = reinterpret_cast<const double2*>(base);
#pragma unroll
    for (int w = 0; w < 6; ++w) {
      double2 v = p[(long long)(w * 4 + mu) * V + idx];
      e[w] = {v.x, v.y};
    }
  }
  __device__ static __forceinline__ void store(char* base, long long V, int mu, int idx,
                                               const cx<T> (&e)[NE]) {
    double2* p = reinterpret_cast<double2*>(base);
#pragma unroll
    for (int w = 0; w < 6; ++w) p[(long long)(w * 4 + mu) * V + idx] = make_double2(e[w].re, e[w].im);
  }
};

// 8-real parametrisation of an SU(3) link (the paper's third storage option, Section 2):
// stored u01, u02, u10 and the phases of u00 and u20.  Unitarity gives the moduli,
//   N = |u01|^2 + |u02|^2,  |u00| = sqrt(1 - N),  |u20| = sqrt(N - |u10|^2),
// and, with conj(U) = cofactor matrix of U (U^-1 = U^+ and det U = 1), the two linear
// equations  u01 u12 - u02 u11 = conj(u20)  and  conj(u00) u10 + conj(u01) u11 +
// conj(u02) u12 = 0  (rows 0 and 1 orthogonal) give, by Cramer's rule (determinant -N),
//   u11 = -(conj(u20) conj(u02) + conj(u00) u01 u10) / N,
//   u12 =  (conj(u20) conj(u01) - conj(u00) u02 u10) / N.
// N is formed from the stored u01, u02 (full relative precision near the identity).
// At N = 0 (row 0 = (e^{i phi}, 0, 0)) the stored reals do not fix the 2x2 block;
// it is taken as e^{-i phi / 2} times the identity (exact for diagonal links with that
// block, e.g. the unit link).  In-register form: rows 0 and 1 (NE = 6, as 12-real).
template <class T>
struct Store8 {
  static constexpr int NE = 6;
  __device__ static __forceinline__ void rebuild(cx<T> u01, cx<T> u02, cx<T> u10, T ph0, T ph2,
                                                 cx<T> (&e)[NE]) {
    const T N = cnorm2(u01) + cnorm2(u02);
    T s0, c0;
    gf_sincos(ph0, &s0, &c0);
    const T m0 = gf_sqrt(N < T(1) ? T(1) - N : T(0));
    const cx<T> u00 = {m0 * c0, m0 * s0};
    cx<T> u11, u12;
    if (N > T(0)) {
      T s2, c2;
      gf_sincos(ph2, &s2, &c2);
      const T d = N - cnorm2(u10);
      const T m2 = gf_sqrt(d > T(0) ? d : T(0));
      const cx<T> c20 = {m2 * c2, -(m2 * s2)};  // conj(u20)
      const cx<T> c00u10 = cmul(cconj(u00), u10);
      const T inv = T(1) / N;
      u11 = cscale(cneg(cadd(cmul(c20, cconj(u02)), cmul(u01, c00u10))), inv);
      u12 = cscale(csub(cmul(c20, cconj(u01)), cmul(u02, c00u10)), inv);
    } else {
      T sh, ch;
      gf_sincos(T(-0.5) * ph0, &sh, &ch);
      u11 = {ch, sh};
      u12 = {T(0), T(0)};
    }
    e[0] = u00;
    e[1] = u01;
    e[2] = u02;
    e[3] = u10;
    e[4] = u11;
    e[5] = u12;
  }
  // the 8 reals of rows 0, 1 (u20 = conj(u01 u12 - u02 u11), element 0 of row 2)
  __device__ static __forceinline__ void reduce(const cx<T> (&e)[NE], T& ph0, T& ph2) {
    const cx<T> u20 = cconj(csub(cmul(e[1], e[5]), cmul(e[2], e[4])));
    ph0 = gf_atan2(e[0].im, e[0].re);
    ph2 = gf_atan2(u20.im, u20.re);
  }
};

template <>
struct Store<GF_FP32_8> {
  using T = float;
  static constexpr int NE = 6;
  static constexpr int LINK_BYTES = 32;
  __device__ static __forceinline__ void load(const char* base, long long V, int mu, int idx,
                                              cx<T> (&e)[NE]) {
    const float4* p = reinterpret_cast<const float4*>(base);
    const float4 a = p[(long long)mu * V + idx];
    const float4 b = p[(long long)(4 + mu) * V + idx];
    Store8<float>::rebuild({a.x, a.y}, {a.z, a.w}, {b.x, b.y}, b.z, b.w, e);
  }
  __device__ static __forceinline__ void store(char* base, long long V, int mu, int idx,
                                               const cx<T> (&e)[NE]) {
    float ph0, ph2;
    Store8<float>::reduce(e, ph0, ph2);
    float4* p = reinterpret_cast<float4*>(base);
    p[(long long)mu * V + idx] = make_float4(e[1].re, e[1].im, e[2].re, e[2].im);
    p[(long long)(4 + mu) * V + idx] = make_float4(e[3].re, e[3].im, ph0, ph2);
  }
};

template <>
struct Store<GF_FP64_8> {
  using T = double;
  static constexpr int NE = 6;
  static constexpr int LINK_BYTES = 64;
  __device__ static __forceinline__ void load(const char* base, long long V, int mu, int idx,
                                              cx<T> (&e)[NE]) {
    const double2* p = reinterpret_cast<const double2*>(base);
    const double2 a = p[(long long)mu * V + idx];
    const double2 b = p[(long long)(4 + mu) * V + idx];
    const double2 c = p[(long long)(8 + mu) * V + idx];
    const double2 f = p[(long long)(12 + mu) * V + idx];
    Store8<double>::rebuild({a.x, a.y}, {b.x, b.y}, {c.x, c.y}, f.x, f.y, e);
  }
  __device__ static __forceinline__ void store(char* base, long long V, int mu, int idx,
                                               const cx<T> (&e)[NE]) {
    double ph0, ph2;
    Store8<double>::reduce(e, ph0, ph2);
    double2* p = reinterpret_cast<double2*>(base);
    p[(long long)mu * V + idx] = make_double2(e[1].re, e[1].im);
    p[(long long)(4 + mu) * V + idx] = make_double2(e[2].re, e[2].im);
    p[(long long)(8 + mu) * V + idx] = make_double2(e[3].re, e[3].im);
    p[(long long)(12 + mu) * V + idx] = make_double2(ph0, ph2);
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

// Site with parity-split index h3 inside time slice t.  The divisions by Lx and Ly are
// multiplications by the ceilings m = ceil(2^32 / L): with n = q L + r and m L = 2^32 + e
// (0 <= e < L), umulhi(n, m) = floor(n / L + n e / (L 2^32)) = q whenever n (L - 1) < 2^32,
// which the handle checks at creation (Lx Ly Lz max(Lx, Ly) < 2^32).
__device__ __forceinline__ Site site_of_slice(const LatDev& lat, int parity, int t, int h3) {
  const unsigned s2 = 2u * (unsigned)h3;  // lexicographic index of (x0, y, z) in the slice
  const unsigned q1 = __umulhi(s2, lat.mx);
  const unsigned q2 = __umulhi(q1, lat.my);
  Site s;
  const int x0 = (int)(s2 - q1 * (unsigned)lat.L[0]);
  s.y = (int)(q1 - q2 * (unsigned)lat.L[1]);
  s.z = (int)q2;
  s.t = t;
  s.x = x0 + ((s.y + s.z + s.t + parity) & 1);
  s.lexi = (long long)t * (2LL * lat.V3h) + (long long)(s2 + (unsigned)(s.x - x0));
  return s;
}

__device__ __forceinline__ Site site_of(const LatDev& lat, int parity, int h) {
  const int t = h / lat.V3h;
  return site_of_slice(lat, parity, t, h - t * lat.V3h);
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
        if (o >= nw) continue;  // lanes >= nw hold zeros: those levels add exact zeros
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

// the same over per-thread pairs (v_hi, v_lo), leaving each total as the unevaluated
// pair (hi, lo) (valid in thread 0)
template <int NV>
__device__ __forceinline__ void block_sum_f32_pairs(const float (&v_hi)[NV], const float (&v_lo)[NV],
                                                    float2 (&out)[NV], float* smem /* 2 * NV * 32 */) {
  float hi[NV], lo[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    hi[k] = v_hi[k];
    lo[k] = v_lo[k];
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
        if (o >= nw) continue;  // lanes >= nw hold zeros: those levels add exact zeros
        const float oh = __shfl_down_sync(0xffffffffu, h, o);
        const float ol = __shfl_down_sync(0xffffffffu, l, o);
        float s, e;
        two_sum(h, oh, s, e);
        h = s;
        l = (l + ol) + e;
      }
      out[k] = make_float2(h, l);
    }
  }
}

template <int NV>
__device__ __forceinline__ void block_sum_f32(const float (&v)[NV], float2 (&out)[NV],
                                              float* smem /* 2 * NV * 32 */) {
  float lo[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) lo[k] = 0.f;
  block_sum_f32_pairs<NV>(v, lo, out, smem);
}

// Unevaluated pairs hi + lo of floats ("double-float"): sums of per-tile partials are
// formed with FP32 instructions only.  pair_of splits a double (48 of its 53 bits kept).
__device__ __forceinline__ float2 pair_of(double d) {
  const float hi = (float)d;
  return make_float2(hi, (float)(d - (double)hi));
}
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e += a.y + b.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}
__device__ __forceinline__ double pair_value(float2 a) { return (double)a.x + (double)a.y; }

}  // namespace gf
