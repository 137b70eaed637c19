// gf_kernels.cuh -- the kernels of libgf, templated on storage and gauge.
//
// Instantiated in exactly one translation unit each (gf_inst_*.cu); see the bottom of
// this file for the launch helpers declared to the host code.
#pragma once

#include "gf_device.cuh"

namespace gf {

// ----------------------------------------------------------------------------------
// Eqs. (4)-(6): maximise Re Tr[R K] in the SU(2) subgroup on rows/columns (i, j),
// then R -> R^omega (Section 1, sentence after Eq. (6); Mandula-Ogilvie).
//   alpha = K_ii + conj(K_jj), beta = K_ji - conj(K_ij): Re Tr[R K] = const +
//   Re(a alpha) + Re(b beta) for R|_(i,j) = [[a, b], [-conj b, conj a]], maximal at
//   (a, b) = conj(alpha, beta) / |(alpha, beta)|; R = 1 when alpha = beta = 0.
// REPRO: IEEE divisions in the order of a plain C implementation; otherwise one
// reciprocal square root and multiplications.
// ----------------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T gf_rsqrt(T x);
template <>
__device__ __forceinline__ double gf_rsqrt<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float gf_rsqrt<float>(float x) { return rsqrtf(x); }

template <class T, bool REPRO, int FORM>
__device__ __forceinline__ void su2_maximiser(const cx<T> (&K)[9], int i, int j, T omega,
                                              cx<T>& a, cx<T>& b) {
  const cx<T> alpha = cadd(K[3 * i + i], cconj(K[3 * j + j]));
  const cx<T> beta = csub(K[3 * j + i], cconj(K[3 * i + j]));
  const T n2 = ((alpha.re * alpha.re + alpha.im * alpha.im) + beta.re * beta.re) + beta.im * beta.im;
  a = {T(1), T(0)};
  b = {T(0), T(0)};
  if constexpr (REPRO) {
    const T n = gf_sqrt(n2);
    if (n > T(0)) {
      a = {alpha.re / n, -alpha.im / n};
      b = {beta.re / n, -beta.im / n};
    }
  } else {
    if (n2 > T(0)) {
      const T rn = gf_rsqrt(n2);
      a = {alpha.re * rn, -alpha.im * rn};
      b = {beta.re * rn, -beta.im * rn};
    }
  }
  if constexpr (FORM == GF_OR_FIRST_ORDER) {
    // g^omega to first order: 1 + omega (g - 1), renormalised onto SU(2)
    const cx<T> a1 = {(T(1) - omega) + omega * a.re, omega * a.im};
    const cx<T> b1 = {omega * b.re, omega * b.im};
    const T m2 = ((a1.re * a1.re + a1.im * a1.im) + b1.re * b1.re) + b1.im * b1.im;
    if constexpr (REPRO) {
      const T m = gf_sqrt(m2);
      if (m > T(0)) {
        a = {a1.re / m, a1.im / m};
        b = {b1.re / m, b1.im / m};
      }
    } else {
      if (m2 > T(0)) {
        const T rm = gf_rsqrt(m2);
        a = cscale(a1, rm);
        b = cscale(b1, rm);
      }
    }
  } else {
    // exact power: R = cos(phi) + i sin(phi) n.sigma  ->  cos(omega phi) + i sin(omega phi) n.sigma
    const T s = gf_sqrt((a.im * a.im + b.re * b.re) + b.im * b.im);
    if (s > T(0)) {
      const T phi = atan2(s, a.re);
      const T c1 = cos(omega * phi), s1 = sin(omega * phi);
      a = {c1, (a.im / s) * s1};
      b = {(b.re / s) * s1, (b.im / s) * s1};
    }
  }
}

// M <- R M for the subgroup element R on rows (i, j)
template <class T>
__device__ __forceinline__ void su2_left_mul(cx<T> (&M)[9], int i, int j, cx<T> a, cx<T> b) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const cx<T> mi = M[3 * i + c], mj = M[3 * j + c];
    M[3 * i + c] = cadd(cmul(a, mi), cmul(b, mj));
    M[3 * j + c] = cadd(cmul(cneg(cconj(b)), mi), cmul(cconj(a), mj));
  }
}

// G = product of the three subgroup maximisers for K (Cabibbo-Marinari order (0,1),
// (0,2), (1,2)), K rotated after each one.
// The first product R1 * 1 is R1 itself (x * 1 = x, x + 0 = x: the values of the plain
// sequence).  K is left as R2 R1 K unless rotate_last asks for the third rotation too,
// which leaves K = G K (used by the fused check, see site_check_from_GK).
template <class T, bool REPRO, int FORM>
__device__ __forceinline__ void su3_update(cx<T> (&K)[9], cx<T> (&G)[9], T omega,
                                           bool rotate_last = false) {
  cx<T> a, b;
  su2_maximiser<T, REPRO, FORM>(K, 0, 1, omega, a, b);
  su2_left_mul(K, 0, 1, a, b);
#pragma unroll
  for (int e = 0; e < 9; ++e) G[e] = {T(0), T(0)};
  G[0] = a;
  G[1] = b;
  G[3] = cneg(cconj(b));
  G[4] = cconj(a);
  G[8] = {T(1), T(0)};
  su2_maximiser<T, REPRO, FORM>(K, 0, 2, omega, a, b);
  su2_left_mul(K, 0, 2, a, b);
  su2_left_mul(G, 0, 2, a, b);
  su2_maximiser<T, REPRO, FORM>(K, 1, 2, omega, a, b);
  su2_left_mul(G, 1, 2, a, b);
  if (rotate_last) su2_left_mul(K, 1, 2, a, b);
}

// K += U_mu(x) + U_mu(x - mu)^dagger (in-place form of Eq. (5))
template <class T, int NE>
__device__ __forceinline__ void add_to_K(cx<T> (&K)[9], const cx<T> (&f)[NE], const cx<T> (&b)[NE]) {
  cx<T> fu[9], bu[9];
  to_full(f, fu);
  to_full(b, bu);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) K[3 * r + c] = cadd(K[3 * r + c], cadd(fu[3 * r + c], cconj(bu[3 * c + r])));
}

// A += U_nu(x - nu) - U_nu(x)  (Eq. (3), one direction)
template <class T, int NE>
__device__ __forceinline__ void add_to_A(cx<T> (&A)[9], const cx<T> (&f)[NE], const cx<T> (&b)[NE]) {
  cx<T> fu[9], bu[9];
  to_full(f, fu);
  to_full(b, bu);
#pragma unroll
  for (int e = 0; e < 9; ++e) A[e] = cadd(A[e], csub(bu[e], fu[e]));
}

// add_to_A and F += Re Tr f + Re Tr b from the same full matrices (Re Tr of a 12-real
// link is e0 + e4 + Re(e0 e4 - e1 e3), the (2,2) element of its rebuilt third row)
template <class T, int NE>
__device__ __forceinline__ void add_to_A_F(cx<T> (&A)[9], T& fs, const cx<T> (&f)[NE], const cx<T> (&b)[NE]) {
  cx<T> fu[9], bu[9];
  to_full(f, fu);
  to_full(b, bu);
#pragma unroll
  for (int e = 0; e < 9; ++e) A[e] = cadd(A[e], csub(bu[e], fu[e]));
  fs = fs + ((fu[0].re + fu[4].re + fu[8].re) + (bu[0].re + bu[4].re + bu[8].re));
}

// Tr[Delta Delta^dagger] with Delta = A - A^dagger - (1/3) Tr(A - A^dagger)
template <class T>
__device__ __forceinline__ T theta_site(const cx<T> (&A)[9]) {
  cx<T> D[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) D[3 * i + j] = csub(A[3 * i + j], cconj(A[3 * j + i]));
  const cx<T> sum = cadd(cadd(D[0], D[4]), D[8]);
  const cx<T> tr = {sum.re / T(3), sum.im / T(3)};
  D[0] = csub(D[0], tr);
  D[4] = csub(D[4], tr);
  D[8] = csub(D[8], tr);
  T q = T(0);
#pragma unroll
  for (int e = 0; e < 9; ++e) q = q + (D[e].re * D[e].re + D[e].im * D[e].im);
  return q;
}

// F and Tr[Delta Delta^dagger] of a site just updated, from K' = G K (K of Eq. (5) before
// the update).  The site's new links are G U_mu(x) and U_mu(x - mu) G^dagger, so
// K' = sum_mu [U'_mu(x) + U'_mu(x - mu)^dagger]; then A' = sum_mu [U'_mu(x - mu) - U'_mu(x)]
// of Eq. (3) has A' - A'^dagger = K'^dagger - K', so Delta(x) is the traceless
// anti-Hermitian part of K' up to its sign, and Re Tr K' is the site's share of Eq. (1)
// (each of its links counted once).  The values are those of the links before any
// reunitarisation of the same sweep.
template <class T>
__device__ __forceinline__ void site_check_from_GK(const cx<T> (&Kp)[9], T& fs, T& q) {
  fs = (Kp[0].re + Kp[4].re) + Kp[8].re;
  q = theta_site(Kp);
}

// Per-tile partial sums: FP64 storage reduces in FP64; FP32 storage in compensated FP32
// with one conversion per block (see block_sum_f32).
template <class T, int NV>
__device__ __forceinline__ void tile_sum(const T (&v)[NV], double (&out)[NV], double* smem64) {
  if constexpr (sizeof(T) == 8) {
    double w[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) w[k] = v[k];
    block_sum<NV>(w, smem64);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = w[k];
  } else {
    block_sum_f32<NV>(v, out, reinterpret_cast<float*>(smem64));
  }
}

// the same with each total as a pair (hi, lo) for the finishing reduction
template <class T, int NV>
__device__ __forceinline__ void tile_sum(const T (&v)[NV], float2 (&out)[NV], double* smem64) {
  if constexpr (sizeof(T) == 8) {
    double w[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) w[k] = v[k];
    block_sum<NV>(w, smem64);
#pragma unroll
    for (int k = 0; k < NV; ++k) out[k] = pair_of(w[k]);
  } else {
    block_sum_f32<NV>(v, out, reinterpret_cast<float*>(smem64));
  }
}

// ----------------------------------------------------------------------------------
// Kernel arguments
// ----------------------------------------------------------------------------------
struct SweepArgs {
  char* links;
  const LatDev* lats;
  const int4* tiles;       // (lat, t, first h3, unit) per block
  const int* active;       // per unit (nullable: all units): a tile runs when its unit's
                           // entry equals `level`
  const DevState* st;      // nullable; when set, the loop state decides everything
  float2* part_theta;      // per tile: theta partial of the updated (odd) sites (hi, lo)
  float2* part_F;          // nullable; per tile: Re Tr of the updated sites' 2 nd links
  int parity;
  int form;
  int reunit;              // used when st == nullptr
  int measure;             // used when st == nullptr
  int n_tiles;
  int reverse;             // walk the tiles last to first (L2 reuse across passes)
  int level;               // precision level these tiles must carry in `active` (1 unless mixed)
  int cta_sums;            // persistent kernels, one unit: F and theta partials per CTA (indexed
                           // by blockIdx.x) instead of per tile
  int dep;                 // launch with programmatic stream serialisation (launch_dep)
  double omega;
};

struct MeasureArgs {
  const char* links;
  const LatDev* lats;
  const int4* tiles;
  const int* active;       // nullable; a tile runs when its unit's entry equals `level`
  const DevState* st;      // nullable; when set, only runs on check sweeps
  float2* part_F;          // nullable: per tile sum of Re Tr over the 2 nd links of each site
  float2* part_theta;      // per tile sum of Tr[Delta Delta^+] (pairs hi, lo)
  int parity;
  int n_tiles;
  int reverse;
  int level;
  int dep;                 // launch with programmatic stream serialisation (launch_dep)
};

constexpr int kFinishThreads = 256;  // threads of a finishing block (one block per unit)
constexpr int kFinishUnroll = 16;    // tile partials a finishing thread loads at once

struct FinishArgs {
  const LatDev* lats;
  const int* unit_tiles;   // n_units + 1 tile boundaries
  int n_tiles;             // tiles of the table (the single unit's range when n_units == 1)
  int n_odd_parts;         // one unit: partials the odd half-sweep wrote (tiles, or its CTAs)
  int* pending;            // per unit: the unit's level when this check needs the even-site
                           // pass (FINISH_ODD sets it), or when FINISH_ENTER is to measure it
  double* hist;            // nullable: records (sweep, F and theta of every lattice) of each check
  int hist_cap;            // records hist can hold
  double* unit_sumTh_odd;  // per unit: odd-site part of the theta sum of the current check
  const int* unit_lat;     // lattice of each unit
  const double* unit_norm;  // per unit 1 / (nd Nc sites), 1 / (Nc sites): F and theta of Eqs. (1), (2)
  int* active;             // per unit: level (> 0) while sweeping, 0 done, -level when the
                           // unit reached the threshold of a level below the final one
  int* iters;
  const float2* part_F;    // per-tile partials as pairs (hi, lo)
  const float2* part_th_even;
  const float2* part_th_odd;
  double* unit_sumF;
  double* unit_sumTh;
  double* unit_F;
  double* unit_theta;
  double* lat_F;
  double* lat_theta;
  DevState* st;
  int n_units;
  int n_lat;
  int nd;
  int mode;                // FINISH_LOOP, FINISH_MEASURE, FINISH_RESET, FINISH_ODD, FINISH_ENTER,
                           // FINISH_OPEN
  int gated;               // FINISH_RESET after FINISH_OPEN: runs only if that left units undecided
  int dep;                 // launch with programmatic stream serialisation (launch_dep)
};

enum { FINISH_LOOP = 0, FINISH_MEASURE = 1, FINISH_RESET = 2, FINISH_ODD = 3, FINISH_ENTER = 4, FINISH_OPEN = 5 };

// Fourier-accelerated steepest descent (kernels in gf_fasd.cuh)
struct FasdArgs {
  char* links;            // link storage (FP32-12 or FP64-18) of the lattice
  LatDev lat;
  void* kbuf;             // 4 complex fields, [f][t][z][y][x]
  char* gbuf;             // g(x): rows 0 and 1, 2 * 3 complex elements, planes [w][lexi]
  float2* plane_F;        // per (z, t) plane, as pairs (hi, lo)
  float2* plane_th;
  const int* unit_planes; // n_units + 1 plane boundaries
  int* active;
  int* iters;
  double* unit_sumF;
  double* unit_sumTh;
  double* unit_F;
  double* unit_theta;
  double* lat_F;
  double* lat_theta;
  DevState* st;           // nullable for a single step
  int nd;                 // 4 Landau, 3 Coulomb
  int n_units;
  int reunit;             // reunitarise the links in the update (single-step use)
  int mode;               // finish: FINISH_LOOP or FINISH_MEASURE
  int logL[4];
  int kx;                 // kx columns per block of the z/t transform (power of 2, <= 8)
  int xy_prefetch;        // inverse x/y transform: two plane buffers (next plane prefetched)
  int zt_prefetch;        // z/t transform: two column buffers (next item prefetched)
  double coef;            // alpha / 2 * p^2_max / N_fft
};

// kx columns per z/t-transform item: up to 4 (Landau: 4 x Lz lines per direction, one
// per thread of a 128-thread block at 32^4) or 32 (Coulomb: one z-line per column),
// halved until two items' columns (nt x (KX Lz + KX) elements of c bytes each) fit in
// 110 KB of shared memory, so that two double-buffered blocks share an SM
inline int fasd_kx(const LatDev& lat, int nd, size_t c) {
  const int cap = nd == 4 ? 4 : 32;
  int kx = lat.L[0] < cap ? lat.L[0] : cap;
  const size_t nt = nd == 4 ? lat.L[3] : 1;
  while (kx > 1 && 2 * nt * ((size_t)kx * lat.L[2] + kx) * c > 110 * 1024) kx /= 2;
  return kx;
}

// Differentiable F(c), theta(c) (kernels in gf_autograd.cuh)
using c64 = cx<double>;

struct AdArgs {
  const char* links;   // FP64-18 storage of the lattice
  LatDev lat;
  const double* c;     // [V][8], canonical site order
  c64* g;              // [V][9] scratch
  c64* delta;          // [V][9] scratch
  double* part;        // [blocks][2]
  double* out;         // F, theta
  const double* upstream;  // dL/dF, dL/dtheta
  double* grad;        // [V][8]
  unsigned int* ticket;
  int nd;
};

// ----------------------------------------------------------------------------------
// Algorithm 1, one half-sweep: every site of one parity, one thread per site.
// KEEP: hold the 8 links in registers (FP32); otherwise stream them twice (FP64).
// ----------------------------------------------------------------------------------
template <int S, int ND, bool REPRO, int FORM>
__global__ void __launch_bounds__(256) k_or_sweep(SweepArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  constexpr int NE = St::NE;
  constexpr bool KEEP = sizeof(T) == 4;
  __shared__ double red[64];

  bool reunit_now = a.reunit != 0, measure_now = a.measure != 0;
  if (a.st) {
    if (!state_sweeping(a.st)) return;
    reunit_now = a.parity == 1 && state_reunit_sweep(a.st);
    measure_now = a.parity == 1 && state_check_sweep(a.st);
  }
  const int ti = a.reverse ? a.n_tiles - 1 - (int)blockIdx.x : (int)blockIdx.x;
  const int4 tile = a.tiles[ti];
  if (a.active && a.active[tile.w] != a.level) return;
  const LatDev lat = a.lats[tile.x];
  const int h3 = tile.z + (int)threadIdx.x;
  T q = T(0), fs = T(0);
  if (h3 < lat.V3h) {
    const int p = a.parity;
    const int h = tile.y * lat.V3h + h3;
    const Site s = site_of_slice(lat, p, tile.y, h3);
    char* base = a.links + lat.off_bytes;
    const long long V = lat.V;
    const int idx_f = p * lat.Vh + h;
    int idx_b[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) idx_b[mu] = (1 - p) * lat.Vh + (int)(back_lexi(lat, s, mu) >> 1);
    const T omega = (T)a.omega;

    cx<T> K[9], G[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) K[e] = {T(0), T(0)};
    // FP32 sweeps take the check from G K; FP64 ones sum the stored links' A (Eq. (3))
    constexpr bool kCheckGK = sizeof(T) == 4;

    if constexpr (KEEP) {
      cx<T> f[4][NE], b[4][NE];
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        St::load(base, V, mu, idx_f, f[mu]);
        St::load(base, V, mu, idx_b[mu], b[mu]);
      }
#pragma unroll
      for (int mu = 0; mu < ND; ++mu) add_to_K(K, f[mu], b[mu]);
      su3_update<T, REPRO, FORM>(K, G, omega, kCheckGK && measure_now);
      if (kCheckGK && measure_now) site_check_from_GK(K, fs, q);
      cx<T> A[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) A[e] = {T(0), T(0)};
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        left_mul(G, f[mu]);
        right_mul_dag(b[mu], G);
        if (reunit_now) {
          reunit(f[mu]);
          reunit(b[mu]);
        }
        if (!kCheckGK && mu < ND && measure_now) add_to_A_F(A, fs, f[mu], b[mu]);
        St::store(base, V, mu, idx_f, f[mu]);
        St::store(base, V, mu, idx_b[mu], b[mu]);
      }
      if (!kCheckGK && measure_now) q = theta_site(A);
    } else {
#pragma unroll
      for (int mu = 0; mu < ND; ++mu) {
        cx<T> f[NE], b[NE];
        St::load(base, V, mu, idx_f, f);
        St::load(base, V, mu, idx_b[mu], b);
        add_to_K(K, f, b);
      }
      su3_update<T, REPRO, FORM>(K, G, omega, kCheckGK && measure_now);
      if (kCheckGK && measure_now) site_check_from_GK(K, fs, q);
      cx<T> A[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) A[e] = {T(0), T(0)};
#pragma unroll 1
      for (int mu = 0; mu < 4; ++mu) {
        cx<T> f[NE], b[NE];
        St::load(base, V, mu, idx_f, f);
        St::load(base, V, mu, idx_b[mu], b);
        left_mul(G, f);
        right_mul_dag(b, G);
        if (reunit_now) {
          reunit(f);
          reunit(b);
        }
        if (!kCheckGK && mu < ND && measure_now) add_to_A_F(A, fs, f, b);
        St::store(base, V, mu, idx_f, f);
        St::store(base, V, mu, idx_b[mu], b);
      }
      if (!kCheckGK && measure_now) q = theta_site(A);
    }
  }
  if (measure_now) {
    const T v[2] = {fs, q};
    float2 o[2];
    tile_sum<T, 2>(v, o, red);
    if (threadIdx.x == 0) {
      if (a.part_F) a.part_F[ti] = o[0];
      a.part_theta[ti] = o[1];
    }
  }
}

// ----------------------------------------------------------------------------------
// Eqs. (1)-(3) over the sites of one parity: Re Tr of their 2 nd links (every link is
// one site's forward or backward link, so parity 0 alone covers all of F) and
// Tr[Delta Delta^+] of Delta(x) at each site.
// ----------------------------------------------------------------------------------
template <int S, int ND>
__global__ void __launch_bounds__(256) k_measure(MeasureArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  constexpr int NE = St::NE;
  __shared__ double red[64];
  if (a.st && !state_even_pass(a.st)) return;
  const int ti = a.reverse ? a.n_tiles - 1 - (int)blockIdx.x : (int)blockIdx.x;
  const int4 tile = a.tiles[ti];
  if (a.active && a.active[tile.w] != a.level) return;
  const LatDev lat = a.lats[tile.x];
  const int h3 = tile.z + (int)threadIdx.x;
  T fsum = T(0), q = T(0);
  if (h3 < lat.V3h) {
    const int p = a.parity;
    const int h = tile.y * lat.V3h + h3;
    const Site s = site_of_slice(lat, p, tile.y, h3);
    const char* base = a.links + lat.off_bytes;
    const int idx_f = p * lat.Vh + h;
    cx<T> A[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) A[e] = {T(0), T(0)};
    T fs = T(0);
    if constexpr (sizeof(T) == 4) {
      // FP32: issue all 2 nd link loads before any arithmetic (memory-level parallelism)
      cx<T> f[ND][NE], b[ND][NE];
#pragma unroll
      for (int nu = 0; nu < ND; ++nu) {
        St::load(base, lat.V, nu, idx_f, f[nu]);
        St::load(base, lat.V, nu, (1 - p) * lat.Vh + (int)(back_lexi(lat, s, nu) >> 1), b[nu]);
      }
#pragma unroll
      for (int nu = 0; nu < ND; ++nu) {
        add_to_A_F(A, fs, f[nu], b[nu]);
      }
    } else {
#pragma unroll
      for (int nu = 0; nu < ND; ++nu) {
        cx<T> f[NE], b[NE];
        St::load(base, lat.V, nu, idx_f, f);
        St::load(base, lat.V, nu, (1 - p) * lat.Vh + (int)(back_lexi(lat, s, nu) >> 1), b);
        add_to_A_F(A, fs, f, b);
      }
    }
    fsum = fs;
    q = theta_site(A);
  }
  const T v[2] = {fsum, q};
  float2 o[2];
  tile_sum<T, 2>(v, o, red);
  if (threadIdx.x == 0) {
    if (a.part_F) a.part_F[ti] = o[0];
    a.part_theta[ti] = o[1];
  }
}

// ----------------------------------------------------------------------------------
// Per-unit F / theta from the tile partials (fixed order), masks, iteration counts,
// lattice totals and the loop state.  One block per unit; the last block to finish
// does the lattice totals (deterministic: fixed summation order everywhere).
// ----------------------------------------------------------------------------------
__global__ void __launch_bounds__(kFinishThreads) k_finish(FinishArgs a);

// ----------------------------------------------------------------------------------
// Element kernels over all links: layout conversion, reunitarisation, FP32 -> FP64.
// ----------------------------------------------------------------------------------
// canonical (site-major complex128) -> storage, for sites [s0, s0 + nsites)
template <int S>
__global__ void k_pack(char* links, LatDev lat, const double2* src, long long s0, long long nsites);
// storage -> canonical
template <int S>
__global__ void k_unpack(const char* links, LatDev lat, double2* dst, long long s0, long long nsites);
// reunitarise every link of one lattice
template <int S>
__global__ void k_reunit(char* links, LatDev lat);
// FP32 storage -> FP64-18 storage of the same lattice with an FP64 reunitarisation
template <int S>
__global__ void k_to_fp64(const char* src, char* dst, LatDev lat_src, LatDev lat_dst);

// ----------------------------------------------------------------------------------
// Host-side launchers (defined in the instantiation units)
// ----------------------------------------------------------------------------------
// A kernel launch with programmatic stream serialization when `dep` is set: the kernel
// (which calls grid_dep_wait() first in every block) may be scheduled while the previous
// kernel of the stream runs, so its launch latency and block start-up overlap that
// kernel's tail.  Captured into a graph, the launch becomes a programmatic dependency
// edge.  The driver sets it for one-unit handles, whose loop it speeds up; the loops of
// many units (five launches per sweep, a finishing block per unit) ran 3-4% slower with
// it, and launch plainly.
template <typename... P, typename... A>
inline cudaError_t launch_dep(bool dep, void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = dep ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

void launch_sweep(int storage, int nd, bool repro, int variant, const SweepArgs& a, int n_tiles,
                  int threads, cudaStream_t s);
void launch_measure(int storage, int nd, int variant, const MeasureArgs& a, int n_tiles, int threads,
                    cudaStream_t s);
void launch_finish(const FinishArgs& a, cudaStream_t s);
void launch_pack(int storage, char* links, const LatDev& lat, const double* src, long long s0,
                 long long nsites, cudaStream_t s);
void launch_unpack(int storage, const char* links, const LatDev& lat, double* dst, long long s0,
                   long long nsites, cudaStream_t s);
void launch_reunit(int storage, char* links, const LatDev& lat, cudaStream_t s);
void launch_to_fp64(int storage, const char* src, char* dst, const LatDev& lat_src,
                    const LatDev& lat_dst, cudaStream_t s);

}  // namespace gf
