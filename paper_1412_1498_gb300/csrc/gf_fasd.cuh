// gf_fasd.cuh -- Fourier-accelerated steepest descent (the paper's Algorithm 2, Eqs. (7)-(9)).
//
// One iteration on one lattice:
//   A  k_fasd_delta_xy   per (z,t) plane: Delta(x) of Eq. (3) (the argument of Eq. (8)),
//                        F / theta partials of the current field, forward FFT along x, y;
//   B  k_fasd_finish     per unit: F, theta, stop rule (the measurement step of Algorithm 2);
//   C  k_fasd_zt         per (kx, ky): forward FFT along z (and t for Landau), the filter
//                        (alpha/2) p^2_max / p^2 / N (k = 0 mode set to 0), inverse FFT;
//   D  k_fasd_xy_inv_g   per (z,t) plane: inverse FFT along y, x, then
//                        g(x) = reunit(1 + Delta~(x)) (first-order exponential, Sec. 1),
//                        rows 0 and 1 stored in lexicographic site order;
//   E  k_fasd_update     per site, in lexicographic order: U_mu(x) <- g(x) U_mu(x)
//                        g(x+mu)^+ for every mu (the g of a block's forward neighbours lie
//                        in its own and the next planes, just written: L2 hits); its last
//                        block counts the iteration.
//
// Delta is anti-Hermitian and traceless and the filter is real and even in k, so the
// filtered field stays anti-Hermitian: only four complex fields are transformed -- the
// three upper off-diagonal elements and Im Delta_00 + i Im Delta_11 -- and the other
// elements follow from them.  FFTs are radix-2 in shared memory (extents powers of 2).
#pragma once

#include "gf_kernels.cuh"

namespace gf {

// threads of the plane kernels (A, D): one x- or y-line of the four fields per thread
// (4 x 32 lines at 32^2 planes), four blocks per SM
constexpr int kFasdThreads = 128;

// ------------------------------------------------------------------------- FFT
// In-place radix-2 FFTs of n_lines lines of length L = 2^logL in shared memory; line l
// starts at d[(l % n_in) * in_stride + (l / n_in) * out_stride], its element k sits
// estride further per k.  sign = -1 forward, +1 inverse (no 1/L).  tw[k] = exp(-2 pi i
// k / L), k < L/2.  n_lines and n_in are powers of 2.  Lines with contiguous elements
// (estride 1) are walked butterfly-fastest; strided lines line-fastest, so that the
// threads of a warp touch consecutive words (no shared-memory bank conflicts beyond the
// two wavefronts of 64-bit accesses).  Contains __syncthreads(): call from all threads.
template <class T>
__device__ __forceinline__ void fft_lines(cx<T>* d, const cx<T>* tw, int n_lines, int logL, int n_in,
                                          int in_stride, int out_stride, int estride, int sign) {
  const int L = 1 << logL;
  const int ll = __ffs(n_lines) - 1, li = __ffs(n_in) - 1;
  const bool lf = estride != 1;
  const int tot = n_lines << logL;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int l = lf ? (i & (n_lines - 1)) : (i >> logL);
    const int k = lf ? (i >> ll) : (i & (L - 1));
    const int r = logL ? (int)(__brev((unsigned)k) >> (32 - logL)) : 0;
    if (k < r) {
      const int o = (l & (n_in - 1)) * in_stride + (l >> li) * out_stride;
      cx<T>* a = d + o + k * estride;
      cx<T>* b = d + o + r * estride;
      const cx<T> t = *a;
      *a = *b;
      *b = t;
    }
  }
  __syncthreads();
  const int hb = tot >> 1;
  for (int s = 1; s <= logL; ++s) {
    const int half = 1 << (s - 1);
    for (int i = threadIdx.x; i < hb; i += blockDim.x) {
      const int l = lf ? (i & (n_lines - 1)) : (i >> (logL - 1));
      const int b = lf ? (i >> ll) : (i & ((L >> 1) - 1));
      const int j = b & (half - 1), k0 = ((b >> (s - 1)) << s) + j, k1 = k0 + half;
      cx<T> w = tw[j << (logL - s)];
      if (sign > 0) w.im = -w.im;
      const int o = (l & (n_in - 1)) * in_stride + (l >> li) * out_stride;
      cx<T>* p0 = d + o + k0 * estride;
      cx<T>* p1 = d + o + k1 * estride;
      const cx<T> u = *p0, v = cmul(*p1, w);
      *p0 = cadd(u, v);
      *p1 = csub(u, v);
    }
    __syncthreads();
  }
}

// Lines of up to 32 points through registers: each thread transforms whole lines
// (natural order in and out), no barrier between butterfly stages.  The transform is
// decimation in frequency (Gentleman-Sande), which leaves the result in bit-reversed
// order; the store undoes it with compile-time indices.  Same arguments and result as
// fft_lines; lines longer than 32 points go to fft_lines.
__host__ __device__ constexpr int bit_rev(int r, int logL) {
  int o = 0;
  for (int b = 0; b < logL; ++b) o |= ((r >> b) & 1) << (logL - 1 - b);
  return o;
}

// exp(-2 pi i m / L), or its conjugate for sign > 0, for a compile-time power of 2 L <= 64
// and 0 <= m < L/2, from cos(2 pi k / 64) for k = 0..16 (the values correctly rounded to
// double, written out below) and the symmetries sin x = cos(pi/2 - x), cos(pi - x) =
// -cos x.  The register transforms call it with indices fixed at compile time, so every
// twiddle is a constant in the instruction stream (none loaded, the trivial ones folded).
template <class T, int L>
__device__ __forceinline__ cx<T> twiddle(int m, int sign) {
  constexpr T c[17] = {T(1.0), T(0.9951847266721969), T(0.9807852804032304), T(0.9569403357322088),
                       T(0.9238795325112867), T(0.881921264348355), T(0.8314696123025452),
                       T(0.773010453362737), T(0.7071067811865476), T(0.6343932841636455),
                       T(0.5555702330196022), T(0.47139673682599764), T(0.3826834323650898),
                       T(0.2902846772544624), T(0.19509032201612828), T(0.0980171403295606), T(0.0)};
  const int k = m * (64 / L);  // 0 <= k < 32
  const T co = k <= 16 ? c[k] : -c[32 - k];
  const T si = k <= 16 ? c[16 - k] : c[k - 16];
  return {co, sign > 0 ? si : -si};
}

// decimation in frequency on registers: natural order in, bit-reversed order out
template <class T, int LOGL>
__device__ __forceinline__ void dif_reg(cx<T> (&v)[1 << LOGL], int sign) {
  constexpr int L = 1 << LOGL;
#pragma unroll
  for (int span = L / 2; span >= 1; span >>= 1) {
#pragma unroll
    for (int s = 0; s < L; s += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const cx<T> a = v[s + j], b = v[s + j + span];
        v[s + j] = cadd(a, b);
        cx<T> e = csub(a, b);
        if (j != 0) e = cmul(e, twiddle<T, L>(j * (L / (2 * span)), sign));  // exp(-2 pi i j / (2 span))
        v[s + j + span] = e;
      }
    }
  }
}

template <class T, int LOGL>
__device__ __forceinline__ void fft_line_reg(cx<T>* d, int estride, int sign) {
  constexpr int L = 1 << LOGL;
  cx<T> v[L];
#pragma unroll
  for (int k = 0; k < L; ++k) v[k] = d[k * estride];
  dif_reg<T, LOGL>(v, sign);
#pragma unroll
  for (int r = 0; r < L; ++r) d[bit_rev(r, LOGL) * estride] = v[r];
}

__device__ __forceinline__ float filter_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double filter_div(double a, double b) { return a / b; }

// One line of the z/t stage through registers, with a single copy of the transform
// code for every pass: the inverse transform is the forward one of the conjugate,
// conjugated (sum_k x_k exp(+2 pi i j k / L) = conj(sum_k conj(x_k) exp(-2 pi i j k /
// L))), so each pass is load (conjugated for kind 3), decimation in frequency, store in
// natural order: kind 0 forward; kind 1 forward, then each mode k scaled by coef / (base
// + s2[k]) (0 where that is not positive: the zero mode) and stored conjugated; kind 2
// the inverse of what kind 1 stored; kind 3 inverse.  A straight-line sequence of both
// directions (and the filter between them in registers) was too long for the
// instruction caches; one transform per pass keeps the stage's code small.
template <class T, int LOGL>
__device__ __forceinline__ void zt_line(cx<T>* d, int es, int kind, T base, const T* s2, T coef) {
  constexpr int L = 1 << LOGL;
  cx<T> v[L];
  const bool conj_in = kind == 3, conj_out = kind != 0;
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const cx<T> x = d[k * es];
    v[k] = {x.re, conj_in ? -x.im : x.im};
  }
  dif_reg<T, LOGL>(v, -1);
  if (kind == 1) {
#pragma unroll
    for (int r = 0; r < L; ++r) {  // v[r] holds mode bit_rev(r)
      const T p2 = base + s2[bit_rev(r, LOGL)];
      v[r] = cscale(v[r], p2 > T(0) ? filter_div(coef, p2) : T(0));
    }
  }
#pragma unroll
  for (int r = 0; r < L; ++r) d[bit_rev(r, LOGL) * es] = {v[r].re, conj_out ? -v[r].im : v[r].im};
}

template <class T>
__device__ __forceinline__ void fft_lines_reg(cx<T>* d, const cx<T>* tw, int n_lines, int logL, int n_in,
                                              int in_stride, int out_stride, int estride, int sign) {
  if (logL > 5) {
    fft_lines(d, tw, n_lines, logL, n_in, in_stride, out_stride, estride, sign);
    return;
  }
  const int li = __ffs(n_in) - 1;
  for (int l = threadIdx.x; l < n_lines; l += blockDim.x) {
    cx<T>* p = d + (l & (n_in - 1)) * in_stride + (l >> li) * out_stride;
    switch (logL) {
      case 1: fft_line_reg<T, 1>(p, estride, sign); break;
      case 2: fft_line_reg<T, 2>(p, estride, sign); break;
      case 3: fft_line_reg<T, 3>(p, estride, sign); break;
      case 4: fft_line_reg<T, 4>(p, estride, sign); break;
      case 5: fft_line_reg<T, 5>(p, estride, sign); break;
      default: break;
    }
  }
  __syncthreads();
}

template <class T>
__device__ __forceinline__ void twiddles(cx<T>* tw, int logL) {
  const int L = 1 << logL;
  for (int k = threadIdx.x; k < (L >> 1); k += blockDim.x) {
    T s, c;
    if constexpr (sizeof(T) == 8) sincospi(-2.0 * k / L, &s, &c);
    else sincospif(-2.0f * k / L, &s, &c);
    tw[k] = {c, s};
  }
}

// ------------------------------------------------------------------------- helpers
__device__ __forceinline__ long long fwd_lexi(const LatDev& lat, const Site& s, int mu) {
  const long long Lx = lat.L[0], LxLy = Lx * lat.L[1], V3 = LxLy * lat.L[2];
  switch (mu) {
    case 0: return s.x == lat.L[0] - 1 ? s.lexi - (Lx - 1) : s.lexi + 1;
    case 1: return s.y == lat.L[1] - 1 ? s.lexi - Lx * (lat.L[1] - 1) : s.lexi + Lx;
    case 2: return s.z == lat.L[2] - 1 ? s.lexi - LxLy * (lat.L[2] - 1) : s.lexi + LxLy;
    default: return s.t == lat.L[3] - 1 ? s.lexi - V3 * (lat.L[3] - 1) : s.lexi + V3;
  }
}
__device__ __forceinline__ bool fasd_running(const DevState* st) {
  return st == nullptr || (st->n_active > 0 && st->sweep < st->limit);
}

// g = reunit(1 + Delta~) from the four transformed fields Delta~_01, Delta~_02,
// Delta~_12 and (Im Delta~_00, Im Delta~_11): Delta~ is anti-Hermitian and traceless, so
// the rest follows.
template <class T>
__device__ __forceinline__ void g_from_delta(cx<T> d01, cx<T> d02, cx<T> d12, cx<T> dd, cx<T> (&g)[9]) {
  g[0] = {T(1), dd.re};
  g[4] = {T(1), dd.im};
  g[8] = {T(1), -(dd.re + dd.im)};
  g[1] = d01; g[2] = d02; g[5] = d12;
  g[3] = cneg(cconj(d01)); g[6] = cneg(cconj(d02)); g[7] = cneg(cconj(d12));
  reunit(g);
}

// g rows 0, 1 in the links' precision, site `at` (lexicographic): FP32 as 3 float4
// words, FP64 as 6 double2 words, each word a plane of V entries
template <class T>
__device__ __forceinline__ void g_store(char* gbuf, long long V, long long at, const cx<T> (&g)[9]) {
  if constexpr (sizeof(T) == 4) {
    float4* p = reinterpret_cast<float4*>(gbuf);
#pragma unroll
    for (int w = 0; w < 3; ++w) p[w * V + at] = make_float4(g[2 * w].re, g[2 * w].im, g[2 * w + 1].re, g[2 * w + 1].im);
  } else {
    double2* p = reinterpret_cast<double2*>(gbuf);
#pragma unroll
    for (int w = 0; w < 6; ++w) p[w * V + at] = make_double2(g[w].re, g[w].im);
  }
}
// rows 0, 1 (and row 2 = conj(row0 x row1) when full)
template <class T, bool FULL>
__device__ __forceinline__ void g_load(const char* gbuf, long long V, long long at, cx<T> (&g)[9]) {
  if constexpr (sizeof(T) == 4) {
    const float4* p = reinterpret_cast<const float4*>(gbuf);
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      const float4 v = p[w * V + at];
      g[2 * w].re = v.x;
      g[2 * w].im = v.y;
      g[2 * w + 1].re = v.z;
      g[2 * w + 1].im = v.w;
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(gbuf);
#pragma unroll
    for (int w = 0; w < 6; ++w) {
      const double2 v = p[w * V + at];
      g[w].re = v.x;
      g[w].im = v.y;
    }
  }
  if constexpr (FULL) third_row(g, g + 6);
}

// ------------------------------------------------------------------------- A: Delta + FFT xy
template <int S, int ND>
__global__ void __launch_bounds__(kFasdThreads, S == GF_FP64_18 ? 2 : 4) k_fasd_delta_xy(FasdArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  constexpr int NE = St::NE;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[64];
  __shared__ cx<T> twx[32], twy[32];
  if (a.st && (a.st->n_active <= 0 || a.st->stop)) return;
  const LatDev& lat = a.lat;
  const int z = blockIdx.x, t = blockIdx.y;
  const int Lx = lat.L[0], Ly = lat.L[1], P = Lx * Ly;
  const int pitch = Lx + 1;                      // padded rows: x-lines without bank conflicts
  cx<T>* pl = reinterpret_cast<cx<T>*>(smraw);  // [4][Ly][pitch]
  twiddles(twx, a.logL[0]);
  twiddles(twy, a.logL[1]);
  T fsum = T(0), q = T(0);
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    const int x = i & (Lx - 1), y = i >> a.logL[0];  // Lx, Ly are powers of 2 here
    Site s;
    s.x = x; s.y = y; s.z = z; s.t = t;
    s.lexi = x + (long long)Lx * (y + (long long)Ly * (z + (long long)lat.L[2] * t));
    const int p = (x + y + z + t) & 1;
    const int idx = p * lat.Vh + (int)(s.lexi >> 1);
    const char* base = a.links + lat.off_bytes;
    cx<T> A[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) A[e] = {T(0), T(0)};
#pragma unroll
    for (int nu = 0; nu < ND; ++nu) {
      cx<T> f[NE], b[NE];
      St::load(base, lat.V, nu, idx, f);
      // all extents are even, so x - nu has the other parity
      St::load(base, lat.V, nu, (1 - p) * lat.Vh + (int)(back_lexi(lat, s, nu) >> 1), b);
      fsum = fsum + re_trace(f);   // forward links only: every link once over all sites
      add_to_A(A, f, b);
    }
    // Delta = A - A^+ - tr/3 (as theta_site) and its four independent complex fields
    cx<T> D[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) D[3 * r + c] = csub(A[3 * r + c], cconj(A[3 * c + r]));
    const cx<T> sum = cadd(cadd(D[0], D[4]), D[8]);
    const cx<T> tr = {sum.re / T(3), sum.im / T(3)};
    D[0] = csub(D[0], tr);
    D[4] = csub(D[4], tr);
    D[8] = csub(D[8], tr);
    T qq = T(0);
#pragma unroll
    for (int e = 0; e < 9; ++e) qq = qq + (D[e].re * D[e].re + D[e].im * D[e].im);
    q = q + qq;
    const int r = y * pitch + x, fs = Ly * pitch;
    pl[r] = D[1];
    pl[fs + r] = D[2];
    pl[2 * fs + r] = D[5];
    pl[3 * fs + r] = {D[0].im, D[4].im};
  }
  const T v[2] = {fsum, q};
  float2 o[2];
  tile_sum<T, 2>(v, o, red);
  if (threadIdx.x == 0) {
    a.plane_F[z + lat.L[2] * t] = o[0];
    a.plane_th[z + lat.L[2] * t] = o[1];
  }
  __syncthreads();
  // forward FFT along x (rows), then along y (columns), all four fields
  fft_lines_reg(pl, twx, 4 * Ly, a.logL[0], 1, 0, pitch, 1, -1);            // rows (f, y), along x
  fft_lines_reg(pl, twy, 4 * Lx, a.logL[1], Lx, 1, Ly * pitch, pitch, -1);  // columns (f, x), along y
  cx<T>* kb = reinterpret_cast<cx<T>*>(a.kbuf);
  const long long plane0 = (long long)P * (z + lat.L[2] * (long long)t);
#pragma unroll 8
  for (int i = threadIdx.x; i < 4 * P; i += blockDim.x) {
    const int f = i >> (a.logL[0] + a.logL[1]), j = i & (P - 1);
    kb[f * lat.V + plane0 + j] = pl[(f * Ly + (j >> a.logL[0])) * pitch + (j & (Lx - 1))];
  }
}

// ------------------------------------------------------------------------- B: finish
// As the overrelaxation loop's finishing kernel: one block per unit adds the unit's
// plane partials (float pairs, FP32 instructions only, fixed order); one unit updates
// the loop state directly, several through a ticket.
__global__ void __launch_bounds__(256) k_fasd_finish(FasdArgs a) {
  __shared__ float2 red[2][256];
  __shared__ int s_last;
  __shared__ int s_cnt[8];
  const int tid = (int)threadIdx.x, u = (int)blockIdx.x;
  const bool loop = a.st && a.mode == FINISH_LOOP;
  int n_active = 1, stop = 0, sweep = 0, limit = 0;
  double eps = 0.0;
  if (a.st) {
    n_active = a.st->n_active;
    stop = a.st->stop;
    sweep = a.st->sweep;
    limit = a.st->limit;
    eps = a.st->eps;
  }
  const bool was_active = a.active == nullptr || a.active[u] != 0;
  const int pb = a.unit_planes[u], pe = a.unit_planes[u + 1];
  if (loop && (n_active <= 0 || stop)) return;
  const bool reduce = a.mode != FINISH_LOOP || was_active;
  if (reduce) {
    float2 acc0 = make_float2(0.f, 0.f), acc1 = acc0;
    for (int i0 = pb + tid; i0 < pe; i0 += 4 * 256) {
      float2 x0[4], x1[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int i = i0 + j * 256;
        x0[j] = i < pe ? a.plane_F[i] : make_float2(0.f, 0.f);
        x1[j] = i < pe ? a.plane_th[i] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc0 = pair_add(acc0, x0[j]);
        acc1 = pair_add(acc1, x1[j]);
      }
    }
    red[0][tid] = acc0;
    red[1][tid] = acc1;
    __syncthreads();
#pragma unroll
    for (int w = 128; w > 0; w >>= 1) {
      if (tid < w) {
        red[0][tid] = pair_add(red[0][tid], red[0][tid + w]);
        red[1][tid] = pair_add(red[1][tid], red[1][tid + w]);
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    const double vol = a.nd == 4 ? (double)a.lat.V : 2.0 * a.lat.V3h;
    bool act = was_active;
    if (reduce) {
      const double sF = pair_value(red[0][0]), sT = pair_value(red[1][0]);
      a.unit_sumF[u] = sF;
      a.unit_sumTh[u] = sT;
      a.unit_F[u] = sF / ((double)a.nd * 3.0 * vol);
      a.unit_theta[u] = sT / (3.0 * vol);
      if (loop && a.active) {
        act = sT / (3.0 * vol) >= eps;
        a.active[u] = act;
      }
      if (a.n_units == 1) {
        a.lat_F[0] = sF / ((double)a.nd * 3.0 * (double)a.lat.V);
        a.lat_theta[0] = sT / (3.0 * (double)a.lat.V);
      }
    }
    if (a.n_units == 1 || a.st == nullptr) {
      if (loop && a.active) {
        a.st->n_active = act ? 1 : 0;
        if (sweep >= limit) a.st->stop = 1;  // the field after the last allowed update is measured
      }
      if (a.st) a.st->ticket = 0u;
      s_last = 0;
    } else {
      __threadfence();
      s_last = atomicAdd(&a.st->ticket, 1u) == (unsigned int)(a.n_units - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid == 0) {
    double sF = 0.0, sT = 0.0;
    for (int k = 0; k < a.n_units; ++k) {
      sF += __ldcg(a.unit_sumF + k);
      sT += __ldcg(a.unit_sumTh + k);
    }
    a.lat_F[0] = sF / ((double)a.nd * 3.0 * (double)a.lat.V);
    a.lat_theta[0] = sT / (3.0 * (double)a.lat.V);
  }
  int c = 0;
  if (a.active)
    for (int k = tid; k < a.n_units; k += blockDim.x) c += __ldcg(a.active + k);
  c = __reduce_add_sync(0xffffffffu, c);
  if ((tid & 31) == 0) s_cnt[tid >> 5] = c;
  __syncthreads();
  if (tid == 0) {
    int n = 0;
    for (int w = 0; w < 8; ++w) n += s_cnt[w];
    if (loop && a.active) {
      a.st->n_active = n;
      if (sweep >= limit) a.st->stop = 1;  // the field after the last allowed update is measured
    }
    a.st->ticket = 0u;
  }
}

// Asynchronous copies of k-space elements into shared memory (8-byte complex floats,
// 16-byte complex doubles; both addresses aligned to the element).
template <class T>
__device__ __forceinline__ void cp_async_cx(cx<T>* s, const cx<T>* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  if constexpr (sizeof(cx<T>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_groups() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------------- C: FFT z(t), filter
// Item: one field, one ky, KX consecutive kx (a.kx, chosen on the host so that two items'
// columns fit in shared memory) and (Coulomb) one t.  Shared layout
// col[kxl + KX z + (KX Lz + KX) tl]: the pad keeps both transform directions free of bank
// conflicts.  Persistent blocks walk the items; with a.zt_prefetch the next item's
// columns arrive by cp.async in a second buffer while the current one is transformed.
template <class T>
__device__ __forceinline__ void column_issue(const FasdArgs& a, int nd, int kx0, int ky, int f, int t0,
                                             cx<T>* col) {
  const LatDev& lat = a.lat;
  const int Lx = lat.L[0], Lz = lat.L[2], lz = a.logL[2];
  const int KX = a.kx, lk = __ffs(KX) - 1, pitch = KX * Lz + KX;
  const int n = (nd == 4 ? lat.L[3] : 1) << (lz + lk);
  const cx<T>* kb = reinterpret_cast<const cx<T>*>(a.kbuf) + f * lat.V;
  const long long P = (long long)Lx * lat.L[1];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int kxl = i & (KX - 1), z = (i >> lk) & (Lz - 1), tl = i >> (lk + lz);
    cp_async_cx(col + kxl + KX * z + pitch * tl,
                kb + P * (z + (long long)Lz * (t0 + tl)) + (long long)Lx * ky + kx0 + kxl);
  }
}

template <class T, int ND>
__global__ void __launch_bounds__(kFasdThreads, 2) k_fasd_zt(FasdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ cx<T> twz[32], twt[32];
  __shared__ T s2x[64], s2y[64], s2z[64], s2t[64];   // 4 sin^2(pi k / L) along x, y, z, t
  if (!fasd_running(a.st)) return;
  const LatDev& lat = a.lat;
  const int Lx = lat.L[0], Ly = lat.L[1], Lz = lat.L[2], Lt = lat.L[3];
  const int lz = a.logL[2];
  const int KX = a.kx, lk = __ffs(KX) - 1, nxg = Lx / KX;
  const int nt = ND == 4 ? Lt : 1;
  const int n_items = nxg * Ly * (ND == 4 ? 4 : 4 * Lt);
  const int pitch = KX * Lz + KX;  // 2 pitch = 2 KX (Lz + 1): z-line groups split the banks evenly
  const int n = nt << (lz + lk);   // elements of an item
  cx<T>* buf[2] = {reinterpret_cast<cx<T>*>(smraw), reinterpret_cast<cx<T>*>(smraw) + pitch * nt};
  twiddles(twz, lz);
  if (ND == 4) twiddles(twt, a.logL[3]);
  for (int k = threadIdx.x; k < 64; k += blockDim.x) {
    T sn;
    if (k < Lx) { sn = sinpi((T)k / (T)Lx); s2x[k] = T(4) * sn * sn; }
    if (k < Ly) { sn = sinpi((T)k / (T)Ly); s2y[k] = T(4) * sn * sn; }
    if (k < Lz) { sn = sinpi((T)k / (T)Lz); s2z[k] = T(4) * sn * sn; }
    if (ND == 4 && k < Lt) { sn = sinpi((T)k / (T)Lt); s2t[k] = T(4) * sn * sn; }
  }
  // item -> (kx0, ky, f, t0); Coulomb items of converged slices are skipped
  auto decode = [&](int it, int& kx0, int& ky, int& f, int& t0) {
    kx0 = (it % nxg) * KX;
    const int r = it / nxg;
    ky = r % Ly;
    const int fz = r / Ly;
    f = ND == 4 ? fz : (fz & 3);
    t0 = ND == 4 ? 0 : (fz >> 2);
  };
  auto skip = [&](int it) {
    if (ND == 3 && a.active)
      while (it < n_items && !a.active[(it / (nxg * Ly)) >> 2]) it += gridDim.x;
    return it;
  };
  int it = skip((int)blockIdx.x);
  if (it >= n_items) return;
  int kx0, ky, f, t0;
  decode(it, kx0, ky, f, t0);
  int cur = 0;
  column_issue<T>(a, ND, kx0, ky, f, t0, buf[0]);
  cp_async_commit_group();
  cp_async_wait_all_groups();
  __syncthreads();
  const T coef = (T)a.coef;
  const int lf = ND == 4 ? a.logL[3] : lz;  // the direction transformed last
  const int mz = Lz - 1, mk = KX - 1;
  const long long P = (long long)Lx * Ly;
  while (it < n_items) {
    const int itn = skip(it + (int)gridDim.x);
    int kx0n = 0, kyn = 0, fn = 0, t0n = 0;
    if (itn < n_items) decode(itn, kx0n, kyn, fn, t0n);
    if (a.zt_prefetch && itn < n_items) column_issue<T>(a, ND, kx0n, kyn, fn, t0n, buf[cur ^ 1]);
    cp_async_commit_group();
    cx<T>* col = buf[cur];
    const T pxy = s2y[ky];
    if (lf <= 5 && lz <= 5) {
      // lines through registers (zt_line), one transform per pass: Landau z forward, t
      // forward and filtered, t back, z back; Coulomb z forward and filtered, z back
#pragma unroll 1
      for (int ph = ND == 4 ? 0 : 1; ph < (ND == 4 ? 4 : 3); ++ph) {
        const bool zl = ND == 4 && (ph == 0 || ph == 3);  // z lines (kxl, tl) of a Landau item
        const int nl = zl ? nt * KX : (ND == 4 ? Lz * KX : KX);
        const int lg = zl ? lz : lf;
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
          cx<T>* p = col + l;
          int es = KX;
          T base = T(0);
          const T* s2 = ND == 4 ? s2t : s2z;
          if (zl) {
            p = col + (l & mk) + (l >> lk) * pitch;
          } else if (ND == 4) {  // t line (kxl, kz)
            es = pitch;
            base = s2x[kx0 + (l & mk)] + pxy + s2z[l >> lk];
          } else {  // z line kxl of the slice
            base = s2x[kx0 + l] + pxy;
          }
          switch (lg) {
            case 1: zt_line<T, 1>(p, es, ph, base, s2, coef); break;
            case 2: zt_line<T, 2>(p, es, ph, base, s2, coef); break;
            case 3: zt_line<T, 3>(p, es, ph, base, s2, coef); break;
            case 4: zt_line<T, 4>(p, es, ph, base, s2, coef); break;
            default: zt_line<T, 5>(p, es, ph, base, s2, coef); break;
          }
        }
        __syncthreads();
      }
    } else {
      fft_lines_reg(col, twz, nt * KX, lz, KX, 1, pitch, KX, -1);          // along z
      if (ND == 4) fft_lines_reg(col, twt, Lz * KX, a.logL[3], Lz * KX, 1, 0, pitch, -1);  // along t
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int kxl = i & mk, kz = (i >> lk) & mz, kt = i >> (lk + lz);
        T p2 = s2x[kx0 + kxl] + pxy + s2z[kz];
        if (ND == 4) p2 += s2t[kt];
        const T fac = p2 > T(0) ? coef / p2 : T(0);
        const int c = kxl + KX * kz + pitch * kt;
        col[c] = cscale(col[c], fac);
      }
      __syncthreads();
      if (ND == 4) fft_lines_reg(col, twt, Lz * KX, a.logL[3], Lz * KX, 1, 0, pitch, +1);
      fft_lines_reg(col, twz, nt * KX, lz, KX, 1, pitch, KX, +1);
    }
    cx<T>* kb = reinterpret_cast<cx<T>*>(a.kbuf) + f * lat.V;
#pragma unroll 8
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int kxl = i & mk, z = (i >> lk) & mz, tl = i >> (lk + lz);
      kb[P * (z + (long long)Lz * (t0 + tl)) + (long long)Lx * ky + kx0 + kxl] = col[kxl + KX * z + pitch * tl];
    }
    if (!a.zt_prefetch && itn < n_items) {
      __syncthreads();  // every thread is done with the single buffer
      column_issue<T>(a, ND, kx0n, kyn, fn, t0n, buf[cur]);
      cp_async_commit_group();
    }
    cp_async_wait_all_groups();
    __syncthreads();
    if (a.zt_prefetch) cur ^= 1;
    it = itn;
    kx0 = kx0n; ky = kyn; f = fn; t0 = t0n;
  }
}

// ------------------------------------------------------------------------- D: inverse xy, g
// Start the copies of one (z, t) plane of the four k-space fields into pl[4][Ly][pitch].
template <class T>
__device__ __forceinline__ void plane_issue(const FasdArgs& a, int plane, cx<T>* pl) {
  const LatDev& lat = a.lat;
  const int Lx = lat.L[0], Ly = lat.L[1], P = Lx * Ly, pitch = Lx + 1;
  const cx<T>* kb = reinterpret_cast<const cx<T>*>(a.kbuf) + (long long)P * plane;
  for (int i = threadIdx.x; i < 4 * P; i += blockDim.x) {
    const int f = i >> (a.logL[0] + a.logL[1]), j = i & (P - 1);
    cp_async_cx(pl + (f * Ly + (j >> a.logL[0])) * pitch + (j & (Lx - 1)), kb + f * lat.V + j);
  }
}

// Persistent blocks walk the (z, t) planes (plane = z + Lz t; Coulomb: the active slices'
// only); with a.xy_prefetch the next plane's k-space arrives by cp.async in a second
// buffer while the current one is transformed, so the copies' latency hides behind the
// transforms.
template <int S, int ND>
__global__ void __launch_bounds__(kFasdThreads, S == GF_FP64_18 ? 2 : 3) k_fasd_xy_inv_g(FasdArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ cx<T> twx[32], twy[32];
  if (!fasd_running(a.st)) return;
  const LatDev& lat = a.lat;
  const int Lx = lat.L[0], Ly = lat.L[1], P = Lx * Ly;
  const int pitch = Lx + 1;
  const int n_planes = lat.L[2] * lat.L[3];
  cx<T>* buf[2] = {reinterpret_cast<cx<T>*>(smraw), reinterpret_cast<cx<T>*>(smraw) + 4 * Ly * pitch};
  twiddles(twx, a.logL[0]);
  twiddles(twy, a.logL[1]);
  auto skip = [&](int p) {  // first plane >= p of this block's stride that needs work
    if (ND == 3 && a.active)
      while (p < n_planes && !a.active[p >> a.logL[2]]) p += gridDim.x;
    return p;
  };
  int p = skip((int)blockIdx.x);
  if (p >= n_planes) return;
  int cur = 0;
  plane_issue<T>(a, p, buf[0]);
  cp_async_commit_group();
  cp_async_wait_all_groups();
  __syncthreads();
  while (p < n_planes) {
    const int pn = skip(p + (int)gridDim.x);
    if (a.xy_prefetch && pn < n_planes) plane_issue<T>(a, pn, buf[cur ^ 1]);
    cp_async_commit_group();
    cx<T>* pl = buf[cur];
    fft_lines_reg(pl, twy, 4 * Lx, a.logL[1], Lx, 1, Ly * pitch, pitch, +1);
    fft_lines_reg(pl, twx, 4 * Ly, a.logL[0], 1, 0, pitch, 1, +1);
    const long long plane0 = (long long)P * p;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
      const int x = i & (Lx - 1), y = i >> a.logL[0];
      // Delta~ (already scaled by alpha/2 p^2_max/p^2/N): anti-Hermitian, traceless
      const int r = y * pitch + x, fs = Ly * pitch;
      cx<T> g[9];
      g_from_delta<T>(pl[r], pl[fs + r], pl[2 * fs + r], pl[3 * fs + r], g);
      g_store<T>(a.gbuf, lat.V, plane0 + i, g);
    }
    if (!a.xy_prefetch && pn < n_planes) {
      __syncthreads();  // every thread is done with the single buffer
      plane_issue<T>(a, pn, buf[cur]);
      cp_async_commit_group();
    }
    cp_async_wait_all_groups();
    __syncthreads();
    if (a.xy_prefetch) cur ^= 1;
    p = pn;
  }
}

// ------------------------------------------------------------------------- E: update
// One site per thread in lexicographic order, so a block's forward neighbours lie in its
// own and the next planes, whose g the previous kernel has just written (L2 hits).
template <int S, int ND>
__global__ void __launch_bounds__(128) k_fasd_update(FasdArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  constexpr int NE = St::NE;
  if (!fasd_running(a.st)) return;
  const LatDev& lat = a.lat;
  const bool reunit_now = a.st ? state_reunit_sweep(a.st) : a.reunit != 0;
  char* base = a.links + lat.off_bytes;
  const long long s0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s0 < lat.V) {
    Site s;
    s.lexi = s0;
    s.x = (int)(s0 & (lat.L[0] - 1));                        // Lx, Ly, Lz are powers of 2
    s.y = (int)((s0 >> a.logL[0]) & (lat.L[1] - 1));
    s.z = (int)((s0 >> (a.logL[0] + a.logL[1])) & (lat.L[2] - 1));
    s.t = (int)(s0 >> (a.logL[0] + a.logL[1] + a.logL[2]));
    const int p = (s.x + s.y + s.z + s.t) & 1;
    const int idx = p * lat.Vh + (int)(s0 >> 1);
    // Coulomb gauge with per-slice masks: g = 1 on the sites of a converged slice, so its
    // spatial links stay as they are while a temporal link into an active slice still
    // takes that slice's g(x + t)^+ on the right
    bool act = true, act_next = true;
    if (ND == 3 && a.active) {
      act = a.active[s.t] != 0;
      act_next = a.active[s.t == lat.L[3] - 1 ? 0 : s.t + 1] != 0;
    }
    if (act || act_next) {
      cx<T> g[9];
      if (act) g_load<T, NE == 9>(a.gbuf, lat.V, s0, g);  // left_mul of 12-real links reads rows 0, 1
#pragma unroll 1
      for (int mu = 0; mu < 4; ++mu) {
        const bool act_fwd = mu == 3 ? act_next : act;
        if (!act && !act_fwd) continue;
        cx<T> u[NE], gn[9];
        St::load(base, lat.V, mu, idx, u);
        if (act) left_mul(g, u);
        if (act_fwd) {
          g_load<T, true>(a.gbuf, lat.V, fwd_lexi(lat, s, mu), gn);
          right_mul_dag(u, gn);
        }
        if (reunit_now) reunit(u);
        St::store(base, lat.V, mu, idx, u);
      }
    }
  }
  // the last block counts the iteration (every block read the state before any count)
  if (a.st == nullptr || a.active == nullptr) return;
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&a.st->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  for (int u = threadIdx.x; u < a.n_units; u += blockDim.x)
    if (a.active[u]) a.iters[u] += 1;
  if (threadIdx.x == 0) {
    a.st->ticket = 0u;
    a.st->sweep += 1;
  }
}

}  // namespace gf
