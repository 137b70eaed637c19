// gf_split.cuh -- the double-float ("split FP32") polish of the mixed-precision fix.
//
// Near convergence every site update g(x) of Algorithm 1 is close to the identity, so a
// sweep can keep links at about 48-bit precision without FP64 arithmetic, which issues
// at a small fraction of the FP32 rate on this GPU:
//
//  - each real number is an unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2);
//    a link is 9 float4 words (hi.re, hi.im, lo.re, lo.im), 144 bytes, in the plane
//    layout of the FP64-18 storage;
//  - K(x) (Eq. (5), in-place form) is summed with error-free transformations (TwoSum),
//    so its small anti-Hermitian part -- the part the subgroup maximisers react to --
//    is exact to ~2^-48;
//  - each SU(2) subgroup maximiser R (Eq. (6), first-order overrelaxation) is formed
//    directly as its deviation eps = R - 1 from closed forms without cancellation
//    (a quaternion's a0 - 1 = -|a_vec|^2 / (1 + a0)), in FP32 with relative error
//    ~1e-7 of eps;
//  - g(x) = 1 + E is accumulated as E in FP32 and applied as U <- U + E U, the small
//    product added to the split link with TwoSum: the update carries FP32 relative
//    error of E, i.e. ~1e-7 |E|, far below the link precision needed for theta < 1e-15
//    (links to ~1e-10 suffice there);
//  - reunitarisation uses exact products (TwoProd with FMA) so that rows stay
//    orthonormal and row 2 = conj(row0 x row1) to ~1e-15.
//
// Only the first-order overrelaxation form is implemented here.
#pragma once

#include "gf_kernels.cuh"

namespace gf {

struct sf {  // hi + lo
  float hi, lo;
};
struct csf {
  sf re, im;
};

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ sf sf_add(sf a, sf b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = e + (a.lo + b.lo);
  sf r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ sf sf_neg(sf a) { return {-a.hi, -a.lo}; }
// a + small float correction
__device__ __forceinline__ sf sf_add_f(sf a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e = e + a.lo;
  sf r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ sf sf_mul(sf a, sf b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  sf r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ float sf_f(sf a) { return a.hi + a.lo; }

__device__ __forceinline__ csf csf_add(csf a, csf b) { return {sf_add(a.re, b.re), sf_add(a.im, b.im)}; }
__device__ __forceinline__ csf csf_sub(csf a, csf b) { return {sf_add(a.re, sf_neg(b.re)), sf_add(a.im, sf_neg(b.im))}; }
__device__ __forceinline__ csf csf_conj(csf a) { return {a.re, sf_neg(a.im)}; }
__device__ __forceinline__ csf csf_mul(csf x, csf y) {
  return {sf_add(sf_mul(x.re, y.re), sf_neg(sf_mul(x.im, y.im))), sf_add(sf_mul(x.re, y.im), sf_mul(x.im, y.re))};
}
__device__ __forceinline__ cx<float> csf_hi(csf a) { return {a.re.hi, a.im.hi}; }
__device__ __forceinline__ cx<float> csf_f(csf a) { return {sf_f(a.re), sf_f(a.im)}; }
// a + small complex correction
__device__ __forceinline__ csf csf_add_c(csf a, cx<float> b) { return {sf_add_f(a.re, b.re), sf_add_f(a.im, b.im)}; }

// ------------------------------------------------------------------------- storage
__device__ __forceinline__ void split_load(const char* base, long long V, int mu, int idx, csf (&u)[9]) {
  const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
  for (int w = 0; w < 9; ++w) {
    const float4 v = p[(long long)(w * 4 + mu) * V + idx];
    u[w] = {{v.x, v.z}, {v.y, v.w}};
  }
}
__device__ __forceinline__ void split_store(char* base, long long V, int mu, int idx, const csf (&u)[9]) {
  float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
  for (int w = 0; w < 9; ++w) p[(long long)(w * 4 + mu) * V + idx] = make_float4(u[w].re.hi, u[w].im.hi, u[w].re.lo, u[w].im.lo);
}
// Apply phase: the reload of a link is the last use of its line and the store streams
// out (cache hints ld.global.lu / st.global.cs), so the updated links do not evict the
// lines that other blocks loaded for their K phase and will reload: 0.537 -> 0.495 ms
// per 32^4 polish sweep.
__device__ __forceinline__ void split_load_last(const char* base, long long V, int mu, int idx, csf (&u)[9]) {
  const float4* p = reinterpret_cast<const float4*>(base);
#pragma unroll
  for (int w = 0; w < 9; ++w) {
    const float4 v = __ldlu(p + (long long)(w * 4 + mu) * V + idx);
    u[w] = {{v.x, v.z}, {v.y, v.w}};
  }
}
__device__ __forceinline__ void split_store_stream(char* base, long long V, int mu, int idx, const csf (&u)[9]) {
  float4* p = reinterpret_cast<float4*>(base);
#pragma unroll
  for (int w = 0; w < 9; ++w) __stcs(p + (long long)(w * 4 + mu) * V + idx, make_float4(u[w].re.hi, u[w].im.hi, u[w].re.lo, u[w].im.lo));
}
__device__ __forceinline__ csf split_of(double re, double im) {
  const float rh = (float)re, ih = (float)im;
  return {{rh, (float)(re - (double)rh)}, {ih, (float)(im - (double)ih)}};
}

// ------------------------------------------------------------------------- K(x)
// accumulator: hi parts with TwoSum, low parts plain; renormalised when read
struct acc2 {
  float hi, lo;
};
__device__ __forceinline__ void acc_add(acc2& a, float xh, float xl) {
  float s, e;
  two_sum(a.hi, xh, s, e);
  a.hi = s;
  a.lo = a.lo + (e + xl);
}

// ------------------------------------------------------------------------- SU(2) step
// Deviation eps = R - 1 of the first-order overrelaxed maximiser in subgroup (i, j):
// returns (a'' - 1, b'') with R|_(i,j) = [[a'', b''], [-conj b'', conj a'']].
__device__ __forceinline__ void su2_deviation(float are, float aim, float bre, float bim, float omega,
                                              cx<float>& am1, cx<float>& b) {
  // alpha = are + i aim, beta = bre + i bim
  const float n2 = are * are + aim * aim + bre * bre + bim * bim;
  am1 = {0.f, 0.f};
  b = {0.f, 0.f};
  if (!(n2 > 0.f)) return;
  const float rn = rsqrtf(n2), n = n2 * rn;
  // a = conj(alpha)/n: a.re - 1 = -(aim^2 + |beta|^2) / (n (n + are)) when are > 0
  const float side = aim * aim + bre * bre + bim * bim;
  const float d = are > 0.f ? -side / (n * (n + are)) : are * rn - 1.f;
  const float ai = -aim * rn;
  const float br = bre * rn, bi = -bim * rn;
  // first-order g^omega: a1 - 1 = omega d, a1.im = omega ai, b1 = omega b; then 1/m
  const float v2 = ai * ai + br * br + bi * bi;
  const float dm = omega * (omega - 1.f) * (d * d + v2);     // m^2 - 1
  const float sq = sqrtf(1.f + dm);
  const float rm1 = -dm / (sq * (1.f + sq));                 // 1/m - 1
  const float od = omega * d;
  am1 = {od + rm1 + od * rm1, omega * ai * (1.f + rm1)};
  b = {omega * br * (1.f + rm1), omega * bi * (1.f + rm1)};
}

// ------------------------------------------------------------------------- reunitarisation
// |x|^2 - 1 of a split complex row, accurate for rows close to unit length
__device__ __forceinline__ float row_norm2_m1(const csf* r) {
  float s = -1.f, lo = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float p, e, t, f;
    two_prod(r[k].re.hi, r[k].re.hi, p, e);
    two_sum(s, p, t, f);
    s = t;
    lo += e + f + 2.f * r[k].re.hi * r[k].re.lo;
    two_prod(r[k].im.hi, r[k].im.hi, p, e);
    two_sum(s, p, t, f);
    s = t;
    lo += e + f + 2.f * r[k].im.hi * r[k].im.lo;
  }
  return s + lo;
}
// conj(a) . b for rows that are nearly orthogonal (result small), with exact products
__device__ __forceinline__ cx<float> row_dot_small(const csf* a, const csf* b) {
  float re = 0.f, rl = 0.f, im = 0.f, il = 0.f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const sf ar = a[k].re, ai = a[k].im, br = b[k].re, bi = b[k].im;
    float p, e, t, f;
    // re += ar br + ai bi ; im += ar bi - ai br
    two_prod(ar.hi, br.hi, p, e); two_sum(re, p, t, f); re = t; rl += e + f + ar.hi * br.lo + ar.lo * br.hi;
    two_prod(ai.hi, bi.hi, p, e); two_sum(re, p, t, f); re = t; rl += e + f + ai.hi * bi.lo + ai.lo * bi.hi;
    two_prod(ar.hi, bi.hi, p, e); two_sum(im, p, t, f); im = t; il += e + f + ar.hi * bi.lo + ar.lo * bi.hi;
    two_prod(ai.hi, br.hi, p, e); two_sum(im, -p, t, f); im = t; il += -e + f - ai.hi * br.lo - ai.lo * br.hi;
  }
  return {re + rl, im + il};
}
__device__ __forceinline__ void split_reunit(csf (&u)[9]) {
  // row 0: scale by 1/sqrt(1 + d) = 1 - d/2 + 3 d^2 / 8
  float d = row_norm2_m1(u);
  float c = -0.5f * d + 0.375f * d * d;
#pragma unroll
  for (int k = 0; k < 3; ++k) u[k] = csf_add_c(u[k], cscale(csf_hi(u[k]), c));
  // row 1 -= (conj(row0) . row1) row0, then normalise
  const cx<float> p = row_dot_small(u, u + 3);
#pragma unroll
  for (int k = 0; k < 3; ++k) u[3 + k] = csf_add_c(u[3 + k], cneg(cmul(p, csf_hi(u[k]))));
  d = row_norm2_m1(u + 3);
  c = -0.5f * d + 0.375f * d * d;
#pragma unroll
  for (int k = 0; k < 3; ++k) u[3 + k] = csf_add_c(u[3 + k], cscale(csf_hi(u[3 + k]), c));
  // row 2 = conj(row0 x row1), exact products
  u[6] = csf_conj(csf_sub(csf_mul(u[1], u[5]), csf_mul(u[2], u[4])));
  u[7] = csf_conj(csf_sub(csf_mul(u[2], u[3]), csf_mul(u[0], u[5])));
  u[8] = csf_conj(csf_sub(csf_mul(u[0], u[4]), csf_mul(u[1], u[3])));
}

// ------------------------------------------------------------------------- theta per site
// A = sum_nu U_nu(x - nu) - U_nu(x) is O(1); Delta = A - A^+ - tr/3 is small, so A is
// summed in split precision and Delta formed from its parts.
__device__ __forceinline__ void split_add_to_A(acc2 (&A)[18], const csf (&f)[9], const csf (&b)[9]) {
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    acc_add(A[2 * e], b[e].re.hi, b[e].re.lo);
    acc_add(A[2 * e], -f[e].re.hi, -f[e].re.lo);
    acc_add(A[2 * e + 1], b[e].im.hi, b[e].im.lo);
    acc_add(A[2 * e + 1], -f[e].im.hi, -f[e].im.lo);
  }
}
__device__ __forceinline__ float split_theta_site(const acc2 (&A)[18]) {
  cx<float> D[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // D_ij = A_ij - conj(A_ji): hi differences are exact when the result is small
      const acc2 ar = A[2 * (3 * i + j)], ai = A[2 * (3 * i + j) + 1];
      const acc2 br = A[2 * (3 * j + i)], bi = A[2 * (3 * j + i) + 1];
      D[3 * i + j] = {(ar.hi - br.hi) + (ar.lo - br.lo), (ai.hi + bi.hi) + (ai.lo + bi.lo)};
    }
  const cx<float> sum = cadd(cadd(D[0], D[4]), D[8]);
  const cx<float> tr = {sum.re / 3.f, sum.im / 3.f};
  D[0] = csub(D[0], tr);
  D[4] = csub(D[4], tr);
  D[8] = csub(D[8], tr);
  float q = 0.f;
#pragma unroll
  for (int e = 0; e < 9; ++e) q = q + (D[e].re * D[e].re + D[e].im * D[e].im);
  return q;
}

// ------------------------------------------------------------------------- the sweep
template <int ND>
__global__ void __launch_bounds__(256) k_or_sweep_split(SweepArgs a) {
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
  float q = 0.f, fsum = 0.f;
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
    const float omega = (float)a.omega;

    // K = sum_{mu<nd} U_mu(x) + U_mu(x-mu)^+ with TwoSum on the hi parts
    acc2 K[18];
#pragma unroll
    for (int e = 0; e < 18; ++e) K[e] = {0.f, 0.f};
#pragma unroll 1
    for (int mu = 0; mu < ND; ++mu) {
      csf f[9], b[9];
      split_load(base, V, mu, idx_f, f);
      split_load(base, V, mu, idx_b[mu], b);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const csf x = f[3 * r + c], y = b[3 * c + r];  // + conj(y)
          acc_add(K[2 * (3 * r + c)], x.re.hi, x.re.lo);
          acc_add(K[2 * (3 * r + c)], y.re.hi, y.re.lo);
          acc_add(K[2 * (3 * r + c) + 1], x.im.hi, x.im.lo);
          acc_add(K[2 * (3 * r + c) + 1], -y.im.hi, -y.im.lo);
        }
    }
    // three subgroup steps; E = g - 1 accumulated in FP32
    cx<float> E[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) E[e] = {0.f, 0.f};
    const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int i = pi[k], j = pj[k];
      // alpha = K_ii + conj(K_jj), beta = K_ji - conj(K_ij), small parts from split sums
      const acc2 kii_r = K[2 * (4 * i)], kii_i = K[2 * (4 * i) + 1];
      const acc2 kjj_r = K[2 * (4 * j)], kjj_i = K[2 * (4 * j) + 1];
      const acc2 kji_r = K[2 * (3 * j + i)], kji_i = K[2 * (3 * j + i) + 1];
      const acc2 kij_r = K[2 * (3 * i + j)], kij_i = K[2 * (3 * i + j) + 1];
      const float are = (kii_r.hi + kjj_r.hi) + (kii_r.lo + kjj_r.lo);
      const float aim = (kii_i.hi - kjj_i.hi) + (kii_i.lo - kjj_i.lo);
      const float bre = (kji_r.hi - kij_r.hi) + (kji_r.lo - kij_r.lo);
      const float bim = (kji_i.hi + kij_i.hi) + (kji_i.lo + kij_i.lo);
      cx<float> am1, bb;
      su2_deviation(are, aim, bre, bim, omega, am1, bb);
      const cx<float> mbc = cneg(cconj(bb));                       // eps_ji
      const cx<float> cam1 = {am1.re, -am1.im};                    // eps_jj = conj(a) - 1
      // K <- K + eps K (rows i, j), eps K from the hi parts
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cx<float> ki = {K[2 * (3 * i + c)].hi, K[2 * (3 * i + c) + 1].hi};
        const cx<float> kj = {K[2 * (3 * j + c)].hi, K[2 * (3 * j + c) + 1].hi};
        const cx<float> di = cadd(cmul(am1, ki), cmul(bb, kj));
        const cx<float> dj = cadd(cmul(mbc, ki), cmul(cam1, kj));
        acc_add(K[2 * (3 * i + c)], di.re, 0.f);
        acc_add(K[2 * (3 * i + c) + 1], di.im, 0.f);
        acc_add(K[2 * (3 * j + c)], dj.re, 0.f);
        acc_add(K[2 * (3 * j + c) + 1], dj.im, 0.f);
      }
      // E <- E + eps (1 + E) on rows i, j
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cx<float> ei = E[3 * i + c], ej = E[3 * j + c];
        cx<float> ni = cadd(ei, cadd(cmul(am1, ei), cmul(bb, ej)));
        cx<float> nj = cadd(ej, cadd(cmul(mbc, ei), cmul(cam1, ej)));
        if (c == i) { ni = cadd(ni, am1); nj = cadd(nj, mbc); }
        if (c == j) { ni = cadd(ni, bb); nj = cadd(nj, cam1); }
        E[3 * i + c] = ni;
        E[3 * j + c] = nj;
      }
    }
    // apply g = 1 + E: U_mu(x) += E U_mu(x);  U_mu(x-mu) += U_mu(x-mu) E^+
    acc2 A[18];
#pragma unroll
    for (int e = 0; e < 18; ++e) A[e] = {0.f, 0.f};
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      // forward link: U_mu(x) += E U_mu(x); then backward: U_mu(x-mu) += U_mu(x-mu) E^+
      // (one split link live at a time)
      float tr[2] = {0.f, 0.f};
#pragma unroll 1
      for (int side = 0; side < 2; ++side) {
        const int idx = side == 0 ? idx_f : idx_b[mu];
        csf u[9];
        split_load_last(base, V, mu, idx, u);
        cx<float> du[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            cx<float> x = {0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 3; ++k)
              x = side == 0 ? cadd(x, cmul(E[3 * r + k], csf_hi(u[3 * k + c])))
                            : cadd(x, cmul(csf_hi(u[3 * r + k]), cconj(E[3 * c + k])));
            du[3 * r + c] = x;
          }
#pragma unroll
        for (int e = 0; e < 9; ++e) u[e] = csf_add_c(u[e], du[e]);
        if (reunit_now) split_reunit(u);
        if (mu < ND && measure_now) {
          // A += U_nu(x - nu) - U_nu(x)
#pragma unroll
          for (int e = 0; e < 9; ++e) {
            const float sg = side == 0 ? -1.f : 1.f;
            acc_add(A[2 * e], sg * u[e].re.hi, sg * u[e].re.lo);
            acc_add(A[2 * e + 1], sg * u[e].im.hi, sg * u[e].im.lo);
          }
          tr[side] = sf_f(u[0].re) + sf_f(u[4].re) + sf_f(u[8].re);
        }
        split_store_stream(base, V, mu, idx, u);
      }
      if (mu < ND && measure_now) fsum = fsum + (tr[0] + tr[1]);
    }
    if (measure_now) q = split_theta_site(A);
  }
  if (measure_now) {
    const float v[2] = {fsum, q};
    float2 o[2];
    block_sum_f32<2>(v, o, reinterpret_cast<float*>(red));
    if (threadIdx.x == 0) {
      if (a.part_F) a.part_F[ti] = o[0];
      a.part_theta[ti] = o[1];
    }
  }
}

// ------------------------------------------------------------------------- measurement
template <int ND>
__global__ void __launch_bounds__(256) k_measure_split(MeasureArgs a) {
  __shared__ double red[64];
  if (a.st && !state_even_pass(a.st)) return;
  const int ti = a.reverse ? a.n_tiles - 1 - (int)blockIdx.x : (int)blockIdx.x;
  const int4 tile = a.tiles[ti];
  if (a.active && a.active[tile.w] != a.level) return;
  const LatDev lat = a.lats[tile.x];
  const int h3 = tile.z + (int)threadIdx.x;
  float fsum = 0.f, q = 0.f;
  if (h3 < lat.V3h) {
    const int p = a.parity;
    const int h = tile.y * lat.V3h + h3;
    const Site s = site_of_slice(lat, p, tile.y, h3);
    const char* base = a.links + lat.off_bytes;
    const int idx_f = p * lat.Vh + h;
    acc2 A[18];
#pragma unroll
    for (int e = 0; e < 18; ++e) A[e] = {0.f, 0.f};
#pragma unroll 1
    for (int nu = 0; nu < ND; ++nu) {
      csf f[9], b[9];
      split_load(base, lat.V, nu, idx_f, f);
      split_load(base, lat.V, nu, (1 - p) * lat.Vh + (int)(back_lexi(lat, s, nu) >> 1), b);
      fsum = fsum + ((sf_f(f[0].re) + sf_f(f[4].re) + sf_f(f[8].re)) + (sf_f(b[0].re) + sf_f(b[4].re) + sf_f(b[8].re)));
      split_add_to_A(A, f, b);
    }
    q = split_theta_site(A);
  }
  const float v[2] = {fsum, q};
  float2 o[2];
  block_sum_f32<2>(v, o, reinterpret_cast<float*>(red));
  if (threadIdx.x == 0) {
    if (a.part_F) a.part_F[ti] = o[0];
    a.part_theta[ti] = o[1];
  }
}

// ------------------------------------------------------------------------- conversions
// FP32 storage -> split: row 2 rebuilt and the link reunitarised in FP64 first
template <int S>
__global__ void __launch_bounds__(256) k_to_split(const char* src, char* dst, LatDev ls, LatDev ld) {
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
  csf u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = split_of(m[k].re, m[k].im);
  split_store(dst + ld.off_bytes, ld.V, mu, idx, u);
}

// split -> FP64-18 in place (same plane layout, 16 bytes per complex element), with an
// FP64 reunitarisation
__global__ void __launch_bounds__(256) k_split_to_fp64(char* links, LatDev lat) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4 * lat.V) return;
  const int mu = (int)(i / lat.V), idx = (int)(i % lat.V);
  csf u[9];
  split_load(links + lat.off_bytes, lat.V, mu, idx, u);
  cx<double> m[9];
#pragma unroll
  for (int k = 0; k < 9; ++k)
    m[k] = {(double)u[k].re.hi + (double)u[k].re.lo, (double)u[k].im.hi + (double)u[k].im.lo};
  reunit(m);
  Store<GF_FP64_18>::store(links + lat.off_bytes, lat.V, mu, idx, m);
}

}  // namespace gf
