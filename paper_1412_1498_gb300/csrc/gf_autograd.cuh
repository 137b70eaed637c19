// gf_autograd.cuh -- F_U[g] and theta as functions of the Lie-algebra parameters of g,
// and their gradient (the backward of an autograd function), FP64.
//
// g(x) = exp(i X(x)), X = sum_a c_a(x) lambda_a (Gell-Mann); U^g_mu(x) = g(x) U_mu(x)
// g(x+mu)^+ (Eq. (1)'s transformed links); F(c) = Eq. (1), theta(c) = Eqs. (2)-(3) of U^g.
//
// Gradient.  With Y = i X and L(Y, E) the Frechet derivative of exp at Y in direction E,
// dg(x) = L(Y(x), i dc_a lambda_a), and Tr[L(Y, E) M] = Tr[E L(Y, M)], so
//   dL/dc_a(x) = Re Tr[i lambda_a L(Y(x), E(x))],
//   E(x) = F_bar / (nd Nc V) * K(x)  -  theta_bar * 4 / (Nc V) * M(x),
// where K(x) = sum_mu U_mu(x) g(x+mu)^+ + U_mu(x-mu)^+ g(x-mu)^+ is Eq. (5) and, with
// B_nu(y) = Delta(y+nu) - Delta(y) the adjoint of link U^g_nu(y) in theta,
//   M(x) = sum_nu U_nu(x) g(x+nu)^+ B_nu(x) - U_nu(x-nu)^+ g(x-nu)^+ B_nu(x-nu).
// The backward recomputes g, the transformed links and Delta from c and U (nothing is
// kept from the forward pass).  exp and L(Y, E) come from one scaling-and-squaring
// Taylor evaluation of the block matrix [[Y, E], [0, Y]] (its exponential is
// [[e^Y, L(Y, E)], [0, e^Y]]), after Al-Mohy and Higham (2009).
#pragma once

#include "gf_kernels.cuh"

namespace gf {



__device__ __forceinline__ void m3_mul(const c64* A, const c64* B, c64* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      c64 acc = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cadd(acc, cmul(A[3 * i + k], B[3 * k + j]));
      C[3 * i + j] = acc;
    }
}
// C = A B^+
__device__ __forceinline__ void m3_mul_dag(const c64* A, const c64* B, c64* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      c64 acc = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cadd(acc, cmul(A[3 * i + k], cconj(B[3 * j + k])));
      C[3 * i + j] = acc;
    }
}
// C = A^+ B
__device__ __forceinline__ void m3_dag_mul(const c64* A, const c64* B, c64* C) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      c64 acc = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cadd(acc, cmul(cconj(A[3 * k + i]), B[3 * k + j]));
      C[3 * i + j] = acc;
    }
}

// Y = i sum_a c_a lambda_a
__device__ __forceinline__ void lie_to_Y(const double* c, c64* Y) {
  const double s3 = 0.57735026918962576451;  // 1/sqrt(3)
  // X = sum c_a lambda_a (Hermitian)
  c64 X[9];
  X[0] = {c[2] + s3 * c[7], 0.0};
  X[4] = {-c[2] + s3 * c[7], 0.0};
  X[8] = {-2.0 * s3 * c[7], 0.0};
  X[1] = {c[0], -c[1]};
  X[3] = {c[0], c[1]};
  X[2] = {c[3], -c[4]};
  X[6] = {c[3], c[4]};
  X[5] = {c[5], -c[6]};
  X[7] = {c[5], c[6]};
#pragma unroll
  for (int e = 0; e < 9; ++e) Y[e] = {-X[e].im, X[e].re};
}

// exp(Y) and, when E != nullptr, L(Y, E): scaling by 2^-s, Taylor of degree 16 on the
// block matrix, s squarings (e^{2Z} = e^Z e^Z, L(2Z, 2W) = e^Z L + L e^Z).
__device__ void expm_frechet(const c64* Y, const c64* E, c64* expY, c64* L) {
  double nrm = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double r = 0.0;
#pragma unroll
    for (int j = 0; j < 3; ++j) r += sqrt(cnorm2(Y[3 * i + j]));
    nrm = fmax(nrm, r);
  }
  int s = 0;
  while (nrm > 0.25 && s < 60) {
    nrm *= 0.5;
    ++s;
  }
  const double sc = ldexp(1.0, -s);
  c64 Ys[9], Es[9], P[9], Q[9], SP[9], SQ[9], T1[9], T2[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    Ys[e] = cscale(Y[e], sc);
    Es[e] = E ? cscale(E[e], sc) : c64{0.0, 0.0};
    P[e] = {0.0, 0.0};
    Q[e] = {0.0, 0.0};
  }
  P[0] = P[4] = P[8] = {1.0, 0.0};
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    SP[e] = P[e];
    SQ[e] = Q[e];
  }
  // T_k = B T_{k-1} / k on [[Ys, Es], [0, Ys]]: P_k = Ys P / k, Q_k = (Ys Q + Es P) / k
#pragma unroll 1
  for (int k = 1; k <= 16; ++k) {
    m3_mul(Ys, P, T1);
    if (E) {
      m3_mul(Ys, Q, T2);
      c64 T3[9];
      m3_mul(Es, P, T3);
#pragma unroll
      for (int e = 0; e < 9; ++e) Q[e] = cscale(cadd(T2[e], T3[e]), 1.0 / k);
    }
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      P[e] = cscale(T1[e], 1.0 / k);
      SP[e] = cadd(SP[e], P[e]);
      if (E) SQ[e] = cadd(SQ[e], Q[e]);
    }
  }
#pragma unroll 1
  for (int k = 0; k < s; ++k) {
    if (E) {
      m3_mul(SP, SQ, T1);
      m3_mul(SQ, SP, T2);
#pragma unroll
      for (int e = 0; e < 9; ++e) SQ[e] = cadd(T1[e], T2[e]);
    }
    m3_mul(SP, SP, T1);
#pragma unroll
    for (int e = 0; e < 9; ++e) SP[e] = T1[e];
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) {
    expY[e] = SP[e];
    if (L) L[e] = SQ[e];
  }
}

__device__ __forceinline__ void load_link(const AdArgs& a, long long lexi, int mu, c64* u) {
  cx<double> e[9];
  Store<GF_FP64_18>::load(a.links + a.lat.off_bytes, a.lat.V, mu, idx_from_lexi(a.lat, lexi), e);
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = e[k];
}

// U^g_nu(y) = g(y) U_nu(y) g(y+nu)^+
__device__ __forceinline__ void gauge_link(const AdArgs& a, long long y, int nu, c64* out) {
  c64 u[9], t[9];
  load_link(a, y, nu, u);
  m3_mul(a.g + 9 * y, u, t);
  m3_mul_dag(t, a.g + 9 * lexi_step(a.lat, y, nu, +1), out);
}

// Delta of the transformed field at site x (Eq. (3))
__device__ __forceinline__ void delta_g(const AdArgs& a, long long x, c64* D, double* Fsite) {
  c64 A[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) A[e] = {0.0, 0.0};
  double f = 0.0;
#pragma unroll 1
  for (int nu = 0; nu < a.nd; ++nu) {
    c64 fw[9], bw[9];
    gauge_link(a, x, nu, fw);
    gauge_link(a, lexi_step(a.lat, x, nu, -1), nu, bw);
    f += fw[0].re + fw[4].re + fw[8].re;
#pragma unroll
    for (int e = 0; e < 9; ++e) A[e] = cadd(A[e], csub(bw[e], fw[e]));
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) D[3 * i + j] = csub(A[3 * i + j], cconj(A[3 * j + i]));
  const c64 sum = cadd(cadd(D[0], D[4]), D[8]);
  const c64 tr = {sum.re / 3.0, sum.im / 3.0};
  D[0] = csub(D[0], tr);
  D[4] = csub(D[4], tr);
  D[8] = csub(D[8], tr);
  if (Fsite) *Fsite = f;
}

}  // namespace gf
