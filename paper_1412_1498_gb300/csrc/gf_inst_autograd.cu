// gf_inst_autograd.cu -- forward and backward of F(c), theta(c) (FP64-18 storage).
#include "gf_autograd.cuh"

namespace gf {

namespace {
constexpr int kT = 128;
}

__global__ void __launch_bounds__(kT) k_ad_exp(AdArgs a) {
  const long long x = blockIdx.x * (long long)kT + threadIdx.x;
  if (x >= a.lat.V) return;
  c64 Y[9], g[9];
  lie_to_Y(a.c + 8 * x, Y);
  expm_frechet(Y, nullptr, g, nullptr);
#pragma unroll
  for (int e = 0; e < 9; ++e) a.g[9 * x + e] = g[e];
}

__global__ void __launch_bounds__(kT) k_ad_forward(AdArgs a) {
  __shared__ double red[64];
  __shared__ int s_last;
  const long long x = blockIdx.x * (long long)kT + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (x < a.lat.V) {
    c64 D[9];
    delta_g(a, x, D, &v[0]);
#pragma unroll
    for (int e = 0; e < 9; ++e) v[1] = v[1] + (D[e].re * D[e].re + D[e].im * D[e].im);
  }
  block_sum<2>(v, red);
  if (threadIdx.x == 0) {
    a.part[2 * blockIdx.x] = v[0];
    a.part[2 * blockIdx.x + 1] = v[1];
    __threadfence();
    s_last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double w[2] = {0.0, 0.0};
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += kT) {
    w[0] += __ldcg(a.part + 2 * k);
    w[1] += __ldcg(a.part + 2 * k + 1);
  }
  block_sum<2>(w, red);
  if (threadIdx.x == 0) {
    a.out[0] = w[0] / ((double)a.nd * 3.0 * (double)a.lat.V);
    a.out[1] = w[1] / (3.0 * (double)a.lat.V);
    *a.ticket = 0u;
  }
}

__global__ void __launch_bounds__(kT) k_ad_delta(AdArgs a) {
  const long long x = blockIdx.x * (long long)kT + threadIdx.x;
  if (x >= a.lat.V) return;
  c64 D[9];
  delta_g(a, x, D, nullptr);
#pragma unroll
  for (int e = 0; e < 9; ++e) a.delta[9 * x + e] = D[e];
}

__global__ void __launch_bounds__(kT) k_ad_backward(AdArgs a) {
  const long long x = blockIdx.x * (long long)kT + threadIdx.x;
  if (x >= a.lat.V) return;
  const double V = (double)a.lat.V;
  const double wF = a.upstream[0] / ((double)a.nd * 3.0 * V);
  const double wT = -a.upstream[1] * 4.0 / (3.0 * V);
  c64 E[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) E[e] = {0.0, 0.0};
#pragma unroll 1
  for (int mu = 0; mu < a.nd; ++mu) {
    const long long xp = lexi_step(a.lat, x, mu, +1), xm = lexi_step(a.lat, x, mu, -1);
    c64 u[9], t[9], t2[9], B[9];
    // U_mu(x) g(x+mu)^+  -> K and, times B_mu(x), M
    load_link(a, x, mu, u);
    m3_mul_dag(u, a.g + 9 * xp, t);
#pragma unroll
    for (int e = 0; e < 9; ++e) B[e] = csub(a.delta[9 * xp + e], a.delta[9 * x + e]);
    m3_mul(t, B, t2);
#pragma unroll
    for (int e = 0; e < 9; ++e) E[e] = cadd(E[e], cadd(cscale(t[e], wF), cscale(t2[e], wT)));
    // U_mu(x-mu)^+ g(x-mu)^+ -> K and, times B_mu(x-mu), -M
    load_link(a, xm, mu, u);
    c64 gu[9];
    m3_mul(a.g + 9 * xm, u, gu);       // g(x-mu) U_mu(x-mu)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) t[3 * i + j] = cconj(gu[3 * j + i]);   // (g U)^+
#pragma unroll
    for (int e = 0; e < 9; ++e) B[e] = csub(a.delta[9 * x + e], a.delta[9 * xm + e]);
    m3_mul(t, B, t2);
#pragma unroll
    for (int e = 0; e < 9; ++e) E[e] = cadd(E[e], csub(cscale(t[e], wF), cscale(t2[e], wT)));
  }
  c64 Y[9], g[9], L[9];
  lie_to_Y(a.c + 8 * x, Y);
  expm_frechet(Y, E, g, L);
  // grad_a = Re Tr[i lambda_a L] = -Im Tr[lambda_a L]
  const double s3 = 0.57735026918962576451;
  double* gr = a.grad + 8 * x;
  gr[0] = -(L[3].im + L[1].im);
  gr[1] = -(-L[3].re + L[1].re);
  gr[2] = -(L[0].im - L[4].im);
  gr[3] = -(L[6].im + L[2].im);
  gr[4] = -(-L[6].re + L[2].re);
  gr[5] = -(L[7].im + L[5].im);
  gr[6] = -(-L[7].re + L[5].re);
  gr[7] = -s3 * (L[0].im + L[4].im - 2.0 * L[8].im);
}

static unsigned int nblk(const AdArgs& a) { return (unsigned int)((a.lat.V + kT - 1) / kT); }

size_t ad_partial_doubles(long long V) { return 2 * (size_t)((V + kT - 1) / kT); }

void launch_ad_forward(const AdArgs& a, cudaStream_t s) {
  k_ad_exp<<<nblk(a), kT, 0, s>>>(a);
  k_ad_forward<<<nblk(a), kT, 0, s>>>(a);
}

void launch_ad_backward(const AdArgs& a, cudaStream_t s) {
  k_ad_exp<<<nblk(a), kT, 0, s>>>(a);
  k_ad_delta<<<nblk(a), kT, 0, s>>>(a);
  k_ad_backward<<<nblk(a), kT, 0, s>>>(a);
}

}  // namespace gf
