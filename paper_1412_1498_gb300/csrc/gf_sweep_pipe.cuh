// gf_sweep_pipe.cuh -- FP32-12 half-sweep with the links staged through shared memory.
//
// The register kernel (k_or_sweep) holds a site's 8 links (96 floats) in registers from
// load to store, which caps it at 8 resident warps per SM and leaves the memory system
// latency-bound.  Here each thread copies its site's 24 link words (8 links x 3 float4)
// into shared memory with cp.async, which holds no registers while in flight, one tile
// ahead of the tile it is computing (double buffer).  The CTAs are persistent: CTA c
// takes tiles c, c + gridDim, ... so that with tiles walked in reverse the whole grid
// moves through the lattice as one front.  Every thread reads back only the words it
// copied itself, so cp.async.wait_group is the only synchronisation the pipeline needs.
// The arithmetic is the register kernel's, in the same order: both give the same bits.
#pragma once

#include "gf_kernels.cuh"

namespace gf {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_newest() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

constexpr int kPipeWords = 24;  // fwd mu = 0..3 (3 words each), then bwd mu = 0..3

struct PipeSite {
  int ti;      // tile index
  int lat;     // lattice index
  int idx_f;   // parity-split index of the site
  int idx_b[4];
  bool active; // unit active (uniform over the block)
  bool valid;  // active and inside the tile's slice
};

// Start the copies of tile k into buffer buf; returns where the site's links live.
__device__ __forceinline__ PipeSite pipe_issue(const SweepArgs& a, int k, int buf, float4* sm) {
  PipeSite ps;
  ps.ti = a.reverse ? a.n_tiles - 1 - k : k;
  const int4 tile = a.tiles[ps.ti];
  ps.lat = tile.x;
  ps.active = a.active == nullptr || a.active[tile.w] == a.level;
  const LatDev lat = a.lats[tile.x];
  const int h3 = tile.z + (int)threadIdx.x;
  ps.valid = ps.active && h3 < lat.V3h;
  if (ps.valid) {
    const int p = a.parity;
    const int h = tile.y * lat.V3h + h3;
    const Site s = site_of_slice(lat, p, tile.y, h3);
    ps.idx_f = p * lat.Vh + h;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) ps.idx_b[mu] = (1 - p) * lat.Vh + (int)(back_lexi(lat, s, mu) >> 1);
    const float4* g = reinterpret_cast<const float4*>(a.links + lat.off_bytes);
    const int B = blockDim.x;
    float4* slot = sm + (buf * kPipeWords) * B + threadIdx.x;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        cp_async16(slot + (3 * mu + w) * B, g + (long long)(w * 4 + mu) * lat.V + ps.idx_f);
        cp_async16(slot + (12 + 3 * mu + w) * B, g + (long long)(w * 4 + mu) * lat.V + ps.idx_b[mu]);
      }
  }
  return ps;
}

__device__ __forceinline__ void pipe_read(const float4* slot, int B, int word0, cx<float> (&e)[6]) {
#pragma unroll
  for (int w = 0; w < 3; ++w) {
    const float4 v = slot[(word0 + w) * B];
    e[2 * w] = {v.x, v.y};
    e[2 * w + 1] = {v.z, v.w};
  }
}

template <int ND, int FORM>
__global__ void __launch_bounds__(256) k_or_sweep_pipe(SweepArgs a) {
  extern __shared__ float4 sm[];
  __shared__ double red[2][64];  // alternate per tile sum: no barrier after the sum
  grid_dep_wait();
  grid_dep_launch();
  int rb = 0;
  bool reunit_now = a.reunit != 0, measure_now = a.measure != 0;
  if (a.st) {
    if (!state_sweeping(a.st)) return;
    reunit_now = a.parity == 1 && state_reunit_sweep(a.st);
    measure_now = a.parity == 1 && state_check_sweep(a.st);
  }
  int k = blockIdx.x;
  if (k >= a.n_tiles) return;
  const int B = blockDim.x;
  const float omega = (float)a.omega;
  // with cta_sums each thread adds its sites' values over the CTA's tiles (compensated,
  // in a fixed order) and the CTA reduces once at the end: no barrier per tile
  const bool per_cta = measure_now && a.cta_sums;
  float acc_hi[2] = {0.f, 0.f}, acc_lo[2] = {0.f, 0.f};
  int buf = 0;
  PipeSite cur = pipe_issue(a, k, 0, sm);
  cp_async_commit();
  for (;;) {
    const int kn = k + (int)gridDim.x;
    PipeSite nxt;
    if (kn < a.n_tiles) nxt = pipe_issue(a, kn, buf ^ 1, sm);
    cp_async_commit();
    cp_async_wait_all_but_newest();  // this thread's copies of tile k have landed
    if (cur.active) {
      float q = 0.f, fs = 0.f;
      if (cur.valid) {
        const LatDev lat = a.lats[cur.lat];
        float4* g = reinterpret_cast<float4*>(a.links + lat.off_bytes);
        const float4* slot = sm + (buf * kPipeWords) * B + threadIdx.x;
        cx<float> K[9], G[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) K[e] = {0.f, 0.f};
#pragma unroll
        for (int mu = 0; mu < ND; ++mu) {
          cx<float> f[6], b[6];
          pipe_read(slot, B, 3 * mu, f);
          pipe_read(slot, B, 12 + 3 * mu, b);
          add_to_K(K, f, b);
        }
        su3_update<float, false, FORM>(K, G, omega, measure_now);
        if (measure_now) site_check_from_GK(K, fs, q);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          cx<float> f[6], b[6];
          pipe_read(slot, B, 3 * mu, f);
          pipe_read(slot, B, 12 + 3 * mu, b);
          left_mul(G, f);
          right_mul_dag(b, G);
          if (reunit_now) {
            reunit(f);
            reunit(b);
          }
#pragma unroll
          for (int w = 0; w < 3; ++w) {
            g[(long long)(w * 4 + mu) * lat.V + cur.idx_f] =
                make_float4(f[2 * w].re, f[2 * w].im, f[2 * w + 1].re, f[2 * w + 1].im);
            g[(long long)(w * 4 + mu) * lat.V + cur.idx_b[mu]] =
                make_float4(b[2 * w].re, b[2 * w].im, b[2 * w + 1].re, b[2 * w + 1].im);
          }
        }
      }
      if (per_cta) {
        const float v[2] = {fs, q};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          float s, e;
          two_sum(acc_hi[j], v[j], s, e);
          acc_hi[j] = s;
          acc_lo[j] = acc_lo[j] + e;
        }
      } else if (measure_now) {
        const float v[2] = {fs, q};
        float2 o[2];
        block_sum_f32<2>(v, o, reinterpret_cast<float*>(red[rb]));
        if (threadIdx.x == 0) {
          if (a.part_F) a.part_F[cur.ti] = o[0];
          a.part_theta[cur.ti] = o[1];
        }
        // red[rb] is written again two sums later, after the next sum's barrier, which
        // warp 0 reaches only once it has read this one
        rb ^= 1;
      }
    }
    if (kn >= a.n_tiles) break;
    k = kn;
    buf ^= 1;
    cur = nxt;
  }
  if (per_cta) {
    float2 o[2];
    block_sum_f32_pairs<2>(acc_hi, acc_lo, o, reinterpret_cast<float*>(red[rb]));
    if (threadIdx.x == 0) {
      if (a.part_F) a.part_F[blockIdx.x] = o[0];
      a.part_theta[blockIdx.x] = o[1];
    }
  }
}

// ----------------------------------------------------------------------------------
// FP32-12 F / theta pass (Eqs. (1)-(3)) over the sites of one parity with the same
// staging: each thread copies the 2 nd links of its site (6 nd words) one tile ahead
// and reads back only what it copied.  The per-site arithmetic and the per-tile
// reduction are k_measure's, so the tile partials are the same.
// ----------------------------------------------------------------------------------
struct MeasSite {
  int ti;
  bool active;
  bool valid;
};

template <int ND>
__device__ __forceinline__ MeasSite meas_issue(const MeasureArgs& a, int k, int buf, float4* sm) {
  MeasSite ms;
  ms.ti = a.reverse ? a.n_tiles - 1 - k : k;
  const int4 tile = a.tiles[ms.ti];
  ms.active = a.active == nullptr || a.active[tile.w] == a.level;
  const LatDev lat = a.lats[tile.x];
  const int h3 = tile.z + (int)threadIdx.x;
  ms.valid = ms.active && h3 < lat.V3h;
  if (ms.valid) {
    const int p = a.parity;
    const Site s = site_of_slice(lat, p, tile.y, h3);
    const int idx_f = p * lat.Vh + tile.y * lat.V3h + h3;
    const float4* g = reinterpret_cast<const float4*>(a.links + lat.off_bytes);
    const int B = blockDim.x;
    float4* slot = sm + (buf * 6 * ND) * B + threadIdx.x;
#pragma unroll
    for (int mu = 0; mu < ND; ++mu) {
      const int idx_b = (1 - p) * lat.Vh + (int)(back_lexi(lat, s, mu) >> 1);
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        cp_async16(slot + (3 * mu + w) * B, g + (long long)(w * 4 + mu) * lat.V + idx_f);
        cp_async16(slot + (3 * ND + 3 * mu + w) * B, g + (long long)(w * 4 + mu) * lat.V + idx_b);
      }
    }
  }
  return ms;
}

template <int ND>
__global__ void __launch_bounds__(256) k_measure_pipe(MeasureArgs a) {
  extern __shared__ float4 sm[];
  __shared__ double red[2][64];  // alternate per tile sum, as in k_or_sweep_pipe
  grid_dep_wait();
  grid_dep_launch();
  int rb = 0;
  if (a.st && !state_even_pass(a.st)) return;
  int k = blockIdx.x;
  if (k >= a.n_tiles) return;
  const int B = blockDim.x;
  int buf = 0;
  MeasSite cur = meas_issue<ND>(a, k, 0, sm);
  cp_async_commit();
  for (;;) {
    const int kn = k + (int)gridDim.x;
    MeasSite nxt;
    if (kn < a.n_tiles) nxt = meas_issue<ND>(a, kn, buf ^ 1, sm);
    cp_async_commit();
    cp_async_wait_all_but_newest();  // this thread's copies of tile k have landed
    if (cur.active) {                // uniform over the block
      float fsum = 0.f, q = 0.f;
      if (cur.valid) {
        const float4* slot = sm + (buf * 6 * ND) * B + threadIdx.x;
        cx<float> f[ND][6], b[ND][6];
#pragma unroll
        for (int nu = 0; nu < ND; ++nu) {
          pipe_read(slot, B, 3 * nu, f[nu]);
          pipe_read(slot, B, 3 * ND + 3 * nu, b[nu]);
        }
        cx<float> A[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) A[e] = {0.f, 0.f};
        float fs = 0.f;
#pragma unroll
        for (int nu = 0; nu < ND; ++nu) {
          add_to_A_F(A, fs, f[nu], b[nu]);
        }
        fsum = fs;
        q = theta_site(A);
      }
      const float v[2] = {fsum, q};
      float2 o[2];
      block_sum_f32<2>(v, o, reinterpret_cast<float*>(red[rb]));
      if (threadIdx.x == 0) {
        if (a.part_F) a.part_F[cur.ti] = o[0];
        a.part_theta[cur.ti] = o[1];
      }
      rb ^= 1;
    }
    if (kn >= a.n_tiles) break;
    k = kn;
    buf ^= 1;
    cur = nxt;
  }
}

}  // namespace gf
