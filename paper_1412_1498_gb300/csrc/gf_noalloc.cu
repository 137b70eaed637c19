// gf_noalloc.cu -- F and theta of a device field without any allocation.
//
// Some callers cannot allocate device memory at all: code running under an allocator
// that forbids new device allocations (a framework's pre-reserved memory pool, a
// real-time loop that must not call cudaMalloc because it can synchronise the device,
// or a library embedded in a host process that owns every device allocation).  For
// them gf_functional_theta_noalloc measures F and theta of a field they already hold on
// the device, in the canonical layout, and needs no handle and no workspace: the block
// partial sums live in the file-scope static device array below.
//
// That array exists once per GPU that loads this library and stays allocated until the
// process exits.  Every call shares it, so two calls that overlap on the GPU (on
// different streams, or from different host threads) race on it and give wrong sums;
// calls on one stream run one after the other and are safe.  The array keeps the last
// call's contents; each call clears the part that must start at zero (the
// last-block ticket) before its kernel runs.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/gf.h"
#include "gf_device.cuh"

namespace gf {
void set_thread_error(const std::string& msg);  // defined with gf_last_error
}

namespace {

constexpr int kThreads = 256;
// control words (ticket) in the first 256 bytes, then one (F, theta) pair per block
constexpr int kControlDoubles = 32;
constexpr long long kScratchDoubles = kControlDoubles + 2LL * GF_NOALLOC_MAX_BLOCKS;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// messages go to the per-thread error text that gf_last_error(NULL) returns
struct ErrorText {
  void clear() { gf::set_thread_error(""); }
  ErrorText& operator=(const std::string& m) {
    gf::set_thread_error(m);
    return *this;
  }
} g_error;

// Device address of g_scratch on the current device (host code cannot use the symbol
// itself: in host code it names a host-side stand-in, not device memory).
int scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return GF_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    g_error = "device index out of range";
    return GF_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) {
      g_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return GF_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return GF_OK;
}

// One thread per site of the canonical (site-major complex128) field: Re Tr of the nd
// forward links (every link counted once over the lattice) and Tr[Delta Delta^+] of
// Delta(x) of Eq. (3).  Block sums go to the scratch; the last block to finish adds
// them in block order and writes out[0] = F, out[1] = theta.
template <int ND>
__global__ void __launch_bounds__(kThreads) k_measure_canonical(const double2* __restrict__ U, int Lx,
                                                                int Ly, int Lz, int Lt, double* scratch,
                                                                double* out) {
  using gf::cx;
  __shared__ double red[64];
  __shared__ int s_last;
  const long long V = (long long)Lx * Ly * Lz * Lt;
  const long long s = blockIdx.x * (long long)kThreads + threadIdx.x;
  double fsum = 0.0, q = 0.0;
  if (s < V) {
    long long r = s;
    const int x = (int)(r % Lx); r /= Lx;
    const int y = (int)(r % Ly); r /= Ly;
    const int z = (int)(r % Lz);
    const int t = (int)(r / Lz);
    const long long stride[4] = {1, Lx, (long long)Lx * Ly, (long long)Lx * Ly * Lz};
    const int c[4] = {x, y, z, t};
    const int L[4] = {Lx, Ly, Lz, Lt};
    cx<double> A[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) A[e] = {0.0, 0.0};
#pragma unroll
    for (int nu = 0; nu < ND; ++nu) {
      const long long sb = c[nu] == 0 ? s + stride[nu] * (L[nu] - 1) : s - stride[nu];
      const double2* f = U + (4 * s + nu) * 9;
      const double2* b = U + (4 * sb + nu) * 9;
      fsum += f[0].x + f[4].x + f[8].x;
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        const double2 fv = f[e], bv = b[e];
        A[e] = gf::cadd(A[e], gf::csub(cx<double>{bv.x, bv.y}, cx<double>{fv.x, fv.y}));
      }
    }
    cx<double> D[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) D[3 * i + j] = gf::csub(A[3 * i + j], gf::cconj(A[3 * j + i]));
    const cx<double> sum = gf::cadd(gf::cadd(D[0], D[4]), D[8]);
    const cx<double> tr = {sum.re / 3.0, sum.im / 3.0};
    D[0] = gf::csub(D[0], tr);
    D[4] = gf::csub(D[4], tr);
    D[8] = gf::csub(D[8], tr);
#pragma unroll
    for (int e = 0; e < 9; ++e) q = q + (D[e].re * D[e].re + D[e].im * D[e].im);
  }
  double v[2] = {fsum, q};
  gf::block_sum<2>(v, red);
  double* partial = scratch + kControlDoubles;
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = v[0];
    partial[2 * blockIdx.x + 1] = v[1];
    __threadfence();
    s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double w[2] = {0.0, 0.0};
  for (unsigned int k = threadIdx.x; k < gridDim.x; k += kThreads) {
    w[0] += __ldcg(partial + 2 * k);
    w[1] += __ldcg(partial + 2 * k + 1);
  }
  gf::block_sum<2>(w, red);
  if (threadIdx.x == 0) {
    out[0] = w[0] / ((double)ND * 3.0 * (double)V);
    out[1] = w[1] / (3.0 * (double)V);
    *ticket = 0u;
  }
}

}  // namespace

extern "C" GF_API int gf_functional_theta_noalloc(const int dims[4], int gauge, const double* links,
                                                   double* out, void* stream) {
  g_error.clear();
  if (!dims || !links || !out) {
    g_error = "null argument";
    return GF_EINVAL;
  }
  if (gauge != GF_LANDAU && gauge != GF_COULOMB) {
    g_error = "gauge must be GF_LANDAU or GF_COULOMB";
    return GF_EINVAL;
  }
  for (int k = 0; k < 4; ++k) {
    if (dims[k] < 2 || dims[k] % 2 != 0) {
      g_error = "every extent must be even and >= 2";
      return GF_EINVAL;
    }
  }
  if (((uintptr_t)links % 16) != 0) {
    g_error = "links must be 16-byte aligned device memory";
    return GF_EINVAL;
  }
  // the volume is formed with an overflow check against the scratch's site limit, so
  // no extents (each below 2^31, any product) can reach the launch below
  const long long max_sites = (long long)GF_NOALLOC_MAX_BLOCKS * kThreads;
  const long long V = gf::lattice_sites_checked(dims, max_sites);
  if (V < 0) {
    g_error = "lattice too large for the static scratch: at most " + std::to_string(max_sites) +
              " sites (got " + std::to_string(dims[0]) + " x " + std::to_string(dims[1]) + " x " +
              std::to_string(dims[2]) + " x " + std::to_string(dims[3]) + ")";
    return GF_EINVAL;
  }
  const long long blocks = (V + kThreads - 1) / kThreads;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != GF_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(scratch, 0, kControlDoubles * sizeof(double), s);
  if (e == cudaSuccess) {
    const double2* U = reinterpret_cast<const double2*>(links);
    if (gauge == GF_LANDAU)
      k_measure_canonical<4><<<(unsigned int)blocks, kThreads, 0, s>>>(U, dims[0], dims[1], dims[2], dims[3], scratch, out);
    else
      k_measure_canonical<3><<<(unsigned int)blocks, kThreads, 0, s>>>(U, dims[0], dims[1], dims[2], dims[3], scratch, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    g_error = std::string("launch: ") + cudaGetErrorString(e);
    return GF_ECUDA;
  }
  return GF_OK;
}
