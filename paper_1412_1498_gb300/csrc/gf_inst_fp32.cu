// gf_inst_fp32.cu -- FP32 sweeps (12- and 18-real storage) and FP32 measurement.
#include "gf_kernels.cuh"
#include "gf_sweep_pipe.cuh"

namespace gf {

namespace {
constexpr int kMaxDev = 64;
int g_pipe_grid[kMaxDev][2][3];  // [device][nd == 4][threads 64/128/256] persistent grid size
int g_meas_grid[kMaxDev][2][3];  // the same for the pipelined F / theta pass
}  // namespace

static int threads_slot(int threads) { return threads == 64 ? 0 : threads == 128 ? 1 : 2; }

// Shared-memory opt-in and persistent grid size for the pipelined sweep (call outside
// any stream capture, before the first launch on a device).
cudaError_t prepare_sweep_pipe() {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= kMaxDev) return cudaErrorInvalidDevice;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  for (int n = 0; n < 2; ++n) {
    // the grid is sized for the first-order kernel; the exact-power one takes the same
    auto kern = n ? k_or_sweep_pipe<4, GF_OR_FIRST_ORDER> : k_or_sweep_pipe<3, GF_OR_FIRST_ORDER>;
    auto kern_exact = n ? k_or_sweep_pipe<4, GF_OR_EXACT> : k_or_sweep_pipe<3, GF_OR_EXACT>;
    e = cudaFuncSetAttribute(kern_exact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * kPipeWords * 256 * sizeof(float4)));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * kPipeWords * 256 * sizeof(float4)));
    if (e != cudaSuccess) return e;
    for (int t : {64, 128, 256}) {
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, t, 2 * kPipeWords * t * sizeof(float4));
      if (e != cudaSuccess) return e;
      g_pipe_grid[dev][n][threads_slot(t)] = per_sm * sms;
    }
    auto mk = n ? k_measure_pipe<4> : k_measure_pipe<3>;
    const int words = 6 * (n ? 4 : 3);
    e = cudaFuncSetAttribute(mk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * words * 256 * sizeof(float4)));
    if (e != cudaSuccess) return e;
    for (int t : {64, 128, 256}) {
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mk, t, 2 * words * t * sizeof(float4));
      if (e != cudaSuccess) return e;
      g_meas_grid[dev][n][threads_slot(t)] = per_sm * sms;
    }
  }
  return cudaSuccess;
}

void launch_measure_fp32_pipe(int nd, const MeasureArgs& a, int n_tiles, int threads, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  int grid = g_meas_grid[dev < kMaxDev ? dev : 0][nd == 4][threads_slot(threads)];
  if (grid <= 0) grid = 1;
  if (grid > n_tiles) grid = n_tiles;
  const size_t smem = 2 * 6 * nd * threads * sizeof(float4);
  launch_dep(a.dep != 0, nd == 4 ? k_measure_pipe<4> : k_measure_pipe<3>, dim3(grid), dim3(threads), smem, s, a);
}

// CTAs of the persistent pipelined sweep over n_tiles tiles (also the number of per-CTA
// partials it writes with cta_sums)
int sweep_pipe_grid(int nd, int threads, int n_tiles) {
  int dev = 0;
  cudaGetDevice(&dev);
  int grid = g_pipe_grid[dev < kMaxDev ? dev : 0][nd == 4][threads_slot(threads)];
  if (grid <= 0) grid = 1;
  if (grid > n_tiles) grid = n_tiles;
  return grid;
}

void launch_sweep_fp32_pipe(int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s) {
  const int grid = sweep_pipe_grid(nd, threads, n_tiles);
  const size_t smem = 2 * kPipeWords * threads * sizeof(float4);
  auto kern = a.form == GF_OR_FIRST_ORDER
                  ? (nd == 4 ? k_or_sweep_pipe<4, GF_OR_FIRST_ORDER> : k_or_sweep_pipe<3, GF_OR_FIRST_ORDER>)
                  : (nd == 4 ? k_or_sweep_pipe<4, GF_OR_EXACT> : k_or_sweep_pipe<3, GF_OR_EXACT>);
  launch_dep(a.dep != 0, kern, dim3(grid), dim3(threads), smem, s, a);
}

void launch_sweep_fp32(int storage, int nd, const SweepArgs& a, int n_tiles, int threads,
                       cudaStream_t s) {
#define GF_CALL(S, F)                                                          \
  if (nd == 4) k_or_sweep<S, 4, false, F><<<n_tiles, threads, 0, s>>>(a);      \
  else k_or_sweep<S, 3, false, F><<<n_tiles, threads, 0, s>>>(a);
  if (a.form == GF_OR_FIRST_ORDER) {
    if (storage == GF_FP32_12) { GF_CALL(GF_FP32_12, GF_OR_FIRST_ORDER) }
    else { GF_CALL(GF_FP32_18, GF_OR_FIRST_ORDER) }
  } else {
    if (storage == GF_FP32_12) { GF_CALL(GF_FP32_12, GF_OR_EXACT) }
    else { GF_CALL(GF_FP32_18, GF_OR_EXACT) }
  }
#undef GF_CALL
}

void launch_measure_fp32(int storage, int nd, const MeasureArgs& a, int n_tiles, int threads,
                         cudaStream_t s) {
  if (storage == GF_FP32_12) {
    if (nd == 4) k_measure<GF_FP32_12, 4><<<n_tiles, threads, 0, s>>>(a);
    else k_measure<GF_FP32_12, 3><<<n_tiles, threads, 0, s>>>(a);
  } else {
    if (nd == 4) k_measure<GF_FP32_18, 4><<<n_tiles, threads, 0, s>>>(a);
    else k_measure<GF_FP32_18, 3><<<n_tiles, threads, 0, s>>>(a);
  }
}

}  // namespace gf
