// gf_inst_fp32.cu -- FP32 sweeps (12- and 18-real storage) and FP32 measurement.
#include "gf_kernels.cuh"

namespace gf {

void launch_sweep_fp32(int storage, int nd, const SweepArgs& a, int n_tiles, int threads,
                       cudaStream_t s) {
  if (storage == GF_FP32_12) {
    if (nd == 4) k_or_sweep<GF_FP32_12, 4, false><<<n_tiles, threads, 0, s>>>(a);
    else k_or_sweep<GF_FP32_12, 3, false><<<n_tiles, threads, 0, s>>>(a);
  } else {
    if (nd == 4) k_or_sweep<GF_FP32_18, 4, false><<<n_tiles, threads, 0, s>>>(a);
    else k_or_sweep<GF_FP32_18, 3, false><<<n_tiles, threads, 0, s>>>(a);
  }
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
