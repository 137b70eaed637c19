// gf_inst_fp64.cu -- FP64-18 sweep (fused multiply-add allowed) and FP64 measurement.
#include "gf_kernels.cuh"

namespace gf {

void launch_sweep_fp64(int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s) {
  if (a.form == GF_OR_FIRST_ORDER) {
    if (nd == 4) k_or_sweep<GF_FP64_18, 4, false, GF_OR_FIRST_ORDER><<<n_tiles, threads, 0, s>>>(a);
    else k_or_sweep<GF_FP64_18, 3, false, GF_OR_FIRST_ORDER><<<n_tiles, threads, 0, s>>>(a);
  } else {
    if (nd == 4) k_or_sweep<GF_FP64_18, 4, false, GF_OR_EXACT><<<n_tiles, threads, 0, s>>>(a);
    else k_or_sweep<GF_FP64_18, 3, false, GF_OR_EXACT><<<n_tiles, threads, 0, s>>>(a);
  }
}

void launch_measure_fp64(int nd, const MeasureArgs& a, int n_tiles, int threads, cudaStream_t s) {
  if (nd == 4) k_measure<GF_FP64_18, 4><<<n_tiles, threads, 0, s>>>(a);
  else k_measure<GF_FP64_18, 3><<<n_tiles, threads, 0, s>>>(a);
}

}  // namespace gf
