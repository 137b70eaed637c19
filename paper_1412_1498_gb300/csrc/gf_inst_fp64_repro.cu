// gf_inst_fp64_repro.cu -- FP64-18 sweep in the reproducible arithmetic: this unit is
// compiled with -fmad=false, so every multiply and add of the sweep is a separate IEEE
// operation in the order written, and divisions / square roots are IEEE-rounded.
#include "gf_kernels.cuh"

namespace gf {

void launch_sweep_fp64_repro(int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s) {
  if (a.form == GF_OR_FIRST_ORDER) {
    if (nd == 4) k_or_sweep<GF_FP64_18, 4, true, GF_OR_FIRST_ORDER><<<n_tiles, threads, 0, s>>>(a);
    else k_or_sweep<GF_FP64_18, 3, true, GF_OR_FIRST_ORDER><<<n_tiles, threads, 0, s>>>(a);
  } else {
    if (nd == 4) k_or_sweep<GF_FP64_18, 4, true, GF_OR_EXACT><<<n_tiles, threads, 0, s>>>(a);
    else k_or_sweep<GF_FP64_18, 3, true, GF_OR_EXACT><<<n_tiles, threads, 0, s>>>(a);
  }
}

}  // namespace gf
