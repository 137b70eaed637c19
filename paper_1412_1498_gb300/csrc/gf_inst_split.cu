// gf_inst_split.cu -- the double-float polish kernels and their conversions.
#include "gf_split.cuh"

namespace gf {

void launch_sweep_split(int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s) {
  if (nd == 4) k_or_sweep_split<4><<<n_tiles, threads, 0, s>>>(a);
  else k_or_sweep_split<3><<<n_tiles, threads, 0, s>>>(a);
}

void launch_measure_split(int nd, const MeasureArgs& a, int n_tiles, int threads, cudaStream_t s) {
  if (nd == 4) k_measure_split<4><<<n_tiles, threads, 0, s>>>(a);
  else k_measure_split<3><<<n_tiles, threads, 0, s>>>(a);
}

void launch_to_split(int storage, const char* src, char* dst, const LatDev& ls, const LatDev& ld,
                     cudaStream_t s) {
  const unsigned int nb = (unsigned int)((4 * ls.V + 255) / 256);
  if (storage == GF_FP32_12) k_to_split<GF_FP32_12><<<nb, 256, 0, s>>>(src, dst, ls, ld);
  else if (storage == GF_FP32_8) k_to_split<GF_FP32_8><<<nb, 256, 0, s>>>(src, dst, ls, ld);
  else k_to_split<GF_FP32_18><<<nb, 256, 0, s>>>(src, dst, ls, ld);
}

void launch_split_to_fp64(char* links, const LatDev& lat, cudaStream_t s) {
  const unsigned int nb = (unsigned int)((4 * lat.V + 255) / 256);
  k_split_to_fp64<<<nb, 256, 0, s>>>(links, lat);
}

}  // namespace gf
