// gf_inst_compact.cu -- sweep and measurement kernels for the compact storages:
// FP64-12 (rows 0, 1 in FP64) and the 8-real parametrisation in FP32 and FP64.
// The arithmetic is the register kernel's; only the load / store of a link differ.
#include "gf_kernels.cuh"

namespace gf {

#define GF_COMPACT_SWITCH(storage, nd, CALL)                         \
  switch (storage) {                                                 \
    case GF_FP64_12: if (nd == 4) CALL(GF_FP64_12, 4); else CALL(GF_FP64_12, 3); break; \
    case GF_FP64_8: if (nd == 4) CALL(GF_FP64_8, 4); else CALL(GF_FP64_8, 3); break;    \
    default: if (nd == 4) CALL(GF_FP32_8, 4); else CALL(GF_FP32_8, 3); break;           \
  }

void launch_sweep_compact(int storage, int nd, const SweepArgs& a, int n_tiles, int threads,
                          cudaStream_t s) {
  if (a.form == GF_OR_FIRST_ORDER) {
#define GF_CALL(S, ND) k_or_sweep<S, ND, false, GF_OR_FIRST_ORDER><<<n_tiles, threads, 0, s>>>(a)
    GF_COMPACT_SWITCH(storage, nd, GF_CALL)
#undef GF_CALL
  } else {
#define GF_CALL(S, ND) k_or_sweep<S, ND, false, GF_OR_EXACT><<<n_tiles, threads, 0, s>>>(a)
    GF_COMPACT_SWITCH(storage, nd, GF_CALL)
#undef GF_CALL
  }
}

void launch_measure_compact(int storage, int nd, const MeasureArgs& a, int n_tiles, int threads,
                            cudaStream_t s) {
#define GF_CALL(S, ND) k_measure<S, ND><<<n_tiles, threads, 0, s>>>(a)
  GF_COMPACT_SWITCH(storage, nd, GF_CALL)
#undef GF_CALL
}

}  // namespace gf
