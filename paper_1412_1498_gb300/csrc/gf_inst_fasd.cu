// gf_inst_fasd.cu -- Fourier-accelerated steepest descent kernels (FP32-12 and FP64-18).
#include "gf_fasd.cuh"

namespace gf {

static size_t plane_smem(int storage, const LatDev& lat) {
  const size_t c = storage == GF_FP64_18 ? 16 : 8;
  return 4 * (size_t)(lat.L[0] + 1) * lat.L[1] * c;  // rows padded by one element
}
static size_t column_smem(int storage, int nd, const LatDev& lat) {
  const size_t c = storage == GF_FP64_18 ? 16 : 8;
  const int KX = fasd_kx(lat, nd, c);
  return (size_t)(nd == 4 ? lat.L[3] : 1) * (lat.L[2] * KX + KX) * c;
}

// Shared-memory opt-in for every FA-SD kernel (outside any stream capture).
cudaError_t prepare_fasd(int storage, int nd, const LatDev& lat) {
  const int sp = (int)plane_smem(storage, lat), sc = (int)column_smem(storage, nd, lat);
  cudaError_t e = cudaSuccess;
#define GF_ATTR(k, n) if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, n)
  if (storage == GF_FP64_18) {
    if (nd == 4) { GF_ATTR((k_fasd_delta_xy<GF_FP64_18, 4>), sp); GF_ATTR((k_fasd_xy_inv_g<GF_FP64_18, 4>), sp); GF_ATTR((k_fasd_zt<double, 4>), sc); }
    else { GF_ATTR((k_fasd_delta_xy<GF_FP64_18, 3>), sp); GF_ATTR((k_fasd_xy_inv_g<GF_FP64_18, 3>), sp); GF_ATTR((k_fasd_zt<double, 3>), sc); }
  } else {
    if (nd == 4) { GF_ATTR((k_fasd_delta_xy<GF_FP32_12, 4>), sp); GF_ATTR((k_fasd_xy_inv_g<GF_FP32_12, 4>), sp); GF_ATTR((k_fasd_zt<float, 4>), sc); }
    else { GF_ATTR((k_fasd_delta_xy<GF_FP32_12, 3>), sp); GF_ATTR((k_fasd_xy_inv_g<GF_FP32_12, 3>), sp); GF_ATTR((k_fasd_zt<float, 3>), sc); }
  }
#undef GF_ATTR
  return e;
}

#define GF_FASD_SWITCH(storage, nd, CALL)                        \
  if (storage == GF_FP64_18) {                                   \
    if (nd == 4) CALL(GF_FP64_18, double, 4); else CALL(GF_FP64_18, double, 3); \
  } else {                                                       \
    if (nd == 4) CALL(GF_FP32_12, float, 4); else CALL(GF_FP32_12, float, 3);   \
  }

void launch_fasd_delta_xy(int storage, int nd, const FasdArgs& a, cudaStream_t s) {
  const dim3 grid(a.lat.L[2], a.lat.L[3]);
  const size_t sm = plane_smem(storage, a.lat);
#define GF_CALL(S, T, ND) k_fasd_delta_xy<S, ND><<<grid, kFasdThreads, sm, s>>>(a)
  GF_FASD_SWITCH(storage, nd, GF_CALL)
#undef GF_CALL
}

void launch_fasd_finish(const FasdArgs& a, cudaStream_t s) { k_fasd_finish<<<a.n_units, 256, 0, s>>>(a); }

void launch_fasd_zt(int storage, int nd, const FasdArgs& a, cudaStream_t s) {
  const dim3 grid(a.lat.L[0] / a.kx, a.lat.L[1], nd == 4 ? 4 : 4 * a.lat.L[3]);
  const size_t sm = column_smem(storage, nd, a.lat);
#define GF_CALL(S, T, ND) k_fasd_zt<T, ND><<<grid, 256, sm, s>>>(a)
  GF_FASD_SWITCH(storage, nd, GF_CALL)
#undef GF_CALL
}

void launch_fasd_xy_inv_g(int storage, int nd, const FasdArgs& a, cudaStream_t s) {
  const dim3 grid(a.lat.L[2], a.lat.L[3]);
  const size_t sm = plane_smem(storage, a.lat);
#define GF_CALL(S, T, ND) k_fasd_xy_inv_g<S, ND><<<grid, kFasdThreads, sm, s>>>(a)
  GF_FASD_SWITCH(storage, nd, GF_CALL)
#undef GF_CALL
}

void launch_fasd_update(int storage, int nd, const FasdArgs& a, cudaStream_t s) {
  const unsigned int nb = (unsigned int)((a.lat.V + 127) / 128);  // one site per thread
#define GF_CALL(S, T, ND) k_fasd_update<S, ND><<<nb, 128, 0, s>>>(a)
  GF_FASD_SWITCH(storage, nd, GF_CALL)
#undef GF_CALL
}


size_t fasd_plane_smem(int storage, const LatDev& lat) { return plane_smem(storage, lat); }

}  // namespace gf
