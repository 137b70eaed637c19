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

// Persistent blocks of the inverse x/y transform: per device, storage and gauge (set by
// prepare_fasd), with whether its plane buffer is doubled (when two fit in a block).
namespace {
constexpr int kMaxDev = 64;
int g_xy_grid[kMaxDev][2][2];
int g_xy_prefetch[kMaxDev][2][2];
int g_zt_grid[kMaxDev][2][2];
int g_zt_prefetch[kMaxDev][2][2];
constexpr int kMaxBlockSmem = 227 * 1024;
}  // namespace

static size_t xy_inv_smem(int storage, const LatDev& lat, bool prefetch) {
  return (prefetch ? 2 : 1) * plane_smem(storage, lat);
}

// Shared-memory opt-in for every FA-SD kernel and the persistent grid of the inverse
// transform (outside any stream capture).
cudaError_t prepare_fasd(int storage, int nd, const LatDev& lat) {
  const int sp = (int)plane_smem(storage, lat), sc = (int)column_smem(storage, nd, lat);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= kMaxDev) return cudaErrorInvalidDevice;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const bool pf = 2 * (size_t)sp <= (size_t)kMaxBlockSmem;
  const int si = (int)xy_inv_smem(storage, lat, pf);
  const bool pz = 2 * (size_t)sc <= (size_t)kMaxBlockSmem;
  const int sz = (pz ? 2 : 1) * sc;
  const int is64 = storage == GF_FP64_18, is4 = nd == 4;
  g_xy_prefetch[dev][is64][is4] = pf;
  g_zt_prefetch[dev][is64][is4] = pz;
#define GF_ATTR(k, n) if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, n)
  if (storage == GF_FP64_18) {
    if (nd == 4) { GF_ATTR((k_fasd_delta_xy<GF_FP64_18, 4>), sp); GF_ATTR((k_fasd_xy_inv_g<GF_FP64_18, 4>), si); GF_ATTR((k_fasd_zt<double, 4>), sz); }
    else { GF_ATTR((k_fasd_delta_xy<GF_FP64_18, 3>), sp); GF_ATTR((k_fasd_xy_inv_g<GF_FP64_18, 3>), si); GF_ATTR((k_fasd_zt<double, 3>), sz); }
  } else {
    if (nd == 4) { GF_ATTR((k_fasd_delta_xy<GF_FP32_12, 4>), sp); GF_ATTR((k_fasd_xy_inv_g<GF_FP32_12, 4>), si); GF_ATTR((k_fasd_zt<float, 4>), sz); }
    else { GF_ATTR((k_fasd_delta_xy<GF_FP32_12, 3>), sp); GF_ATTR((k_fasd_xy_inv_g<GF_FP32_12, 3>), si); GF_ATTR((k_fasd_zt<float, 3>), sz); }
  }
#undef GF_ATTR
  if (e != cudaSuccess) return e;
  int per_sm = 0;
#define GF_OCC(k) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFasdThreads, si)
  if (storage == GF_FP64_18) { if (nd == 4) GF_OCC((k_fasd_xy_inv_g<GF_FP64_18, 4>)); else GF_OCC((k_fasd_xy_inv_g<GF_FP64_18, 3>)); }
  else { if (nd == 4) GF_OCC((k_fasd_xy_inv_g<GF_FP32_12, 4>)); else GF_OCC((k_fasd_xy_inv_g<GF_FP32_12, 3>)); }
#undef GF_OCC
  if (e != cudaSuccess) return e;
  g_xy_grid[dev][is64][is4] = (per_sm > 0 ? per_sm : 1) * sms;
#define GF_OCC(k) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFasdThreads, sz)
  if (storage == GF_FP64_18) { if (nd == 4) GF_OCC((k_fasd_zt<double, 4>)); else GF_OCC((k_fasd_zt<double, 3>)); }
  else { if (nd == 4) GF_OCC((k_fasd_zt<float, 4>)); else GF_OCC((k_fasd_zt<float, 3>)); }
#undef GF_OCC
  if (e != cudaSuccess) return e;
  g_zt_grid[dev][is64][is4] = (per_sm > 0 ? per_sm : 1) * sms;
  return cudaSuccess;
}

int fasd_zt_prefetch(int storage, int nd) {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_zt_prefetch[dev < kMaxDev ? dev : 0][storage == GF_FP64_18][nd == 4];
}

// whether the inverse x/y transform of this device, storage and gauge double-buffers
int fasd_xy_prefetch(int storage, int nd) {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_xy_prefetch[dev < kMaxDev ? dev : 0][storage == GF_FP64_18][nd == 4];
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
  int dev = 0;
  cudaGetDevice(&dev);
  const int n_items = a.lat.L[0] / a.kx * a.lat.L[1] * (nd == 4 ? 4 : 4 * a.lat.L[3]);
  int g = g_zt_grid[dev < kMaxDev ? dev : 0][storage == GF_FP64_18][nd == 4];
  if (g <= 0) g = 1;
  const unsigned int grid = (unsigned int)(g < n_items ? g : n_items);
  const size_t sm = (a.zt_prefetch ? 2 : 1) * column_smem(storage, nd, a.lat);
#define GF_CALL(S, T, ND) k_fasd_zt<T, ND><<<grid, kFasdThreads, sm, s>>>(a)
  GF_FASD_SWITCH(storage, nd, GF_CALL)
#undef GF_CALL
}

void launch_fasd_xy_inv_g(int storage, int nd, const FasdArgs& a, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  const int n_planes = a.lat.L[2] * a.lat.L[3];
  int g = g_xy_grid[dev < kMaxDev ? dev : 0][storage == GF_FP64_18][nd == 4];
  if (g <= 0) g = 1;
  const unsigned int grid = (unsigned int)(g < n_planes ? g : n_planes);
  const size_t sm = xy_inv_smem(storage, a.lat, a.xy_prefetch != 0);
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
