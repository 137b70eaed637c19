// gf_api.cu -- host implementation of the C ABI declared in include/gf.h.
//
// Algorithm 1 of the paper as a device-driven loop: each sweep is five launches (even
// half-sweep; odd half-sweep with fused reunitarisation, F and odd-site theta; the
// odd-part finish, which decides every unit whose odd-site theta alone reaches eps;
// the even-site theta pass for the undecided units; the loop finish) that read and
// update a small DevState in device memory, so that a captured CUDA graph of many
// sweeps needs no host decision between them.  The host synchronises once per graph
// replay to read the number of still-active convergence units.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/gf.h"
#include "gf_kernels.cuh"

namespace gf {
void launch_sweep_fp64(int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s);
void launch_sweep_fp64_repro(int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s);
void launch_sweep_fp32(int storage, int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s);
void launch_sweep_fp32_pipe(int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s);
void launch_measure_fp32_pipe(int nd, const MeasureArgs& a, int n_tiles, int threads, cudaStream_t s);
cudaError_t prepare_sweep_pipe();
int sweep_pipe_grid(int nd, int threads, int n_tiles);
void launch_sweep_split(int nd, const SweepArgs& a, int n_tiles, int threads, cudaStream_t s);
void launch_measure_split(int nd, const MeasureArgs& a, int n_tiles, int threads, cudaStream_t s);
void launch_to_split(int storage, const char* src, char* dst, const LatDev& ls, const LatDev& ld,
                     cudaStream_t s);
void launch_split_to_fp64(char* links, const LatDev& lat, cudaStream_t s);

// internal storage code of the double-float polish copy (never visible in the C ABI)
constexpr int kSplit18 = 100;

cudaError_t prepare_fasd(int storage, int nd, const LatDev& lat);
int fasd_xy_prefetch(int storage, int nd);
int fasd_zt_prefetch(int storage, int nd);
void launch_fasd_delta_xy(int storage, int nd, const FasdArgs& a, cudaStream_t s);
void launch_fasd_finish(const FasdArgs& a, cudaStream_t s);
void launch_fasd_zt(int storage, int nd, const FasdArgs& a, cudaStream_t s);
void launch_fasd_xy_inv_g(int storage, int nd, const FasdArgs& a, cudaStream_t s);
void launch_fasd_update(int storage, int nd, const FasdArgs& a, cudaStream_t s);
size_t ad_partial_doubles(long long V);
void launch_ad_forward(const AdArgs& a, cudaStream_t s);
void launch_ad_backward(const AdArgs& a, cudaStream_t s);
void launch_measure_fp64(int nd, const MeasureArgs& a, int n_tiles, int threads, cudaStream_t s);
void launch_measure_fp32(int storage, int nd, const MeasureArgs& a, int n_tiles, int threads,
                         cudaStream_t s);
void launch_fill_int(int* p, int value, int n, cudaStream_t s);

void launch_sweep_compact(int storage, int nd, const SweepArgs& a, int n_tiles, int threads,
                          cudaStream_t s);
void launch_measure_compact(int storage, int nd, const MeasureArgs& a, int n_tiles, int threads,
                            cudaStream_t s);

bool is_fp64_storage(int storage) {
  return storage == GF_FP64_18 || storage == GF_FP64_12 || storage == GF_FP64_8;
}
bool is_compact_storage(int storage) {
  return storage == GF_FP64_12 || storage == GF_FP64_8 || storage == GF_FP32_8;
}

void launch_sweep(int storage, int nd, bool repro, int variant, const SweepArgs& a, int n_tiles,
                  int threads, cudaStream_t s) {
  if (storage == kSplit18) {
    launch_sweep_split(nd, a, n_tiles, threads, s);
  } else if (is_compact_storage(storage)) {
    launch_sweep_compact(storage, nd, a, n_tiles, threads, s);
  } else if (storage == GF_FP64_18) {
    if (repro) launch_sweep_fp64_repro(nd, a, n_tiles, threads, s);
    else launch_sweep_fp64(nd, a, n_tiles, threads, s);
  } else if (storage == GF_FP32_12 && variant != GF_SWEEP_REGISTER) {
    launch_sweep_fp32_pipe(nd, a, n_tiles, threads, s);
  } else {
    launch_sweep_fp32(storage, nd, a, n_tiles, threads, s);
  }
}

void launch_measure(int storage, int nd, int variant, const MeasureArgs& a, int n_tiles,
                    int threads, cudaStream_t s) {
  if (storage == GF_FP32_12 && variant != GF_SWEEP_REGISTER) {
    launch_measure_fp32_pipe(nd, a, n_tiles, threads, s);
    return;
  }
  if (storage == kSplit18) launch_measure_split(nd, a, n_tiles, threads, s);
  else if (is_compact_storage(storage)) launch_measure_compact(storage, nd, a, n_tiles, threads, s);
  else if (storage == GF_FP64_18) launch_measure_fp64(nd, a, n_tiles, threads, s);
  else launch_measure_fp32(storage, nd, a, n_tiles, threads, s);
}
}  // namespace gf

using namespace gf;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace gf {
void set_thread_error(const std::string& msg) { g_create_error = msg; }
}  // namespace gf

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kStagingMax = 32u << 20;  // bytes of canonical links per host copy
constexpr int kMinThreads = 64;
constexpr int kGraphSweeps = 16;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int link_bytes(int storage) {
  switch (storage) {
    case GF_FP64_18: return 144;
    case GF_FP64_12: return 96;
    case GF_FP32_18: return 72;
    case GF_FP64_8: return 64;
    case GF_FP32_8: return 32;
    default: return 48;  // GF_FP32_12
  }
}

struct Layout {
  size_t links, links64, staging, lats, lats64, tiles, unit_tiles, unit_lat, active, iters, partF,
      pthe, ptho, pending, usTo, unit_norm, usF, usT, uF, uT, lF, lT, state, kbuf, gbuf, planeF, planeT,
      unit_planes, ad_g, ad_delta, ad_part, ad_ticket, total;
  size_t staging_bytes;
  int max_tiles, n_units;
};

bool valid_dims(const int* d) {
  for (int k = 0; k < 4; ++k)
    if (d[k] < 2 || (d[k] % 2) != 0) return false;
  // half-volumes and plane indices stay in 32 bits: V < 2^31
  return lattice_sites_checked(d, (1LL << 31) - 1) > 0;
}

int tiles_for(const int* d, int threads) {
  const long long V3h = (long long)d[0] * d[1] * d[2] / 2;
  return (int)(d[3] * ((V3h + threads - 1) / threads));
}

// Carve the workspace: every region 256-byte aligned.
bool plan(int n_lat, const int* dims, int gauge, int storage, int flags, Layout* L) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  long long sites = 0, vmax = 0;
  int max_tiles = 0, n_units = 0;
  for (int l = 0; l < n_lat; ++l) {
    const int* d = dims + 4 * l;
    long long V = (long long)d[0] * d[1] * d[2] * d[3];
    sites += V;
    vmax = std::max(vmax, V);
    max_tiles += tiles_for(d, kMinThreads);
    n_units += gauge == GF_LANDAU ? 1 : d[3];
  }
  L->links = take((size_t)sites * 4 * link_bytes(storage));
  const bool mixed = (flags & GF_FLAG_MIXED) && !is_fp64_storage(storage);
  L->links64 = mixed ? take((size_t)sites * 4 * 144) : (size_t)-1;
  size_t canon = (size_t)vmax * 4 * 144;
  size_t site_bytes = 4 * 144;
  L->staging_bytes = std::max(site_bytes, std::min(canon, kStagingMax) / site_bytes * site_bytes);
  L->staging = take(L->staging_bytes);
  L->lats = take(sizeof(LatDev) * n_lat);
  L->lats64 = take(sizeof(LatDev) * n_lat);
  L->tiles = take(sizeof(int4) * max_tiles);
  L->unit_tiles = take(sizeof(int) * (n_units + 1));
  L->unit_lat = take(sizeof(int) * n_units);
  L->active = take(sizeof(int) * n_units);
  L->partF = take(sizeof(float2) * max_tiles);
  L->pthe = take(sizeof(float2) * max_tiles);
  L->ptho = take(sizeof(float2) * max_tiles);
  L->pending = take(sizeof(int) * n_units);
  L->usTo = take(sizeof(double) * n_units);
  L->unit_norm = take(sizeof(double) * 2 * n_units);
  L->usF = take(sizeof(double) * n_units);
  L->usT = take(sizeof(double) * n_units);
  L->uF = take(sizeof(double) * n_units);
  L->uT = take(sizeof(double) * n_units);
  // the result block, contiguous: iteration counts, lattice F and theta, loop state
  L->iters = take(sizeof(int) * n_units);
  L->lF = take(sizeof(double) * n_lat);
  L->lT = take(sizeof(double) * n_lat);
  L->state = take(sizeof(DevState));
  if (flags & GF_FLAG_FASD) {
    const int* d = dims;  // one lattice
    const size_t c = storage == GF_FP64_18 ? 16 : 8;
    const long long V = (long long)d[0] * d[1] * d[2] * d[3];
    L->kbuf = take(4 * (size_t)V * c);
    L->gbuf = take(6 * (size_t)V * c);
    L->planeF = take(sizeof(float2) * d[2] * d[3]);
    L->planeT = take(sizeof(float2) * d[2] * d[3]);
    L->unit_planes = take(sizeof(int) * (n_units + 1));
  } else {
    L->kbuf = L->gbuf = L->planeF = L->planeT = L->unit_planes = (size_t)-1;
  }
  if (flags & GF_FLAG_AUTOGRAD) {
    const long long V = (long long)dims[0] * dims[1] * dims[2] * dims[3];
    L->ad_g = take(9 * 16 * (size_t)V);
    L->ad_delta = take(9 * 16 * (size_t)V);
    L->ad_part = take(sizeof(double) * ad_partial_doubles(V));
    L->ad_ticket = take(sizeof(unsigned int));
  } else {
    L->ad_g = L->ad_delta = L->ad_part = L->ad_ticket = (size_t)-1;
  }
  L->total = off;
  L->max_tiles = max_tiles;
  L->n_units = n_units;
  return true;
}

int check_common(int n_lat, const int* dims, int gauge, int storage, int flags, std::string* why) {
  if (n_lat < 1 || !dims) { *why = "need at least one lattice"; return GF_EINVAL; }
  if (gauge != GF_LANDAU && gauge != GF_COULOMB) { *why = "gauge must be GF_LANDAU or GF_COULOMB"; return GF_EINVAL; }
  if (storage < GF_FP64_18 || storage > GF_FP64_8) {
    *why = "storage must be one of GF_FP64_18, GF_FP32_18, GF_FP32_12, GF_FP64_12, GF_FP32_8, GF_FP64_8";
    return GF_EINVAL;
  }
  if (flags & ~(GF_FLAG_MIXED | GF_FLAG_FASD | GF_FLAG_AUTOGRAD)) { *why = "unknown flag"; return GF_EINVAL; }
  if ((flags & GF_FLAG_AUTOGRAD) && (n_lat != 1 || storage != GF_FP64_18)) {
    *why = "the differentiable functional takes one lattice in GF_FP64_18 storage";
    return GF_EINVAL;
  }
  if (flags & GF_FLAG_FASD) {
    if (n_lat != 1) { *why = "Fourier-accelerated steepest descent takes one lattice per handle"; return GF_EINVAL; }
    if (storage != GF_FP32_12 && storage != GF_FP64_18) { *why = "Fourier acceleration supports GF_FP32_12 and GF_FP64_18 storage"; return GF_EINVAL; }
    const int nfft = gauge == GF_LANDAU ? 4 : 3;
    for (int k = 0; k < nfft; ++k) {
      const int L = dims[k];
      if (L > 64 || (L & (L - 1)) != 0) {
        *why = "Fourier acceleration needs power-of-two extents <= 64 in the transformed directions";
        return GF_EINVAL;
      }
    }
    const size_t c = storage == GF_FP64_18 ? 16 : 8;
    if (4 * (size_t)(dims[0] + 1) * dims[1] * c > 200 * 1024) {
      *why = "Lx * Ly too large for the shared-memory plane FFT";
      return GF_EINVAL;
    }
  }
  for (int l = 0; l < n_lat; ++l) {
    const int* d = dims + 4 * l;
    if (!valid_dims(d)) {
      char buf[200];
      bool even = true;
      for (int k = 0; k < 4; ++k) even = even && d[k] >= 2 && d[k] % 2 == 0;
      if (even)
        snprintf(buf, sizeof buf, "lattice %d: %d x %d x %d x %d sites; fewer than 2^31 are supported", l,
                 d[0], d[1], d[2], d[3]);
      else
        snprintf(buf, sizeof buf, "lattice %d: every extent must be even and >= 2 (got %d %d %d %d)", l,
                 d[0], d[1], d[2], d[3]);
      *why = buf;
      return GF_EINVAL;
    }
    // the kernels divide slice indices by Lx and Ly with 32-bit reciprocal multiplies
    const unsigned long long v3 = (unsigned long long)d[0] * d[1] * d[2];
    if (v3 * (unsigned long long)(d[0] > d[1] ? d[0] : d[1]) >= (1ULL << 32)) {
      *why = "Lx * Ly * Lz * max(Lx, Ly) must be below 2^32";
      return GF_EINVAL;
    }
  }
  return GF_OK;
}

}  // namespace

struct gf_handle {
  int n_lat = 0, gauge = 0, nd = 4, storage = 0, flags = 0;
  std::vector<int> dims;
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  bool own_ws = false;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  Layout L{};
  // device regions
  char *links = nullptr, *links64 = nullptr, *staging = nullptr;
  LatDev *d_lats = nullptr, *d_lats64 = nullptr;
  int4* d_tiles = nullptr;
  int *d_unit_tiles = nullptr, *d_unit_lat = nullptr, *d_active = nullptr, *d_iters = nullptr;
  float2 *d_partF = nullptr, *d_pthe = nullptr, *d_ptho = nullptr;  // per-tile pairs (hi, lo)
  double* d_usTo = nullptr;
  int* d_pending = nullptr;
  double* hist = nullptr;  // caller's device buffer of check records (gf_set_history)
  int hist_cap = 0, hist_n = 0, hist_sweeps = 0;
  double* d_unit_norm = nullptr;
  double *d_usF = nullptr, *d_usT = nullptr, *d_uF = nullptr, *d_uT = nullptr, *d_lF = nullptr,
         *d_lT = nullptr;
  DevState* d_state = nullptr;
  // host copies
  std::vector<LatDev> lats, lats64;
  int n_tiles = 0, n_units = 0, threads = 128;
  // settings
  double omega = 1.7, eps_switch = 1e-8;
  int form = GF_OR_FIRST_ORDER, reunit_interval = 20, check_interval = 1;
  int variant = GF_SWEEP_AUTO;
  int polish = GF_POLISH_SPLIT;
  int method = GF_METHOD_OR;
  double alpha = 0.08;
  void* kbuf = nullptr;
  char* gbuf = nullptr;
  float2 *d_planeF = nullptr, *d_planeT = nullptr;
  int* d_unit_planes = nullptr;
  void *ad_g = nullptr, *ad_delta = nullptr;
  double* ad_part = nullptr;
  unsigned int* ad_ticket = nullptr;
  bool repro = false;
  // state
  int cur = 0;  // 0: primary buffer holds the field, 1: polish buffer in FP64-18,
                // 2: polish buffer in double-float (only inside gf_fix)
  int phase_sweeps[2] = {0, 0};
  int sweeps_done = 0;  // since the last upload: the reunitarisation / check schedule
  // graphs: per buffer state (OR) one of each length 16, 8, 4, 2, 1 sweeps, one per set
  // of precision levels of a mixed run, one for Fourier acceleration
  cudaGraphExec_t graph[3][5] = {};
  cudaGraphExec_t graph_mix[8] = {};
  cudaGraphExec_t graph_fasd = nullptr;
  // pinned host ring: slots 0 and 1 receive the result block (iteration counts, lattice
  // F and theta, loop state) behind each replay in flight, whose events follow the
  // copies; slot 2 holds the loop state uploaded at the start of a phase
  char* res_host = nullptr;
  size_t res_bytes = 0, res_stride = 0;
  int res_slot = -1;  // slot with the results of the loop that just ended, else -1
  cudaEvent_t st_ev[2] = {nullptr, nullptr};
  char* out_host = nullptr;  // pinned staging of the values gf_fix / gf_functional_theta return
  int last_active = 0;  // active units when the last OR loop (run_phase / run_mixed) ended
  std::string err;
};

namespace {

int fail(gf_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

#define GF_CK(h, call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(h, GF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

#define GF_CK_LAUNCH(h) GF_CK(h, cudaGetLastError())

void drop_graphs(gf_handle* h) {
  for (auto& gs : h->graph)
    for (auto& g : gs)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  for (auto& g : h->graph_mix)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  if (h->graph_fasd) {
    cudaGraphExecDestroy(h->graph_fasd);
    h->graph_fasd = nullptr;
  }
}

int cur_storage(const gf_handle* h) {
  return h->cur == 2 ? kSplit18 : h->cur == 1 ? GF_FP64_18 : h->storage;
}
char* cur_links(const gf_handle* h) { return h->cur >= 1 ? h->links64 : h->links; }
LatDev* cur_lats(const gf_handle* h) { return h->cur >= 1 ? h->d_lats64 : h->d_lats; }
const LatDev& cur_lat_host(const gf_handle* h, int l) { return h->cur >= 1 ? h->lats64[l] : h->lats[l]; }

// Build the tile table for the current block size and upload it.  `keep` (nullable)
// lists per unit whether its tiles go into the table: a mixed run drops the tiles of
// finished units (their range becomes empty) so that the launches of its last sweeps
// cover only the units still working.
int build_tiles(gf_handle* h, const std::vector<int>* keep = nullptr) {
  std::vector<int4> tiles;
  std::vector<int> unit_tiles, unit_lat;
  for (int l = 0; l < h->n_lat; ++l) {
    const LatDev& lat = h->lats[l];
    if (h->gauge == GF_LANDAU) {
      unit_tiles.push_back((int)tiles.size());
      unit_lat.push_back(l);
    }
    for (int t = 0; t < lat.L[3]; ++t) {
      if (h->gauge == GF_COULOMB) {
        unit_tiles.push_back((int)tiles.size());
        unit_lat.push_back(l);
      }
      const int unit = lat.unit0 + (h->gauge == GF_COULOMB ? t : 0);
      if (keep && !(*keep)[unit]) continue;
      for (int h3 = 0; h3 < lat.V3h; h3 += h->threads) tiles.push_back(make_int4(l, t, h3, unit));
    }
  }
  unit_tiles.push_back((int)tiles.size());
  if ((int)tiles.size() > h->L.max_tiles) return fail(h, GF_EINVAL, "tile table overflow");
  h->n_tiles = (int)tiles.size();
  GF_CK(h, cudaMemcpyAsync(h->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice, h->stream));
  GF_CK(h, cudaMemcpyAsync(h->d_unit_tiles, unit_tiles.data(), sizeof(int) * unit_tiles.size(),
                           cudaMemcpyHostToDevice, h->stream));
  GF_CK(h, cudaMemcpyAsync(h->d_unit_lat, unit_lat.data(), sizeof(int) * unit_lat.size(),
                           cudaMemcpyHostToDevice, h->stream));
  std::vector<double> unit_norm;
  for (int l : unit_lat) {
    const LatDev& lat = h->lats[l];
    const double vol = h->gauge == GF_LANDAU ? (double)lat.V : 2.0 * lat.V3h;
    unit_norm.push_back(1.0 / ((double)h->nd * 3.0 * vol));
    unit_norm.push_back(1.0 / (3.0 * vol));
  }
  GF_CK(h, cudaMemcpyAsync(h->d_unit_norm, unit_norm.data(), sizeof(double) * unit_norm.size(),
                           cudaMemcpyHostToDevice, h->stream));
  GF_CK(h, cudaStreamSynchronize(h->stream));  // host vectors die on return
  drop_graphs(h);
  return GF_OK;
}

SweepArgs sweep_args(gf_handle* h, int parity, bool loop, int reverse) {
  SweepArgs a{};
  a.n_tiles = h->n_tiles;
  a.reverse = reverse;
  a.links = cur_links(h);
  a.lats = cur_lats(h);
  a.tiles = h->d_tiles;
  a.active = loop ? h->d_active : nullptr;
  a.st = loop ? h->d_state : nullptr;
  a.part_theta = h->d_ptho;
  a.part_F = loop && parity == 1 ? h->d_partF : nullptr;
  a.parity = parity;
  a.form = h->form;
  a.reunit = 0;
  a.measure = 0;
  a.level = 1;
  a.dep = h->n_units == 1;
  a.omega = h->omega;
  return a;
}

MeasureArgs measure_args(gf_handle* h, int parity, bool loop, int reverse) {
  MeasureArgs a{};
  a.n_tiles = h->n_tiles;
  a.reverse = reverse;
  a.links = cur_links(h);
  a.lats = cur_lats(h);
  a.tiles = h->d_tiles;
  // in the loop the even-site pass serves the units pending after the odd half-sweep,
  // which already measured F
  a.active = loop ? h->d_pending : nullptr;
  a.st = loop ? h->d_state : nullptr;
  a.part_F = parity == 0 && !loop ? h->d_partF : nullptr;
  a.part_theta = parity == 0 ? h->d_pthe : h->d_ptho;
  a.parity = parity;
  a.level = 1;
  a.dep = h->n_units == 1;
  return a;
}

FinishArgs finish_args(gf_handle* h, int mode) {
  FinishArgs a{};
  a.lats = cur_lats(h);
  a.unit_tiles = h->d_unit_tiles;
  a.n_tiles = h->n_tiles;
  a.n_odd_parts = h->n_tiles;
  a.unit_lat = h->d_unit_lat;
  a.unit_norm = h->d_unit_norm;
  a.active = h->d_active;
  a.iters = h->d_iters;
  a.part_F = h->d_partF;
  a.part_th_even = h->d_pthe;
  a.part_th_odd = h->d_ptho;
  a.pending = h->d_pending;
  a.unit_sumTh_odd = h->d_usTo;
  a.hist = h->hist;
  a.hist_cap = h->hist_cap;
  a.unit_sumF = h->d_usF;
  a.unit_sumTh = h->d_usT;
  a.unit_F = h->d_uF;
  a.unit_theta = h->d_uT;
  a.lat_F = h->d_lF;
  a.lat_theta = h->d_lT;
  a.st = h->d_state;
  a.n_units = h->n_units;
  a.n_lat = h->n_lat;
  a.nd = h->nd;
  a.mode = mode;
  a.dep = h->n_units == 1;
  return a;
}

// F and theta of every unit and lattice, all units (mode MEASURE or RESET), async.
int enqueue_measure_all(gf_handle* h, int mode) {
  const int st = cur_storage(h);
  launch_measure(st, h->nd, h->variant, measure_args(h, 0, false, 0), h->n_tiles, h->threads, h->stream);
  GF_CK_LAUNCH(h);
  launch_measure(st, h->nd, h->variant, measure_args(h, 1, false, 1), h->n_tiles, h->threads, h->stream);
  GF_CK_LAUNCH(h);
  launch_finish(finish_args(h, mode), h->stream);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

// The opening check of a phase (Algorithm 1 stops before its first sweep when theta <
// eps): the odd-site pass (F and the odd-site part of theta), then FINISH_OPEN, which
// starts every unit whose odd part alone reaches its threshold (theta >= its odd part,
// so the full theta decides the same).  Only if some unit is undecided (or a history is
// kept) do the even-site pass and a reset run, gated on the loop state; they measure
// every unit with the same sums as enqueue_measure_all.  The odd pass walks the tiles
// backwards so that the first even half-sweep starts where it ended.
int enqueue_opening(gf_handle* h) {
  const int st = cur_storage(h);
  MeasureArgs mo = measure_args(h, 1, false, 1);
  mo.part_F = h->d_partF;
  launch_measure(st, h->nd, h->variant, mo, h->n_tiles, h->threads, h->stream);
  GF_CK_LAUNCH(h);
  launch_finish(finish_args(h, FINISH_OPEN), h->stream);
  GF_CK_LAUNCH(h);
  MeasureArgs me = measure_args(h, 0, false, 0);
  me.st = h->d_state;
  launch_measure(st, h->nd, h->variant, me, h->n_tiles, h->threads, h->stream);
  GF_CK_LAUNCH(h);
  FinishArgs fr = finish_args(h, FINISH_RESET);
  fr.gated = 1;
  launch_finish(fr, h->stream);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

// One sweep of the device-driven loop: even half-sweep, odd half-sweep (F and odd-site
// theta fused on check sweeps), FINISH_ODD, which decides every unit whose odd part alone
// settles the stop (theta >= its odd part) and closes the sweep.  When some unit is
// undecided it leaves the sweep open (DevState.hold) for the even-site theta pass and
// FINISH_LOOP.  With one unit that happens on the last sweeps of a run only, so those
// two are not captured: the rest of the replay does nothing and the host runs them
// (resolve_open_sweep) before the next replay, and a sweep is three launches.  With many
// units some unit is undecided on many sweeps (theta is not monotone and units hover
// about their thresholds), so they are captured after FINISH_ODD and run (as no-ops when
// nothing is pending) on every sweep.  Consecutive half-sweeps walk the tiles in
// opposite directions, so each starts on the lines the previous one left in L2.  A
// one-unit lattice swept by the persistent pipelined kernel takes F and the odd-site
// theta as one partial per CTA.  `pass` counts half-sweeps (2 per sweep).
int enqueue_loop_sweep(gf_handle* h, cudaStream_t s, int* pass) {
  const int st = cur_storage(h);
  launch_sweep(st, h->nd, h->repro, h->variant, sweep_args(h, 0, true, (*pass)++ & 1), h->n_tiles,
               h->threads, s);
  GF_CK_LAUNCH(h);
  SweepArgs ao = sweep_args(h, 1, true, (*pass)++ & 1);
  FinishArgs fo = finish_args(h, FINISH_ODD);
  if (h->n_units == 1 && st == GF_FP32_12 && h->variant != GF_SWEEP_REGISTER) {
    ao.cta_sums = 1;
    fo.n_odd_parts = sweep_pipe_grid(h->nd, h->threads, h->n_tiles);
  }
  launch_sweep(st, h->nd, h->repro, h->variant, ao, h->n_tiles, h->threads, s);
  GF_CK_LAUNCH(h);
  launch_finish(fo, s);
  GF_CK_LAUNCH(h);
  if (h->n_units > 1) {
    launch_measure(st, h->nd, h->variant, measure_args(h, 0, true, ao.reverse ^ 1), h->n_tiles, h->threads, s);
    GF_CK_LAUNCH(h);
    launch_finish(finish_args(h, FINISH_LOOP), s);
    GF_CK_LAUNCH(h);
  }
  return GF_OK;
}

// The even-site theta pass for the units an open sweep left undecided, then FINISH_LOOP
// (their theta, masks and iteration counts; the sweep is counted and the hold released).
int resolve_open_sweep(gf_handle* h) {
  launch_measure(cur_storage(h), h->nd, h->variant, measure_args(h, 0, true, 0), h->n_tiles, h->threads,
                 h->stream);
  GF_CK_LAUNCH(h);
  launch_finish(finish_args(h, FINISH_LOOP), h->stream);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

// Capture the loop graphs of the current buffer state, 16 >> k sweeps for k = 0..4 (each
// an even number of half-sweeps, so replays keep alternating the tile direction), all at
// once on first use so that no later gf_fix captures inside its run.  Each graph ends
// with the even-site pass and the loop finish, which act only on a sweep left open: a
// replay ends with every sweep resolved (the rest of a replay after an open sweep does
// nothing), so the host reads the state without resolving anything.
int ensure_graphs(gf_handle* h) {
  for (int k = 0; k < 5; ++k) {
    if (h->graph[h->cur][k]) continue;
    GF_CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = GF_OK, pass = 0;
    for (int j = 0; j < (kGraphSweeps >> k) && rc == GF_OK; ++j) rc = enqueue_loop_sweep(h, h->cap_stream, &pass);
    if (rc == GF_OK) {
      launch_measure(cur_storage(h), h->nd, h->variant, measure_args(h, 0, true, 0), h->n_tiles, h->threads,
                     h->cap_stream);
      launch_finish(finish_args(h, FINISH_LOOP), h->cap_stream);
      if (cudaGetLastError() != cudaSuccess) rc = fail(h, GF_ECUDA, "launch in the loop capture failed");
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc != GF_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(h, GF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph[h->cur][k], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, GF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  return GF_OK;
}

// The graph for the next replay when `left` sweeps of the budget remain: the shortest
// length >= left, halved when that would run more than two gated sweeps past the budget
// (a gated sweep costs about three idle launches, a further replay one host round trip).
int graph_index(int left) {
  int k = 0;  // 16 >> k sweeps
  while (k < 4 && (kGraphSweeps >> (k + 1)) >= left) ++k;
  if ((kGraphSweeps >> k) - left > 2 && k < 4) ++k;
  return k;
}

// The loop state, through the pinned upload slot of the result ring (stream-ordered after
// any upload from it).
int read_state(gf_handle* h, DevState* out) {
  char* slot = h->res_host + 2 * h->res_stride;
  GF_CK(h, cudaMemcpyAsync(slot, h->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  GF_CK(h, cudaStreamSynchronize(h->stream));
  std::memcpy(out, slot, sizeof(DevState));
  return GF_OK;
}

DevState* res_state(gf_handle* h, int slot) {
  return reinterpret_cast<DevState*>(h->res_host + slot * h->res_stride + (h->L.state - h->L.iters));
}

// One phase of Algorithm 1 on the current buffer: measure, then sweeps until every
// unit is below eps or `budget` sweeps were done.  *done receives the sweeps done.
// Two graph replays are kept in flight: each one's result block (loop state, iteration
// counts, lattice F and theta) is copied to a pinned host slot behind it, and the host
// reads a replay's state while the next one runs; the
// replay after the one that ends the run (every unit below eps) finds nothing to do.
// Replays are planned as if all their sweeps ran; a sweep left open idles the rest of
// its replay, so whenever nothing is in flight the plan restarts from the sweeps done.
int run_phase(gf_handle* h, double eps, int budget, int* done) {
  DevState s{};
  const int offset = h->sweeps_done;
  s.sweep = offset;
  s.limit = offset + budget;
  s.check_interval = h->check_interval;
  s.reunit_interval = h->reunit_interval;
  s.n_active = 0;
  s.ticket = 0;
  s.eps = eps;
  s.eps_mid = eps;
  s.final_level = 1;
  s.hist_n = h->hist_n;
  s.hist_base = h->hist_sweeps - offset;
  h->res_slot = -1;
  // from pinned memory: no staging copy on the host (the previous upload from this slot
  // completed before the previous phase read any replay)
  std::memcpy(h->res_host + 2 * h->res_stride, &s, sizeof s);
  GF_CK(h, cudaMemcpyAsync(h->d_state, h->res_host + 2 * h->res_stride, sizeof s, cudaMemcpyHostToDevice,
                           h->stream));
  int rc = budget == 0 ? enqueue_measure_all(h, FINISH_RESET) : enqueue_opening(h);
  if (rc != GF_OK) return rc;
  if ((rc = ensure_graphs(h)) != GF_OK) return rc;
  int planned = 0, inflight = 0, w = 0, r = 0, drained_at = -1, last = -1;
  bool stop = budget == 0;
  for (;;) {
    while (!stop && inflight < 2 && planned < budget) {
      const int k = graph_index(budget - planned);
      GF_CK(h, cudaGraphLaunch(h->graph[h->cur][k], h->stream));
      GF_CK(h, cudaMemcpyAsync(h->res_host + w * h->res_stride, h->ws + h->L.iters, h->res_bytes,
                               cudaMemcpyDeviceToHost, h->stream));
      GF_CK(h, cudaEventRecord(h->st_ev[w], h->stream));
      planned += kGraphSweeps >> k;
      w ^= 1;
      ++inflight;
    }
    if (inflight == 0) break;
    GF_CK(h, cudaEventSynchronize(h->st_ev[r]));
    s = *res_state(h, r);
    last = r;
    r ^= 1;
    --inflight;
    if (s.n_active == 0 || s.sweep >= s.limit) stop = true;
    if (inflight == 0) {
      // every replay sweeps at least once while units are active: no progress since the
      // previous drain means a broken loop state, not a slow unit
      if (!stop && s.sweep == drained_at) return fail(h, GF_ECUDA, "sweep loop made no progress");
      drained_at = s.sweep;
      planned = s.sweep - offset;
    }
  }
  // the last replay read is the last work of the phase: its slot holds the results
  int slot = last;
  if (budget == 0 || planned == 0) {
    if ((rc = read_state(h, &s)) != GF_OK) return rc;
    slot = -1;
  }
  if (s.hold) {  // not expected: every replay ends with its open sweep resolved
    if ((rc = resolve_open_sweep(h)) != GF_OK) return rc;
    if ((rc = read_state(h, &s)) != GF_OK) return rc;
    slot = -1;
  }
  *done = s.sweep - offset;
  h->hist_n = s.hist_n;
  h->last_active = s.n_active;
  h->res_slot = slot;
  return GF_OK;
}

// ---------------------------------------------------------------------------------
// Mixed precision with a precision level per lattice.  Level 1 is the handle's FP32
// storage, level 2 the double-float polish copy, level 3 the FP64-18 copy (levels 2 and 3
// share the polish buffer).  A unit's mask entry is its level while it sweeps, 0 once it
// is below eps at level 3, and -level once it is below the threshold of a lower level
// (eps_switch for level 1, eps for level 2).  Between graph replays the host moves every
// lattice whose units all wait to the next level (a lattice is the unit of storage: the
// time slices of a Coulomb lattice share its temporal links, which every slice's site
// updates transform, so they change precision together), and measures the moved units
// in the new precision before they sweep again.  Each replay runs the kernels of the
// levels that have sweeping units; a unit that starts waiting in the middle of a replay
// idles until its end (at most kGraphSweeps - 1 sweeps).
// ---------------------------------------------------------------------------------
int level_storage(const gf_handle* h, int L) { return L == 1 ? h->storage : L == 2 ? kSplit18 : GF_FP64_18; }
char* level_links(const gf_handle* h, int L) { return L == 1 ? h->links : h->links64; }
LatDev* level_lats(const gf_handle* h, int L) { return L == 1 ? h->d_lats : h->d_lats64; }

SweepArgs sweep_args_level(gf_handle* h, int L, int parity, int reverse) {
  SweepArgs a = sweep_args(h, parity, true, reverse);
  a.links = level_links(h, L);
  a.lats = level_lats(h, L);
  a.level = L;
  return a;
}

// loop: the even-site pass of a check sweep (units the odd part cannot decide);
// otherwise both parities of the units entering level L (their F from the even pass)
MeasureArgs measure_args_level(gf_handle* h, int L, int parity, int reverse, bool loop) {
  MeasureArgs a = measure_args(h, parity, loop, reverse);
  a.links = level_links(h, L);
  a.lats = level_lats(h, L);
  a.active = h->d_pending;
  a.level = L;
  if (!loop) a.part_F = parity == 0 ? h->d_partF : nullptr;
  return a;
}

// One sweep of the mixed loop over the levels in `mask` (bit L-1 for level L): the
// half-sweeps of every level, then FINISH_ODD; as in the one-level loop, the even-site
// pass of every level and FINISH_LOOP follow in the graph when there are many units,
// and an open sweep of one unit is resolved by the host (resolve_open_sweep_levels).
int enqueue_mixed_sweep(gf_handle* h, cudaStream_t s, int* pass, int mask) {
  int rev = 0;
  for (int parity = 0; parity < 2; ++parity) {
    rev = (*pass)++ & 1;
    for (int L = 1; L <= 3; ++L)
      if (mask & (1 << (L - 1))) {
        launch_sweep(level_storage(h, L), h->nd, h->repro, h->variant, sweep_args_level(h, L, parity, rev),
                     h->n_tiles, h->threads, s);
        GF_CK_LAUNCH(h);
      }
  }
  launch_finish(finish_args(h, FINISH_ODD), s);
  GF_CK_LAUNCH(h);
  if (h->n_units > 1) {
    for (int L = 1; L <= 3; ++L)
      if (mask & (1 << (L - 1))) {
        launch_measure(level_storage(h, L), h->nd, h->variant, measure_args_level(h, L, 0, rev ^ 1, true),
                       h->n_tiles, h->threads, s);
        GF_CK_LAUNCH(h);
      }
    launch_finish(finish_args(h, FINISH_LOOP), s);
    GF_CK_LAUNCH(h);
  }
  return GF_OK;
}

// even-site pass of every level in `mask` (each serves its undecided units) + FINISH_LOOP
int resolve_open_sweep_levels(gf_handle* h, int mask) {
  for (int L = 1; L <= 3; ++L)
    if (mask & (1 << (L - 1))) {
      launch_measure(level_storage(h, L), h->nd, h->variant, measure_args_level(h, L, 0, 0, true), h->n_tiles,
                     h->threads, h->stream);
      GF_CK_LAUNCH(h);
    }
  launch_finish(finish_args(h, FINISH_LOOP), h->stream);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

int ensure_mixed_graph(gf_handle* h, int mask) {
  if (h->graph_mix[mask]) return GF_OK;
  GF_CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = GF_OK, pass = 0;
  for (int j = 0; j < kGraphSweeps && rc == GF_OK; ++j) rc = enqueue_mixed_sweep(h, h->cap_stream, &pass, mask);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (rc != GF_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(h, GF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph_mix[mask], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(h, GF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return GF_OK;
}

// Copy lattice l from level `from` to level `to` (> from).
int convert_lattice(gf_handle* h, int l, int from, int to) {
  if (from == 1 && to == 2) {
    launch_to_split(h->storage, h->links, h->links64, h->lats[l], h->lats64[l], h->stream);
  } else if (from == 1) {
    launch_to_fp64(h->storage, h->links, h->links64, h->lats[l], h->lats64[l], h->stream);
  } else {
    launch_split_to_fp64(h->links64, h->lats64[l], h->stream);
  }
  GF_CK_LAUNCH(h);
  return GF_OK;
}

// Measure the units whose pending entry names the level they just entered (both parities
// in that level's precision), then FINISH_ENTER decides them and recounts the active units.
int enqueue_enter(gf_handle* h, const std::vector<int>& pend) {
  GF_CK(h, cudaMemcpyAsync(h->d_pending, pend.data(), sizeof(int) * pend.size(), cudaMemcpyHostToDevice, h->stream));
  int levels = 0;
  for (int v : pend)
    if (v > 0) levels |= 1 << (v - 1);
  for (int L = 1; L <= 3; ++L)
    if (levels & (1 << (L - 1)))
      for (int parity = 0; parity < 2; ++parity) {
        launch_measure(level_storage(h, L), h->nd, h->variant, measure_args_level(h, L, parity, parity, false),
                       h->n_tiles, h->threads, h->stream);
        GF_CK_LAUNCH(h);
      }
  launch_finish(finish_args(h, FINISH_ENTER), h->stream);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

int run_mixed(gf_handle* h, double eps, int budget, int* sweeps_fp32, int* sweeps_polish, int* sweeps) {
  const bool split = h->polish == GF_POLISH_SPLIT && h->form == GF_OR_FIRST_ORDER;
  const int nu = h->n_units;
  std::vector<int> lev(h->n_lat, 1), act(nu), pend(nu);
  DevState s{};
  s.sweep = 0;
  s.limit = budget;
  s.check_interval = h->check_interval;
  s.reunit_interval = h->reunit_interval;
  s.eps = eps;
  s.eps_mid = std::max(eps, h->eps_switch);
  s.final_level = 3;
  s.hist_n = h->hist_n;
  s.hist_base = 0;
  GF_CK(h, cudaMemcpyAsync(h->d_state, &s, sizeof s, cudaMemcpyHostToDevice, h->stream));
  int rc = enqueue_measure_all(h, FINISH_RESET);  // every unit at level 1
  if (rc != GF_OK) return rc;
  *sweeps_fp32 = *sweeps_polish = 0;
  int mask_prev = 0, sweep_prev = 0;
  // tiles per unit, for the compaction of the tile table as units finish
  std::vector<long long> unit_ntiles(nu, 0);
  for (int l = 0; l < h->n_lat; ++l) {
    const LatDev& d = h->lats[l];
    const long long per_slice = (d.V3h + h->threads - 1) / h->threads;
    for (int k = 0; k < d.n_units; ++k) unit_ntiles[d.unit0 + k] = per_slice * (d.L[3] / d.n_units);
  }
  bool compacted = false;
  // the units of lattice l are lats[l].unit0 .. + n_units - 1
  auto move_lattices = [&](bool to_final) -> int {
    bool moved = false;
    std::fill(pend.begin(), pend.end(), 0);
    for (int l = 0; l < h->n_lat; ++l) {
      const int L = lev[l], u0 = h->lats[l].unit0, n = h->lats[l].n_units;
      if (L == 3) continue;
      bool sweeping = false, waiting = false;
      for (int u = u0; u < u0 + n; ++u) {
        sweeping = sweeping || act[u] == L;
        waiting = waiting || act[u] == -L;
      }
      if (!to_final && (sweeping || !waiting)) continue;
      const int next = to_final ? 3 : (L == 1 && split ? 2 : 3);
      if (to_final && L == 1 && split) {  // the double-float copy on the way, as a polish would
        if ((rc = convert_lattice(h, l, 1, 2)) != GF_OK) return rc;
        if ((rc = convert_lattice(h, l, 2, 3)) != GF_OK) return rc;
      } else if ((rc = convert_lattice(h, l, L, next)) != GF_OK) {
        return rc;
      }
      for (int u = u0; u < u0 + n; ++u)
        if (act[u] != 0) act[u] = pend[u] = next;
      lev[l] = next;
      moved = true;
    }
    if (!moved) return 1;
    GF_CK(h, cudaMemcpyAsync(h->d_active, act.data(), sizeof(int) * nu, cudaMemcpyHostToDevice, h->stream));
    if ((rc = enqueue_enter(h, pend)) != GF_OK) return rc;
    return GF_OK;
  };
  for (;;) {
    if (mask_prev) {  // a replay ran: resolve a sweep it left open
      if ((rc = read_state(h, &s)) != GF_OK) return rc;
      if (s.hold && (rc = resolve_open_sweep_levels(h, mask_prev)) != GF_OK) return rc;
    }
    GF_CK(h, cudaMemcpyAsync(act.data(), h->d_active, sizeof(int) * nu, cudaMemcpyDeviceToHost, h->stream));
    if ((rc = read_state(h, &s)) != GF_OK) return rc;
    if (mask_prev) {
      const int d = s.sweep - sweep_prev;
      if (mask_prev & 1) *sweeps_fp32 += d;
      if (mask_prev & 6) *sweeps_polish += d;
      mask_prev = 0;
    }
    rc = move_lattices(false);
    if (rc < 0) return rc;
    if (rc == GF_OK) continue;  // moved units were measured at their new level: read again
    if (s.n_active == 0 || s.sweep >= s.limit) break;
    int mask = 0;
    long long need = 0;
    for (int u = 0; u < nu; ++u) {
      if (act[u] > 0) mask |= 1 << (act[u] - 1);
      if (act[u] != 0) need += unit_ntiles[u];
    }
    if (nu > 1 && 2 * need <= h->n_tiles) {  // half the table or more belongs to finished units
      std::vector<int> keep(nu);
      for (int u = 0; u < nu; ++u) keep[u] = act[u] != 0;
      if ((rc = build_tiles(h, &keep)) != GF_OK) return rc;  // drops the captured graphs
      compacted = true;
    }
    if ((rc = ensure_mixed_graph(h, mask)) != GF_OK) return rc;
    GF_CK(h, cudaGraphLaunch(h->graph_mix[mask], h->stream));
    mask_prev = mask;
    sweep_prev = s.sweep;
  }
  // every lattice ends in the FP64 copy (what gf_download and the next calls read); the
  // ones moved here are measured and decided in FP64
  if (compacted && (rc = build_tiles(h)) != GF_OK) return rc;  // every unit for the final measurement
  rc = move_lattices(true);
  if (rc < 0) return rc;
  if ((rc = read_state(h, &s)) != GF_OK) return rc;
  h->cur = 1;
  h->hist_n = s.hist_n;
  h->last_active = s.n_active;
  *sweeps = s.sweep;
  return GF_OK;
}

// The requested results: from the result block that the loop which just ended copied
// behind its last replay (lattice totals and iteration counts), else through the
// handle's pinned staging with asynchronous copies and one synchronisation (a copy into
// pageable memory would block on each call).
int copy_out(gf_handle* h, double* F, double* theta, double* uF, double* uT, int* iters) {
  const int slot = h->res_slot;
  h->res_slot = -1;
  if (slot >= 0 && !uF && !uT) {
    const char* b = h->res_host + slot * h->res_stride;
    if (iters) std::memcpy(iters, b, sizeof(int) * h->n_units);
    if (F) std::memcpy(F, b + (h->L.lF - h->L.iters), sizeof(double) * h->n_lat);
    if (theta) std::memcpy(theta, b + (h->L.lT - h->L.iters), sizeof(double) * h->n_lat);
    return GF_OK;
  }
  double* sF = reinterpret_cast<double*>(h->out_host);
  double* sT = sF + h->n_lat;
  double* suF = sT + h->n_lat;
  double* suT = suF + h->n_units;
  int* sI = reinterpret_cast<int*>(suT + h->n_units);
  const size_t bl = sizeof(double) * h->n_lat, bu = sizeof(double) * h->n_units;
  if (F) GF_CK(h, cudaMemcpyAsync(sF, h->d_lF, bl, cudaMemcpyDeviceToHost, h->stream));
  if (theta) GF_CK(h, cudaMemcpyAsync(sT, h->d_lT, bl, cudaMemcpyDeviceToHost, h->stream));
  if (uF) GF_CK(h, cudaMemcpyAsync(suF, h->d_uF, bu, cudaMemcpyDeviceToHost, h->stream));
  if (uT) GF_CK(h, cudaMemcpyAsync(suT, h->d_uT, bu, cudaMemcpyDeviceToHost, h->stream));
  if (iters) GF_CK(h, cudaMemcpyAsync(sI, h->d_iters, sizeof(int) * h->n_units, cudaMemcpyDeviceToHost, h->stream));
  GF_CK(h, cudaStreamSynchronize(h->stream));
  if (F) std::memcpy(F, sF, bl);
  if (theta) std::memcpy(theta, sT, bl);
  if (uF) std::memcpy(uF, suF, bu);
  if (uT) std::memcpy(uT, suT, bu);
  if (iters) std::memcpy(iters, sI, sizeof(int) * h->n_units);
  return GF_OK;
}

// ---------------------------------------------------------------------------------
// Fourier-accelerated steepest descent (Algorithm 2)
// ---------------------------------------------------------------------------------
FasdArgs fasd_args(gf_handle* h, bool loop, int mode) {
  FasdArgs a{};
  a.links = h->links;
  a.lat = h->lats[0];
  a.kbuf = h->kbuf;
  a.gbuf = h->gbuf;
  a.plane_F = h->d_planeF;
  a.plane_th = h->d_planeT;
  a.unit_planes = h->d_unit_planes;
  a.active = loop ? h->d_active : nullptr;
  a.iters = h->d_iters;
  a.unit_sumF = h->d_usF;
  a.unit_sumTh = h->d_usT;
  a.unit_F = h->d_uF;
  a.unit_theta = h->d_uT;
  a.lat_F = h->d_lF;
  a.lat_theta = h->d_lT;
  a.st = loop ? h->d_state : nullptr;
  a.nd = h->nd;
  a.n_units = h->n_units;
  a.reunit = 0;
  a.mode = mode;
  for (int k = 0; k < 4; ++k) {
    int l = 0;
    while ((1 << l) < a.lat.L[k]) ++l;
    a.logL[k] = l;
  }
  const double nfft = h->nd == 4 ? (double)a.lat.V : 2.0 * a.lat.V3h;
  a.coef = 0.5 * h->alpha * (4.0 * h->nd) / nfft;
  a.kx = fasd_kx(a.lat, h->nd, h->storage == GF_FP64_18 ? 16 : 8);
  a.xy_prefetch = fasd_xy_prefetch(h->storage, h->nd);
  a.zt_prefetch = fasd_zt_prefetch(h->storage, h->nd);
  return a;
}

// One iteration: Delta + F/theta (A, B), then, while running, C, D, E (E counts it).
int enqueue_fasd_iteration(gf_handle* h, cudaStream_t s) {
  const FasdArgs a = fasd_args(h, true, FINISH_LOOP);
  launch_fasd_delta_xy(h->storage, h->nd, a, s);
  GF_CK_LAUNCH(h);
  launch_fasd_finish(a, s);
  GF_CK_LAUNCH(h);
  launch_fasd_zt(h->storage, h->nd, a, s);
  GF_CK_LAUNCH(h);
  launch_fasd_xy_inv_g(h->storage, h->nd, a, s);
  GF_CK_LAUNCH(h);
  launch_fasd_update(h->storage, h->nd, a, s);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

int run_fasd(gf_handle* h, double eps, int budget, int* done) {
  DevState st{};
  const int offset = h->sweeps_done;
  st.sweep = offset;
  st.limit = offset + budget;
  st.check_interval = 1;
  st.reunit_interval = h->reunit_interval;
  st.n_active = h->n_units;
  st.ticket = 0;
  st.stop = 0;
  st.eps = eps;
  GF_CK(h, cudaMemcpyAsync(h->d_state, &st, sizeof st, cudaMemcpyHostToDevice, h->stream));
  launch_fill_int(h->d_active, 1, h->n_units, h->stream);
  GF_CK_LAUNCH(h);
  if (!h->graph_fasd) {
    GF_CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = GF_OK;
    for (int j = 0; j < kGraphSweeps && rc == GF_OK; ++j) rc = enqueue_fasd_iteration(h, h->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (rc != GF_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(h, GF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->graph_fasd, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, GF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  int rc;
  do {  // until every unit converged or the field after the budget has been measured
    GF_CK(h, cudaGraphLaunch(h->graph_fasd, h->stream));
    if ((rc = read_state(h, &st)) != GF_OK) return rc;
  } while (st.n_active > 0 && !st.stop);
  *done = st.sweep - offset;
  return GF_OK;
}

}  // namespace

// ===================================================================================
// C ABI
// ===================================================================================
extern "C" {

int gf_workspace_bytes(int n_lat, const int* dims, int gauge, int storage, int flags, size_t* bytes) {
  std::string why;
  g_create_error.clear();
  if (!bytes) {
    g_create_error = "bytes must not be NULL";
    return GF_EINVAL;
  }
  int rc = check_common(n_lat, dims, gauge, storage, flags, &why);
  if (rc != GF_OK) {
    g_create_error = why;
    return rc;
  }
  Layout L;
  plan(n_lat, dims, gauge, storage, flags, &L);
  *bytes = L.total;
  return GF_OK;
}

int gf_create_batch(int n_lat, const int* dims, int gauge, int storage, int flags, void* stream,
                    void* workspace, size_t workspace_bytes, gf_handle** out) {
  if (!out) return GF_EINVAL;
  *out = nullptr;
  g_create_error.clear();
  std::string why;
  int rc = check_common(n_lat, dims, gauge, storage, flags, &why);
  if (rc != GF_OK) {
    g_create_error = why;
    return rc;
  }
  gf_handle* h = new (std::nothrow) gf_handle();
  if (!h) {
    g_create_error = "host allocation failed";
    return GF_ENOMEM;
  }
  h->n_lat = n_lat;
  h->gauge = gauge;
  h->nd = gauge == GF_LANDAU ? 4 : 3;
  h->storage = storage;
  h->flags = is_fp64_storage(storage) ? (flags & ~GF_FLAG_MIXED) : flags;
  h->dims.assign(dims, dims + 4 * n_lat);
  h->stream = (cudaStream_t)stream;
  plan(n_lat, dims, gauge, storage, h->flags, &h->L);
  auto bail = [&](int code, const std::string& msg) {
    g_create_error = msg;
    gf_destroy(h);
    return code;
  };
  if (workspace) {
    if (workspace_bytes < h->L.total) return bail(GF_ENOMEM, "workspace smaller than gf_workspace_bytes()");
    if (((uintptr_t)workspace % 16) != 0) return bail(GF_EINVAL, "workspace must be 16-byte aligned");
    h->ws = (char*)workspace;
    h->ws_bytes = workspace_bytes;
  } else {
    cudaError_t e = cudaMalloc(&h->ws, h->L.total);
    if (e != cudaSuccess) {
      h->ws = nullptr;
      return bail(GF_ENOMEM, std::string("cudaMalloc of the workspace: ") + cudaGetErrorString(e));
    }
    h->own_ws = true;
    h->ws_bytes = h->L.total;
  }
  if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(GF_ECUDA, "cudaStreamCreate failed");
  h->res_bytes = h->L.state + sizeof(DevState) - h->L.iters;
  h->res_stride = align_up(h->res_bytes);
  if (cudaHostAlloc((void**)&h->res_host, 3 * h->res_stride, cudaHostAllocDefault) != cudaSuccess) {
    h->res_host = nullptr;
    return bail(GF_ENOMEM, "pinned host memory for the loop state");
  }
  if (cudaHostAlloc((void**)&h->out_host, sizeof(double) * (2 * (size_t)n_lat + 2 * (size_t)h->L.n_units) +
                                              sizeof(int) * (size_t)h->L.n_units,
                    cudaHostAllocDefault) != cudaSuccess) {
    h->out_host = nullptr;
    return bail(GF_ENOMEM, "pinned host memory for the results");
  }
  for (auto& ev : h->st_ev)
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      ev = nullptr;
      return bail(GF_ECUDA, "event creation failed");
    }
  {
    cudaError_t e = prepare_sweep_pipe();
    if (e != cudaSuccess) return bail(GF_ECUDA, std::string("sweep kernel set-up: ") + cudaGetErrorString(e));
  }
  const Layout& L = h->L;
  char* w = h->ws;
  h->links = w + L.links;
  h->links64 = L.links64 == (size_t)-1 ? nullptr : w + L.links64;
  h->staging = w + L.staging;
  h->d_lats = (LatDev*)(w + L.lats);
  h->d_lats64 = (LatDev*)(w + L.lats64);
  h->d_tiles = (int4*)(w + L.tiles);
  h->d_unit_tiles = (int*)(w + L.unit_tiles);
  h->d_unit_lat = (int*)(w + L.unit_lat);
  h->d_active = (int*)(w + L.active);
  h->d_iters = (int*)(w + L.iters);
  h->d_partF = (float2*)(w + L.partF);
  h->d_pthe = (float2*)(w + L.pthe);
  h->d_ptho = (float2*)(w + L.ptho);
  h->d_pending = (int*)(w + L.pending);
  h->d_usTo = (double*)(w + L.usTo);
  h->d_unit_norm = (double*)(w + L.unit_norm);
  if (cudaMemsetAsync(h->d_pending, 0, sizeof(int) * L.n_units, h->stream) != cudaSuccess)
    return bail(GF_ECUDA, "initialisation of the pending masks failed");
  h->d_usF = (double*)(w + L.usF);
  h->d_usT = (double*)(w + L.usT);
  h->d_uF = (double*)(w + L.uF);
  h->d_uT = (double*)(w + L.uT);
  h->d_lF = (double*)(w + L.lF);
  h->d_lT = (double*)(w + L.lT);
  h->d_state = (DevState*)(w + L.state);
  h->n_units = L.n_units;
  if (h->flags & GF_FLAG_AUTOGRAD) {
    h->ad_g = w + L.ad_g;
    h->ad_delta = w + L.ad_delta;
    h->ad_part = (double*)(w + L.ad_part);
    h->ad_ticket = (unsigned int*)(w + L.ad_ticket);
    if (cudaMemsetAsync(h->ad_ticket, 0, sizeof(unsigned int), h->stream) != cudaSuccess)
      return bail(GF_ECUDA, "initialisation of the autograd ticket failed");
  }
  if (h->flags & GF_FLAG_FASD) {
    h->kbuf = w + L.kbuf;
    h->gbuf = w + L.gbuf;
    h->d_planeF = (float2*)(w + L.planeF);
    h->d_planeT = (float2*)(w + L.planeT);
    h->d_unit_planes = (int*)(w + L.unit_planes);
  }

  long long off = 0, off64 = 0;
  int unit = 0;
  for (int l = 0; l < n_lat; ++l) {
    LatDev d{};
    for (int k = 0; k < 4; ++k) d.L[k] = dims[4 * l + k];
    d.V = (long long)d.L[0] * d.L[1] * d.L[2] * d.L[3];
    d.Vh = (int)(d.V / 2);
    d.V3h = d.L[0] * d.L[1] * d.L[2] / 2;
    d.mx = (unsigned int)(((1ULL << 32) + (unsigned long long)d.L[0] - 1) / (unsigned long long)d.L[0]);
    d.my = (unsigned int)(((1ULL << 32) + (unsigned long long)d.L[1] - 1) / (unsigned long long)d.L[1]);
    d.unit0 = unit;
    d.n_units = gauge == GF_LANDAU ? 1 : d.L[3];
    unit += d.n_units;
    d.off_bytes = off;
    off += d.V * 4 * link_bytes(storage);
    h->lats.push_back(d);
    d.off_bytes = off64;
    off64 += d.V * 4 * 144;
    h->lats64.push_back(d);
  }
  if (cudaMemcpyAsync(h->d_lats, h->lats.data(), sizeof(LatDev) * n_lat, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(h->d_lats64, h->lats64.data(), sizeof(LatDev) * n_lat, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return bail(GF_ECUDA, "copy of the lattice tables failed");
  launch_fill_int(h->d_active, 1, h->n_units, h->stream);
  if (cudaMemsetAsync(h->d_iters, 0, sizeof(int) * h->n_units, h->stream) != cudaSuccess ||
      cudaGetLastError() != cudaSuccess)
    return bail(GF_ECUDA, "initialisation of the unit tables failed");
  if (build_tiles(h) != GF_OK) return bail(GF_ECUDA, h->err);
  if (h->flags & GF_FLAG_FASD) {
    // unit plane ranges: planes (z, t) in order; Landau one unit, Coulomb one per t
    const LatDev& d = h->lats[0];
    std::vector<int> up;
    if (gauge == GF_LANDAU) up = {0, d.L[2] * d.L[3]};
    else
      for (int t = 0; t <= d.L[3]; ++t) up.push_back(t * d.L[2]);
    if (cudaMemcpyAsync(h->d_unit_planes, up.data(), sizeof(int) * up.size(), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return bail(GF_ECUDA, "copy of the plane table failed");
    cudaError_t e = prepare_fasd(storage, h->nd, d);
    if (e != cudaSuccess) return bail(GF_ECUDA, std::string("Fourier kernels set-up: ") + cudaGetErrorString(e));
  }
  *out = h;
  return GF_OK;
}

int gf_create(const int dims[4], int nc, int gauge, int storage, int flags, void* stream, void* workspace,
              size_t workspace_bytes, gf_handle** out) {
  if (nc != 3) {
    g_create_error = "only Nc = 3 (SU(3)) is supported";
    if (out) *out = nullptr;
    return GF_EINVAL;
  }
  return gf_create_batch(1, dims, gauge, storage, flags, stream, workspace, workspace_bytes, out);
}

void gf_destroy(gf_handle* h) {
  if (!h) return;
  drop_graphs(h);
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (auto& ev : h->st_ev)
    if (ev) cudaEventDestroy(ev);
  if (h->res_host) cudaFreeHost(h->res_host);
  if (h->out_host) cudaFreeHost(h->out_host);
  if (h->own_ws && h->ws) cudaFree(h->ws);
  delete h;
}

const char* gf_last_error(const gf_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int gf_num_lattices(const gf_handle* h) { return h ? h->n_lat : GF_EINVAL; }
int gf_num_units(const gf_handle* h) { return h ? h->n_units : GF_EINVAL; }

// Device address of host memory that kernels may access directly (pinned with
// cudaHostAlloc or registered, and mapped into the device's address space); nullptr for
// pageable memory, which then goes through the staging buffer.
const double* host_mapped(const double* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of a pointer CUDA does not know
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return nullptr;
  if (((uintptr_t)at.devicePointer % 16) != 0) return nullptr;
  return static_cast<const double*>(at.devicePointer);
}

int gf_upload(gf_handle* h, int lat, const double* links, int on_device) {
  if (!h) return GF_EINVAL;
  if (lat < 0 || lat >= h->n_lat || !links) return fail(h, GF_EINVAL, "bad lattice index or null buffer");
  if (on_device && ((uintptr_t)links % 16) != 0) return fail(h, GF_EINVAL, "device buffer must be 16-byte aligned");
  h->cur = 0;
  h->sweeps_done = 0;
  const LatDev& d = h->lats[lat];
  const double* mapped = on_device ? nullptr : host_mapped(links);
  if (on_device || mapped) {
    // device memory, or pinned host memory the kernel reads directly over the host link
    launch_pack(h->storage, h->links, d, on_device ? links : mapped, 0, d.V, h->stream);
    GF_CK_LAUNCH(h);
  } else {
    const long long per = (long long)(h->L.staging_bytes / (4 * 144));
    for (long long s0 = 0; s0 < d.V; s0 += per) {
      const long long n = std::min(per, d.V - s0);
      GF_CK(h, cudaMemcpyAsync(h->staging, links + s0 * 4 * 18, (size_t)n * 4 * 144, cudaMemcpyHostToDevice, h->stream));
      launch_pack(h->storage, h->links, d, (const double*)h->staging, s0, n, h->stream);
      GF_CK_LAUNCH(h);
    }
  }
  launch_fill_int(h->d_active, 1, h->n_units, h->stream);
  GF_CK_LAUNCH(h);
  GF_CK(h, cudaMemsetAsync(h->d_iters, 0, sizeof(int) * h->n_units, h->stream));
  if (!on_device) GF_CK(h, cudaStreamSynchronize(h->stream));
  return GF_OK;
}

int gf_download(gf_handle* h, int lat, double* links, int on_device) {
  if (!h) return GF_EINVAL;
  if (lat < 0 || lat >= h->n_lat || !links) return fail(h, GF_EINVAL, "bad lattice index or null buffer");
  if (on_device && ((uintptr_t)links % 16) != 0) return fail(h, GF_EINVAL, "device buffer must be 16-byte aligned");
  const LatDev& d = cur_lat_host(h, lat);
  const int st = cur_storage(h);
  double* mapped = on_device ? nullptr : const_cast<double*>(host_mapped(links));
  if (on_device || mapped) {
    launch_unpack(st, cur_links(h), d, on_device ? links : mapped, 0, d.V, h->stream);
    GF_CK_LAUNCH(h);
    if (mapped) GF_CK(h, cudaStreamSynchronize(h->stream));
  } else {
    const long long per = (long long)(h->L.staging_bytes / (4 * 144));
    for (long long s0 = 0; s0 < d.V; s0 += per) {
      const long long n = std::min(per, d.V - s0);
      launch_unpack(st, cur_links(h), d, (double*)h->staging, s0, n, h->stream);
      GF_CK_LAUNCH(h);
      GF_CK(h, cudaMemcpyAsync(links + s0 * 4 * 18, h->staging, (size_t)n * 4 * 144, cudaMemcpyDeviceToHost, h->stream));
    }
    GF_CK(h, cudaStreamSynchronize(h->stream));
  }
  return GF_OK;
}

int gf_functional_theta(gf_handle* h, double* F, double* theta, double* unit_F, double* unit_theta) {
  if (!h) return GF_EINVAL;
  // the finishing kernel needs a valid ticket; the loop fields stay as they are
  GF_CK(h, cudaMemsetAsync(&h->d_state->ticket, 0, sizeof(unsigned int), h->stream));
  int rc = enqueue_measure_all(h, FINISH_MEASURE);
  if (rc != GF_OK) return rc;
  return copy_out(h, F, theta, unit_F, unit_theta, nullptr);
}

int gf_or_sweep(gf_handle* h, int parity, double omega) {
  if (!h) return GF_EINVAL;
  if (parity < 0 || parity > 2) return fail(h, GF_EINVAL, "parity must be 0, 1 or 2");
  if (!(omega >= 1.0 && omega < 2.0)) return fail(h, GF_EINVAL, "omega must lie in [1, 2)");
  const int st = cur_storage(h);
  for (int p = 0; p < 2; ++p) {
    if (parity != 2 && p != parity) continue;
    SweepArgs a = sweep_args(h, p, false, p);
    a.omega = omega;
    launch_sweep(st, h->nd, h->repro, h->variant, a, h->n_tiles, h->threads, h->stream);
    GF_CK_LAUNCH(h);
  }
  return GF_OK;
}

int gf_reunitarize(gf_handle* h) {
  if (!h) return GF_EINVAL;
  for (int l = 0; l < h->n_lat; ++l) {
    launch_reunit(cur_storage(h), cur_links(h), cur_lat_host(h, l), h->stream);
    GF_CK_LAUNCH(h);
  }
  return GF_OK;
}

int gf_fix(gf_handle* h, double eps, int maxiter, int* iters, double* F, double* theta) {
  if (!h) return GF_EINVAL;
  if (!(eps > 0.0) || maxiter < 0) return fail(h, GF_EINVAL, "need eps > 0 and maxiter >= 0");
  GF_CK(h, cudaMemsetAsync(h->d_iters, 0, sizeof(int) * h->n_units, h->stream));
  h->phase_sweeps[0] = h->phase_sweeps[1] = 0;
  h->hist_n = 0;
  h->hist_sweeps = 0;
  int rc, done = 0;
  if (h->method == GF_METHOD_FASD) {
    if (!(h->flags & GF_FLAG_FASD)) return fail(h, GF_ESTATE, "create the handle with GF_FLAG_FASD for Fourier acceleration");
    if (h->cur != 0) return fail(h, GF_ESTATE, "upload the field before a Fourier-accelerated fix");
    if ((rc = run_fasd(h, eps, maxiter, &done)) != GF_OK) return rc;
    h->sweeps_done += done;
    h->phase_sweeps[is_fp64_storage(h->storage) ? 1 : 0] = done;
    if ((rc = copy_out(h, F, theta, nullptr, nullptr, iters)) != GF_OK) return rc;
    DevState s{};
    if ((rc = read_state(h, &s)) != GF_OK) return rc;
    return s.n_active > 0 ? GF_ENOTCONVERGED : GF_OK;
  }
  const bool mixed = (h->flags & GF_FLAG_MIXED) && h->cur == 0;
  if (mixed) {
    // one loop over all precision levels; the reunitarisation and check schedules count
    // the loop's sweeps from the start of this call
    if ((rc = run_mixed(h, eps, maxiter, &h->phase_sweeps[0], &h->phase_sweeps[1], &done)) != GF_OK) return rc;
    h->sweeps_done = done;
  } else {
    if ((rc = run_phase(h, eps, maxiter, &done)) != GF_OK) return rc;
    h->sweeps_done += done;
    h->phase_sweeps[h->cur == 1 || is_fp64_storage(h->storage) ? 1 : 0] = done;
  }
  if ((rc = copy_out(h, F, theta, nullptr, nullptr, iters)) != GF_OK) return rc;
  return h->last_active > 0 ? GF_ENOTCONVERGED : GF_OK;
}

int gf_set_omega(gf_handle* h, double omega) {
  if (!h) return GF_EINVAL;
  if (!(omega >= 1.0 && omega < 2.0)) return fail(h, GF_EINVAL, "omega must lie in [1, 2)");
  if (omega != h->omega) drop_graphs(h);
  h->omega = omega;
  return GF_OK;
}

int gf_set_overrelax_form(gf_handle* h, int form) {
  if (!h) return GF_EINVAL;
  if (form != GF_OR_FIRST_ORDER && form != GF_OR_EXACT) return fail(h, GF_EINVAL, "unknown overrelaxation form");
  if (form != h->form) drop_graphs(h);
  h->form = form;
  return GF_OK;
}

int gf_set_reunit_interval(gf_handle* h, int n) {
  if (!h) return GF_EINVAL;
  if (n < 0) return fail(h, GF_EINVAL, "reunit interval must be >= 0");
  h->reunit_interval = n;
  return GF_OK;
}

int gf_set_check_interval(gf_handle* h, int n) {
  if (!h) return GF_EINVAL;
  if (n < 1) return fail(h, GF_EINVAL, "check interval must be >= 1");
  h->check_interval = n;
  return GF_OK;
}

int gf_set_mixed_switch(gf_handle* h, double eps_sw) {
  if (!h) return GF_EINVAL;
  if (!(eps_sw > 0.0)) return fail(h, GF_EINVAL, "switch threshold must be > 0");
  h->eps_switch = eps_sw;
  return GF_OK;
}

int gf_set_reproducible(gf_handle* h, int on) {
  if (!h) return GF_EINVAL;
  if ((on != 0) != h->repro) drop_graphs(h);
  h->repro = on != 0;
  return GF_OK;
}

int gf_set_block_size(gf_handle* h, int threads) {
  if (!h) return GF_EINVAL;
  if (threads != 64 && threads != 128 && threads != 256) return fail(h, GF_EINVAL, "block size must be 64, 128 or 256");
  if (threads == h->threads) return GF_OK;
  h->threads = threads;
  return build_tiles(h);
}

static int ad_args(gf_handle* h, const double* c, AdArgs* a) {
  if (!(h->flags & GF_FLAG_AUTOGRAD)) return fail(h, GF_ESTATE, "create the handle with GF_FLAG_AUTOGRAD");
  if (h->cur != 0) return fail(h, GF_ESTATE, "upload the field first");
  if (!c || ((uintptr_t)c % 8) != 0) return fail(h, GF_EINVAL, "c must be 8-byte aligned device memory");
  *a = AdArgs{};
  a->links = h->links;
  a->lat = h->lats[0];
  a->c = c;
  a->g = (c64*)h->ad_g;
  a->delta = (c64*)h->ad_delta;
  a->part = h->ad_part;
  a->ticket = h->ad_ticket;
  a->nd = h->nd;
  return GF_OK;
}

int gf_ad_functional(gf_handle* h, const double* c, double* out) {
  if (!h) return GF_EINVAL;
  AdArgs a;
  int rc = ad_args(h, c, &a);
  if (rc != GF_OK) return rc;
  if (!out) return fail(h, GF_EINVAL, "out must be device memory for 2 doubles");
  a.out = out;
  launch_ad_forward(a, h->stream);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

int gf_ad_backward(gf_handle* h, const double* c, const double* upstream, double* grad) {
  if (!h) return GF_EINVAL;
  AdArgs a;
  int rc = ad_args(h, c, &a);
  if (rc != GF_OK) return rc;
  if (!upstream || !grad) return fail(h, GF_EINVAL, "upstream and grad must be device memory");
  a.upstream = upstream;
  a.grad = grad;
  launch_ad_backward(a, h->stream);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

int gf_fa_sd_step(gf_handle* h, double alpha) {
  if (!h) return GF_EINVAL;
  if (!(h->flags & GF_FLAG_FASD)) return fail(h, GF_ESTATE, "create the handle with GF_FLAG_FASD for Fourier acceleration");
  if (h->cur != 0) return fail(h, GF_ESTATE, "upload the field before a Fourier-accelerated step");
  if (!(alpha > 0.0)) return fail(h, GF_EINVAL, "alpha must be > 0");
  const double keep = h->alpha;
  h->alpha = alpha;
  FasdArgs a = fasd_args(h, false, FINISH_MEASURE);
  h->alpha = keep;
  launch_fasd_delta_xy(h->storage, h->nd, a, h->stream);
  GF_CK_LAUNCH(h);
  launch_fasd_zt(h->storage, h->nd, a, h->stream);
  GF_CK_LAUNCH(h);
  launch_fasd_xy_inv_g(h->storage, h->nd, a, h->stream);
  GF_CK_LAUNCH(h);
  launch_fasd_update(h->storage, h->nd, a, h->stream);
  GF_CK_LAUNCH(h);
  return GF_OK;
}

int gf_set_method(gf_handle* h, int method) {
  if (!h) return GF_EINVAL;
  if (method != GF_METHOD_OR && method != GF_METHOD_FASD) return fail(h, GF_EINVAL, "unknown method");
  if (method == GF_METHOD_FASD && !(h->flags & GF_FLAG_FASD))
    return fail(h, GF_ESTATE, "create the handle with GF_FLAG_FASD for Fourier acceleration");
  h->method = method;
  return GF_OK;
}

int gf_set_alpha(gf_handle* h, double alpha) {
  if (!h) return GF_EINVAL;
  if (!(alpha > 0.0)) return fail(h, GF_EINVAL, "alpha must be > 0");
  if (alpha != h->alpha) drop_graphs(h);
  h->alpha = alpha;
  return GF_OK;
}

int gf_set_polish(gf_handle* h, int polish) {
  if (!h) return GF_EINVAL;
  if (polish != GF_POLISH_FP64 && polish != GF_POLISH_SPLIT) return fail(h, GF_EINVAL, "unknown polish mode");
  h->polish = polish;
  return GF_OK;
}

int gf_set_sweep_variant(gf_handle* h, int variant) {
  if (!h) return GF_EINVAL;
  if (variant != GF_SWEEP_AUTO && variant != GF_SWEEP_REGISTER && variant != GF_SWEEP_PIPELINED)
    return fail(h, GF_EINVAL, "unknown sweep variant");
  if (variant == GF_SWEEP_PIPELINED && h->storage != GF_FP32_12)
    return fail(h, GF_EINVAL, "the pipelined sweep exists for GF_FP32_12 storage only");
  if (variant != h->variant) drop_graphs(h);
  h->variant = variant;
  return GF_OK;
}

int gf_autotune(gf_handle* h, int* threads_out, int* variant_out) {
  if (!h) return GF_EINVAL;
  // Time a few sweeps of the current field for every launch shape and keep the fastest.
  // The tuning sweeps act on the field itself: they are gauge transformations (the
  // gauge-invariant content is unchanged), but a run meant to start from the original
  // configuration uploads it again afterwards.
  const int st = cur_storage(h);
  std::vector<std::pair<int, int>> cands;
  for (int t : {64, 128, 256}) {
    cands.push_back({t, GF_SWEEP_REGISTER});
    if (st == GF_FP32_12) cands.push_back({t, GF_SWEEP_PIPELINED});
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail(h, GF_ECUDA, "event creation failed");
  }
  float best = 1e30f;
  int bt = h->threads, bv = h->variant;
  int rc = GF_OK;
  for (auto& c : cands) {
    h->variant = c.second;
    if ((rc = gf_set_block_size(h, c.first)) != GF_OK) break;
    for (int k = 0; k < 2 && rc == GF_OK; ++k) rc = gf_or_sweep(h, 2, h->omega);  // warm-up
    if (rc != GF_OK) break;
    if (cudaEventRecord(e0, h->stream) != cudaSuccess) { rc = fail(h, GF_ECUDA, "event record failed"); break; }
    for (int k = 0; k < 5 && rc == GF_OK; ++k) rc = gf_or_sweep(h, 2, h->omega);
    if (rc != GF_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = fail(h, GF_ECUDA, "event timing failed");
      break;
    }
    if (ms < best) {
      best = ms;
      bt = c.first;
      bv = c.second;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GF_OK) return rc;
  h->variant = bv;
  drop_graphs(h);
  if ((rc = gf_set_block_size(h, bt)) != GF_OK) return rc;
  if (threads_out) *threads_out = bt;
  if (variant_out) *variant_out = bv;
  return GF_OK;
}

int gf_get_sweeps_done(const gf_handle* h, int* n) {
  if (!h || !n) return GF_EINVAL;
  *n = h->sweeps_done;
  return GF_OK;
}

int gf_set_sweeps_done(gf_handle* h, int n) {
  if (!h) return GF_EINVAL;
  if (n < 0) return fail(h, GF_EINVAL, "sweep count must be >= 0");
  h->sweeps_done = n;
  return GF_OK;
}

int gf_fix_phase_sweeps(const gf_handle* h, int* fp32_sweeps, int* fp64_sweeps) {
  if (!h) return GF_EINVAL;
  if (fp32_sweeps) *fp32_sweeps = h->phase_sweeps[0];
  if (fp64_sweeps) *fp64_sweeps = h->phase_sweeps[1];
  return GF_OK;
}

int gf_set_history(gf_handle* h, double* buf, int capacity) {
  if (!h) return GF_EINVAL;
  if (capacity < 0 || (capacity > 0 && buf == nullptr)) return fail(h, GF_EINVAL, "history needs a buffer for capacity > 0 records");
  if (buf && ((uintptr_t)buf % 8) != 0) return fail(h, GF_EINVAL, "history buffer must be 8-byte aligned");
  h->hist = capacity > 0 ? buf : nullptr;
  h->hist_cap = capacity > 0 ? capacity : 0;
  h->hist_n = 0;
  drop_graphs(h);  // the finishing kernels of the captured loop carry the buffer
  return GF_OK;
}

int gf_history_count(const gf_handle* h, int* n) {
  if (!h || !n) return GF_EINVAL;
  *n = h->hist_n;
  return GF_OK;
}

}  // extern "C"
