// Host side of the C ABI declared in include/eik.h: argument checks, the
// per-device workspace, host<->device staging, launch sequence, capacity
// retries and status read-back.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/eik.h"
#include "eik_internal.h"

namespace {

using eik::Ctl;
using eik::Prob;
using eik::SeedItem;
using eik::SolveParams;

std::mutex g_mu;
char g_err[512] = "";

void set_err(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

constexpr int64_t kMaxCells = int64_t(1) << 40;
constexpr uint64_t kMaxCapEntries = uint64_t(1) << 30;   // whole ring storage limit
// Defaults per dimension (from parameter sweeps on the 2D layered and 3D
// checkerboard workloads): bucket width in cell travel times, look-ahead
// window in buckets, in-tile acceptance band, persistent CTAs per SM.
// Defaults per dimension (2D, 3D), from sweeps over the 2D layered, constant
// and tomography workloads and the 3D checkerboard and batched workloads.
// adjoint schedule by default: the tile schedule (else level-synchronous)
constexpr bool kAdjTilesDefault = true;
constexpr double kDefaultKDelta[2] = {16.0, 2.0};   // single 2D front, 3D integer d-bar
constexpr int kDefaultWindow[2] = {16, 31};      // single 2D front, 3D (2D batches: 16)
constexpr double kDefaultBand[2] = {16.0, 6.0};  // single 2D front, 3D (2D batches: 8)
constexpr int kDefaultCtasPerSm[2] = {1, 2};   // per 256 cells of tile (single 2D front)
// 3D on the FP64 unit: 4x4x4 tiles; a single front (under 8 sources) takes
// buckets of 0.75 cell travel times and 14 CTAs of 64 cells per SM, many
// fronts (a batch) buckets of 0.375 and the 20 CTAs of the wide lean build.  A single
// front's extra CTAs pick up tiles ahead of it and redo them; a batch has
// enough independent fronts to keep them busy, and narrow buckets cut its
// speculative evaluations.
constexpr int kShape3 = 4;
constexpr double kKDelta3[2] = {0.75, 0.375};   // single front, many fronts
constexpr int kSingleFrontCtas3Small = 14;      // 3D tiles of at most 64 cells
constexpr int kManyFronts = 8;                  // sources at which a solve counts as many fronts
constexpr int kMaxRetries = 4;
// eik_opts.sched_flags bits of the tomography interface
constexpr int kFlagSlowness = 1 << 6;     // speed arrays hold slowness s; v = fl(1/s) is used
constexpr int kFlagSumShared = 1 << 7;    // eik_adjoint: equal outputs receive the ordered sum
int from_slowness(const eik_opts *opts) { return opts && (opts->sched_flags & kFlagSlowness) ? 1 : 0; }

// Grow-only device buffer.
template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t want) {
    if (want <= n && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(want, 1) * sizeof(T));
    if (e == cudaSuccess) n = std::max<size_t>(want, 1);
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

struct Workspace {
  int device = -1;
  DevBuf<double> r;            // c = fl(fl(h/v)^2) per cell, all problems
  DevBuf<double> t_stage;      // host out_t staging
  DevBuf<double> v_stage;      // host speed staging
  DevBuf<unsigned long long> state;
  DevBuf<unsigned char> tile_src;
  DevBuf<unsigned> pend;
  DevBuf<unsigned long long> slots;
  DevBuf<unsigned> seq;
  DevBuf<int64_t> src_idx;
  DevBuf<double> src_t;
  DevBuf<SeedItem> seeds;
  DevBuf<Prob> probs;
  DevBuf<Ctl> ctl;
  DevBuf<unsigned long long> count;
  DevBuf<const double *> sum_ptr;   // eik_sum_ordered's pointer table
  DevBuf<eik::CopyItem> copies;     // host outputs written by the copy kernel
  DevBuf<double> slab_t;       // eik_solve_slabs: each slab's field (own rows + ghost rows)
  DevBuf<double> slab_x;       // eik_solve_slabs: exchanged boundary rows
  Ctl *ctl_host = nullptr;     // pinned
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  uint64_t cap = 0;            // entries per slot

  void release_all() {
    r.release(); t_stage.release(); v_stage.release(); state.release(); tile_src.release();
    pend.release();
    slots.release(); seq.release(); src_idx.release(); src_t.release(); seeds.release();
    copies.release();
    probs.release(); ctl.release(); count.release(); sum_ptr.release(); slab_t.release();
    slab_x.release();
    if (ctl_host) cudaFreeHost(ctl_host);
    ctl_host = nullptr;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    ev0 = ev1 = nullptr;
    cap = 0;
    device = -1;
  }
};

// Workspaces are kept per device (indexed by the CUDA device ordinal); g_dev
// is the device of the call in progress, set under the API lock.
constexpr int kMaxDevices = 64;
int g_dev = 0;
Workspace g_ws_dev[kMaxDevices];
Workspace &ws() { return g_ws_dev[g_dev]; }

struct AdjWorkspace {
  int device = -1;
  DevBuf<int> cnt, cnt_out;
  DevBuf<double> W, lam;
  DevBuf<unsigned char> mask, status;
  DevBuf<unsigned long long> front, ring;
  DevBuf<unsigned> tile_state;
  DevBuf<eik::AdjProb> probs;
  DevBuf<eik::AdjCtl> ctl;
  DevBuf<int64_t> src;
  DevBuf<double> gsum;                   // per-problem gradients summed into shared outputs
  DevBuf<const double *> gptr;           // their addresses, grouped by output
  eik::AdjCtl *ctl_host = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  void release_all() {
    cnt.release(); cnt_out.release(); W.release(); lam.release(); mask.release();
    status.release(); front.release(); ring.release(); tile_state.release();
    probs.release(); ctl.release(); src.release(); gsum.release(); gptr.release();
    if (ctl_host) cudaFreeHost(ctl_host);
    ctl_host = nullptr;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    ev0 = ev1 = nullptr;
    device = -1;
  }
};
AdjWorkspace g_adj_dev[kMaxDevices];
AdjWorkspace &adj() { return g_adj_dev[g_dev]; }

// Workspace of the comparison schedules (opts.schedule 1, 2).
struct BspWorkspace {
  int device = -1;
  DevBuf<double> c;
  DevBuf<unsigned char> fixed;
  DevBuf<unsigned> mark;
  DevBuf<unsigned long long> front;
  DevBuf<eik::BspCtl> ctl;
  DevBuf<int64_t> src;
  DevBuf<double> src_t;
  eik::BspCtl *ctl_host = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  void release_all() {
    c.release(); fixed.release(); mark.release(); front.release(); ctl.release(); src.release();
    src_t.release();
    if (ctl_host) cudaFreeHost(ctl_host);
    ctl_host = nullptr;
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    ev0 = ev1 = nullptr;
    device = -1;
  }
};
BspWorkspace g_bsp_dev[kMaxDevices];
BspWorkspace &bsp() { return g_bsp_dev[g_dev]; }

}  // namespace

namespace eik {
std::mutex &api_mutex() { return g_mu; }
void set_last_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
}  // namespace eik

namespace {

eik_status cuda_fail(cudaError_t e, const char *what) {
  set_err("%s: %s", what, cudaGetErrorString(e));
  return EIK_ECUDA;
}

#define CK(call, what)                                            \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) {                                      \
      if (e_ == cudaErrorMemoryAllocation) {                      \
        set_err("%s: %s", what, cudaGetErrorString(e_));          \
        cudaGetLastError();                                       \
        return EIK_ENOMEM;                                        \
      }                                                           \
      return cuda_fail(e_, what);                                 \
    }                                                             \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Page-locked (pinned or registered) host memory: copies from and to it can
// be enqueued asynchronously and captured in a CUDA graph.
#ifndef EIK_MAPPED_COPIES
#define EIK_MAPPED_COPIES 1
#endif
bool is_pinned_host(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// The device's address of pinned host memory (mapped: with unified addressing
// all pinned memory is), or NULL when it has none.
const void *mapped_ptr(const void *host) {
#if EIK_MAPPED_COPIES
  void *d = nullptr;
  if (cudaHostGetDevicePointer(&d, const_cast<void *>(host), 0) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return d;
#else
  (void)host;
  return nullptr;
#endif
}

uint64_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

struct HostProblem {
  const double *speed;
  bool speed_dev;
  double h;
  int ndim;
  int64_t dims[3];
  int64_t n;
  std::vector<int64_t> src;    // sorted unique
  std::vector<double> t0;
  double *out;
  bool out_dev;
};

eik_status check_problem(const double *speed, double h, int ndim, const int64_t *dims,
                         const int64_t *src_idx, const double *src_t, int64_t nsrc,
                         double *out_t, HostProblem &hp, cudaStream_t stream) {
  if (ndim != 2 && ndim != 3) { set_err("ndim must be 2 or 3 (got %d)", ndim); return EIK_EINVAL; }
  if (!dims) { set_err("dims is NULL"); return EIK_EINVAL; }
  int64_t n = 1;
  for (int k = 0; k < ndim; ++k) {
    if (dims[k] < 1) { set_err("dims[%d] = %lld < 1", k, (long long)dims[k]); return EIK_EINVAL; }
    if (dims[k] > kMaxCells || n > kMaxCells / dims[k]) { set_err("grid too large"); return EIK_EINVAL; }
    n *= dims[k];
  }
  if (!(h > 0.0) || !std::isfinite(h)) { set_err("h must be finite and > 0"); return EIK_EINVAL; }
  if (!speed || !out_t) { set_err("speed and out_t must not be NULL"); return EIK_EINVAL; }
  if (nsrc < 0 || (nsrc > 0 && !src_idx)) { set_err("bad source arguments"); return EIK_EINVAL; }
  hp.speed = speed;
  hp.speed_dev = is_device_ptr(speed);
  hp.h = h;
  hp.ndim = ndim;
  hp.dims[0] = hp.dims[1] = hp.dims[2] = 1;
  for (int k = 0; k < ndim; ++k) hp.dims[3 - ndim + k] = dims[k];
  hp.n = n;
  hp.out = out_t;
  hp.out_dev = is_device_ptr(out_t);
  std::vector<int64_t> idx(static_cast<size_t>(nsrc));
  std::vector<double> tt(static_cast<size_t>(nsrc), 0.0);
  if (nsrc > 0) {
    bool copied = false;
    if (is_device_ptr(src_idx)) {
      CK(cudaMemcpyAsync(idx.data(), src_idx, nsrc * sizeof(int64_t), cudaMemcpyDeviceToHost, stream),
         "copy src_idx");
      copied = true;
    } else {
      std::memcpy(idx.data(), src_idx, nsrc * sizeof(int64_t));
    }
    if (src_t) {
      if (is_device_ptr(src_t)) {
        CK(cudaMemcpyAsync(tt.data(), src_t, nsrc * sizeof(double), cudaMemcpyDeviceToHost, stream),
           "copy src_t");
        copied = true;
      } else {
        std::memcpy(tt.data(), src_t, nsrc * sizeof(double));
      }
    }
    if (copied) CK(cudaStreamSynchronize(stream), "sync sources");
  }
  std::vector<std::pair<int64_t, double>> st(static_cast<size_t>(nsrc));
  for (int64_t i = 0; i < nsrc; ++i) {
    if (idx[i] < 0 || idx[i] >= n) { set_err("source %lld index %lld out of range", (long long)i, (long long)idx[i]); return EIK_EINVAL; }
    double v = tt[i];
    if (!(v >= 0.0) || !std::isfinite(v)) { set_err("source %lld time must be finite and >= 0", (long long)i); return EIK_EINVAL; }
    if (v == 0.0) v = 0.0;   // -0 -> +0
    st[i] = {idx[i], v};
  }
  std::sort(st.begin(), st.end());
  hp.src.clear();
  hp.t0.clear();
  for (auto &e : st) {
    if (!hp.src.empty() && hp.src.back() == e.first) continue;   // sorted: first is the min
    hp.src.push_back(e.first);
    hp.t0.push_back(e.second);
  }
  return EIK_OK;
}

// Automatic tile shape and bucket width.  With many independent wavefronts
// (3D grids, 2D batches of at least 8 sources) every CTA has work and smaller
// tiles with narrower buckets finish sooner; a single 2D front is latency-bound
// and wants large tiles and wide buckets.  (Chosen with the autotuner on the
// layered, tomography, checkerboard and batched workloads.)  The integer-pipe
// arithmetic has the first shape only.
struct AutoCfg {
  int shape;
  double k_delta;
  double band;
  int window;
};
AutoCfg auto_config(int ndim, int64_t total_sources, bool int_arith) {
  if (int_arith) return {0, kDefaultKDelta[ndim == 3 ? 1 : 0], ndim == 3 ? 8.0 : 16.0, 16};
  if (ndim == 3)
    return {kShape3, kKDelta3[total_sources >= kManyFronts ? 1 : 0], kDefaultBand[1], kDefaultWindow[1]};
  if (total_sources >= kManyFronts) return {3, 4.0, 8.0, 16};
  return {0, kDefaultKDelta[0], kDefaultBand[0], kDefaultWindow[0]};
}

int64_t count_sources(const std::vector<HostProblem> &hps) {
  int64_t n = 0;
  for (const HostProblem &hp : hps) n += (int64_t)hp.src.size();
  return n;
}

// Tile shape of opts (validated): shape index and cells per axis.  opts.tile 0
// is automatic; 1..kNumTileShapes name shape tile - 1.
eik_status tile_shape(const eik_opts *opts, int ndim, int64_t total_sources, int &shape,
                      int64_t &tx, int64_t &ty, int64_t &tz) {
  const int t = opts ? opts->tile : 0;
  const bool int_arith = opts && opts->arith == 2;
  if (t < 0 || t > eik::kNumTileShapes) {
    set_err("opts.tile must be in 0..%d", eik::kNumTileShapes);
    return EIK_EINVAL;
  }
  shape = t == 0 ? auto_config(ndim, total_sources, int_arith).shape : t - 1;
  if (shape != 0 && int_arith) {
    set_err("integer-pipe arithmetic (arith 2) runs the first tile shape only (opts.tile 0 or 1)");
    return EIK_EINVAL;
  }
  const eik::TileShape ts = eik::tile_shape_of(ndim, shape);
  tx = ts.tx;
  ty = ts.ty;
  tz = ts.tz;
  return EIK_OK;
}

// Update form of opts (validated): 0 = d-bar; 1 = d-tilde, 2 = d-hat (2D).
eik_status update_form(const eik_opts *opts, int ndim, int &form) {
  form = opts ? opts->update : 0;
  if (opts && (opts->sched_flags & 32) && form == 0) {
    set_err("change tracking (sched_flags bit 5) applies to the explicit update forms only");
    return EIK_EINVAL;
  }
  if (form == 0) return EIK_OK;
  if (form < 0 || form > 3) { set_err("opts.update must be 0, 1, 2 or 3"); return EIK_EINVAL; }
  if (ndim != 2) { set_err("the explicit update forms (opts.update 1-3) are 2D only"); return EIK_EINVAL; }
  return EIK_OK;
}

// Lane-group d-bar (several lanes per listed cell) pays when a solve is
// latency-bound, i.e. has few tiles per persistent CTA; with many tiles per
// CTA the FP64 pipe is better spent on one lane per cell.  sched_flags bits
// 1-2 override: 1 = never, 2 = lists of up to a quarter of the tile, 3 = an
// eighth.
int lane_group_cells(const eik_opts *opts, int64_t tile_cells, int64_t total_tiles, int64_t grid) {
  const int mode = opts ? (opts->sched_flags >> 1) & 3 : 0;
  if (mode == 1) return 0;
  if (mode == 2) return (int)(tile_cells / 4);
  if (mode == 3) return (int)(tile_cells / 8);
  return total_tiles < 8 * grid ? (int)(tile_cells / 4) : 0;
}

// Default persistent CTAs per SM: the per-dimension default for 256-cell
// tiles, scaled up for smaller tiles.  A 2D batch with many sources has as
// many independent wavefronts, enough work for two CTAs per SM (the 32-source
// 1024^2 tomography forward: 75 ms against 93 ms with one); a single front
// runs faster with one.  wide_occ: resident CTAs per SM of the shape's wide
// lean build (0: none), which many fronts fill (the 88-problem 3D batch:
// 110.9 ms at 20 CTAs per SM against 112.8 ms at 16).
int default_ctas_per_sm(int di, int64_t tile_cells, int64_t total_sources, int wide_occ) {
  // one 2D front is latency-bound on few tiles: one CTA per SM; otherwise as
  // many CTAs as the register budget of the tile size allows
  if (di == 0 && total_sources < kManyFronts)
    return (int)std::max<int64_t>(1, kDefaultCtasPerSm[0] * 256 / tile_cells);
  // one 3D front on 64-cell tiles: a little short of the register budget
  if (di == 1 && total_sources < kManyFronts && tile_cells <= 64)
    return std::min(kSingleFrontCtas3Small, eik::resident_ctas((int)tile_cells));
  if (total_sources >= kManyFronts && wide_occ > 0) return wide_occ;
  return eik::resident_ctas((int)tile_cells);
}

// Persistent grid of a launch: the CTAs per SM requested (else the default),
// capped by what the instantiation to launch holds resident, so that every
// CTA is resident.  More CTAs than the normal build holds take the wide lean
// build where the shape has one and the launch is lean (every other field of
// sp already set); else the normal build's count.  Sets sp.lane_group_cells
// and sp.wide.
int64_t size_grid(SolveParams &sp, const eik_opts *opts, int ndim, int shape, int64_t tile_cells,
                  int64_t total_sources, int64_t total_tiles, int sms) {
  const int occ = eik::persistent_blocks_per_sm(ndim, sp.arith, shape);
  const int occ_wide = eik::persistent_wide_blocks_per_sm(ndim, sp.arith, shape);
  const int per_sm = opts && opts->ctas_per_sm > 0
                         ? opts->ctas_per_sm
                         : default_ctas_per_sm(ndim == 3 ? 1 : 0, tile_cells, total_sources, occ_wide);
  auto grid_of = [&](int per) {
    return std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per, total_tiles));
  };
  sp.wide = 0;
  int64_t grid = grid_of(std::min(per_sm, std::max(occ, occ_wide)));
  sp.lane_group_cells = lane_group_cells(opts, tile_cells, total_tiles, grid);
  if (per_sm > occ) {
    if (occ_wide > 0 && eik::persistent_launch_is_lean(sp)) {
      sp.wide = 1;
    } else {
      grid = grid_of(occ);
      sp.lane_group_cells = lane_group_cells(opts, tile_cells, total_tiles, grid);
    }
  }
  return grid;
}

// Select the current device's workspaces for the call in progress.
eik_status select_device() {
  int dev = 0;
  CK(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) { set_err("device ordinal %d beyond %d", dev, kMaxDevices); return EIK_EINVAL; }
  g_dev = dev;
  ws().device = dev;
  adj().device = dev;
  bsp().device = dev;
  return EIK_OK;
}

eik_status ensure_device() {
  eik_status st = select_device();
  if (st != EIK_OK) return st;
  if (!ws().ctl_host) {
    CK(cudaMallocHost(&ws().ctl_host, sizeof(Ctl)), "pinned control block");
  }
  if (!ws().ev0) {
    CK(cudaEventCreate(&ws().ev0), "event");
    CK(cudaEventCreate(&ws().ev1), "event");
  }
  return EIK_OK;
}

// A single problem with one of the comparison schedules (Algorithm 3, 4 or 5).
eik_status run_schedule(HostProblem &hp, const eik_opts *opts, eik_stats *stats,
                        cudaStream_t stream) {
  const int schedule = opts->schedule;
  if (schedule != eik::kScheduleFim && schedule != eik::kScheduleTopo &&
      schedule != eik::kScheduleFsm) {
    set_err("opts.schedule must be 0, 1, 2 or 3");
    return EIK_EINVAL;
  }
  if (!hp.speed_dev || !hp.out_dev) { set_err("opts.schedule 1-3 take device pointers only"); return EIK_EINVAL; }
  if (opts->update != 0 || opts->arith == 2) {
    set_err("opts.schedule 1-3 run the exact update on the FP64 unit only");
    return EIK_EINVAL;
  }
  eik_status st = ensure_device();
  if (st != EIK_OK) return st;
  const int64_t n = hp.n;
  const size_t ns = hp.src.size();
  CK(bsp().c.ensure((size_t)n), "schedule: c");
  CK(bsp().fixed.ensure((size_t)n), "schedule: flags");
  CK(bsp().mark.ensure((size_t)n * 2), "schedule: marks");
  CK(bsp().front.ensure((size_t)n * 2), "schedule: worklists");
  CK(bsp().ctl.ensure(1), "schedule: control");
  CK(ws().ctl.ensure(1), "schedule: validation block");
  CK(bsp().src.ensure(std::max<size_t>(ns, 1)), "schedule: sources");
  CK(bsp().src_t.ensure(std::max<size_t>(ns, 1)), "schedule: source times");
  if (!bsp().ctl_host) CK(cudaMallocHost(&bsp().ctl_host, sizeof(eik::BspCtl)), "schedule: pinned");
  if (!bsp().ev0) {
    CK(cudaEventCreate(&bsp().ev0), "schedule: event");
    CK(cudaEventCreate(&bsp().ev1), "schedule: event");
  }
  if (ns) {
    CK(cudaMemcpyAsync(bsp().src.p, hp.src.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, stream),
       "schedule: upload sources");
    CK(cudaMemcpyAsync(bsp().src_t.p, hp.t0.data(), ns * sizeof(double), cudaMemcpyHostToDevice, stream),
       "schedule: upload source times");
  }
  CK(cudaMemsetAsync(bsp().fixed.p, 0, (size_t)n, stream), "schedule: clear flags");
  CK(cudaMemsetAsync(bsp().mark.p, 0, (size_t)n * 2 * sizeof(unsigned), stream), "schedule: clear marks");
  CK(cudaMemsetAsync(bsp().ctl.p, 0, sizeof(eik::BspCtl), stream), "schedule: clear control");
  CK(cudaMemsetAsync(ws().ctl.p, 0, sizeof(Ctl), stream), "schedule: clear validation");
  CK(eik::launch_init_c(hp.speed, hp.h, bsp().c.p, n, ws().ctl.p, stream, 0, from_slowness(opts)),
     "schedule: c");
  CK(eik::launch_init_t(hp.out, n, stream), "schedule: t");
  eik::BspParams bp;
  std::memset(&bp, 0, sizeof(bp));
  bp.t = hp.out;
  bp.c = bsp().c.p;
  bp.ndim = hp.ndim;
  bp.nx = hp.dims[2];
  bp.ny = hp.dims[1];
  bp.nz = hp.dims[0];
  bp.fixed = bsp().fixed.p;
  bp.mark[0] = bsp().mark.p;
  bp.mark[1] = bsp().mark.p + n;
  bp.front[0] = bsp().front.p;
  bp.front[1] = bsp().front.p + n;
  bp.ctl = bsp().ctl.p;
  bp.timeout_ns = (opts->timeout_ms > 0 ? opts->timeout_ms : 60000) * 1000000ll;
  CK(eik::launch_bsp_seed(bp, bsp().src.p, bsp().src_t.p, (int64_t)ns, stream), "schedule: seed");
  CK(cudaMemcpyAsync(ws().ctl_host, ws().ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, stream),
     "schedule: validation");
  CK(cudaStreamSynchronize(stream), "schedule: set-up");
  if (ws().ctl_host->status == eik::kEinval) {
    set_err("invalid input data (cell %llu: speed must be finite and > 0, h/v finite and > 0)",
            (unsigned long long)ws().ctl_host->error_info[0]);
    return EIK_EINVAL;
  }
  CK(cudaEventRecord(bsp().ev0, stream), "schedule: event");
  CK(eik::launch_schedule(schedule, bp, stream), "schedule launch");
  CK(cudaEventRecord(bsp().ev1, stream), "schedule: event");
  CK(cudaMemcpyAsync(bsp().ctl_host, bsp().ctl.p, sizeof(eik::BspCtl), cudaMemcpyDeviceToHost, stream),
     "schedule: status");
  unsigned long long finite = 0;
  if (opts->counters) {
    CK(ws().count.ensure(1), "schedule: count");
    CK(cudaMemsetAsync(ws().count.p, 0, sizeof(unsigned long long), stream), "schedule: count");
    eik::Prob P;
    std::memset(&P, 0, sizeof(P));
    P.t = hp.out;
    P.nx = bp.nx;
    P.ny = bp.ny;
    P.nz = bp.nz;
    CK(eik::launch_count_finite(&P, 1, ws().count.p, stream), "schedule: count");
    CK(cudaMemcpyAsync(&finite, ws().count.p, sizeof(finite), cudaMemcpyDeviceToHost, stream),
       "schedule: count");
  }
  CK(cudaStreamSynchronize(stream), "schedule");
  const eik::BspCtl &c = *bsp().ctl_host;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->evals = (int64_t)c.evals;
    stats->decreases = (int64_t)c.decreases;
    stats->rounds = (int64_t)c.rounds;
    if (opts->counters) stats->good = (int64_t)finite - (int64_t)ns;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, bsp().ev0, bsp().ev1) == cudaSuccess) stats->solve_ms = ms;
  }
  if (c.status == eik::kEtimeout) { set_err("device wait timed out"); return EIK_ETIMEOUT; }
  if (c.status != 0) return EIK_ECUDA;
  return EIK_OK;
}

// The whole solve for a list of host-checked problems (1 = eik_solve).
eik_status run(std::vector<HostProblem> &hps, const eik_opts *opts, eik_stats *stats,
               cudaStream_t stream) {
  eik_status st = ensure_device();
  if (st != EIK_OK) return st;
  const int ndim = hps[0].ndim;
  for (auto &hp : hps) {
    if (hp.ndim != ndim) { set_err("all problems of a batch must have the same ndim"); return EIK_EINVAL; }
  }
  if (opts && opts->schedule != 0) {
    if (hps.size() != 1) { set_err("opts.schedule 1-3 solve single problems only"); return EIK_EINVAL; }
    return run_schedule(hps[0], opts, stats, stream);
  }
  int64_t tx, ty, tz;
  int shape = 0;
  st = tile_shape(opts, ndim, count_sources(hps), shape, tx, ty, tz);
  if (st != EIK_OK) return st;
  int form = 0;
  st = update_form(opts, ndim, form);
  if (st != EIK_OK) return st;
  // distinct speed arrays share one r array
  std::vector<const double *> speeds;
  std::vector<int64_t> speed_off, speed_n;
  std::vector<double> speed_h;
  std::vector<int> prob_speed(hps.size());
  int64_t r_total = 0;
  for (size_t i = 0; i < hps.size(); ++i) {
    int found = -1;
    for (size_t j = 0; j < speeds.size(); ++j)
      if (speeds[j] == hps[i].speed && speed_n[j] == hps[i].n && speed_h[j] == hps[i].h) found = (int)j;
    if (found < 0) {
      found = (int)speeds.size();
      speeds.push_back(hps[i].speed);
      speed_off.push_back(r_total);
      speed_n.push_back(hps[i].n);
      speed_h.push_back(hps[i].h);
      r_total += hps[i].n;
    }
    prob_speed[i] = found;
  }
  // tiles and sources
  std::vector<Prob> probs(hps.size());
  std::vector<SeedItem> seeds;
  int64_t total_tiles = 0, total_src = 0, host_out_cells = 0, host_speed_cells = 0;
  for (auto &hp : hps) {
    total_src += (int64_t)hp.src.size();
    if (!hp.out_dev) host_out_cells += hp.n;
  }
  for (size_t j = 0; j < speeds.size(); ++j) {
    const HostProblem *owner = nullptr;
    for (size_t i = 0; i < hps.size(); ++i) if (prob_speed[i] == (int)j) { owner = &hps[i]; break; }
    if (!owner->speed_dev && !mapped_ptr(speeds[j])) host_speed_cells += speed_n[j];
  }
  CK(ws().r.ensure((size_t)r_total), "alloc r");
  CK(ws().src_idx.ensure((size_t)std::max<int64_t>(total_src, 1)), "alloc src_idx");
  CK(ws().src_t.ensure((size_t)std::max<int64_t>(total_src, 1)), "alloc src_t");
  CK(ws().seeds.ensure((size_t)std::max<int64_t>(total_src, 1)), "alloc seeds");
  CK(ws().probs.ensure(hps.size()), "alloc probs");
  CK(ws().ctl.ensure(1), "alloc ctl");
  CK(ws().count.ensure(1), "alloc count");
  if (host_out_cells) CK(ws().t_stage.ensure((size_t)host_out_cells), "alloc t staging");
  if (host_speed_cells) CK(ws().v_stage.ensure((size_t)host_speed_cells), "alloc speed staging");

  std::vector<int64_t> all_src;
  std::vector<double> all_t0;
  all_src.reserve((size_t)total_src);
  all_t0.reserve((size_t)total_src);
  int64_t out_stage_off = 0;
  for (size_t i = 0; i < hps.size(); ++i) {
    HostProblem &hp = hps[i];
    Prob &P = probs[i];
    P.nx = hp.dims[2];
    P.ny = hp.dims[1];
    P.nz = hp.dims[0];
    P.ntx = (P.nx + tx - 1) / tx;
    P.nty = (P.ny + ty - 1) / ty;
    P.ntz = (P.nz + tz - 1) / tz;
    P.tile_base = total_tiles;
    total_tiles += P.ntx * P.nty * P.ntz;
    P.c = ws().r.p + speed_off[prob_speed[i]];
    if (hp.out_dev) {
      P.t = hp.out;
    } else {
      P.t = ws().t_stage.p + out_stage_off;
      out_stage_off += hp.n;
    }
    P.src_idx = ws().src_idx.p + all_src.size();
    P.src_t = ws().src_t.p + all_src.size();
    P.nsrc = (int64_t)hp.src.size();
    for (size_t k = 0; k < hp.src.size(); ++k) {
      seeds.push_back(SeedItem{(int64_t)i, hp.src[k], hp.t0[k]});
      all_src.push_back(hp.src[k]);
      all_t0.push_back(hp.t0[k]);
    }
  }
  if (total_tiles >= (int64_t(1) << 32)) { set_err("too many tiles"); return EIK_EINVAL; }
  CK(ws().state.ensure((size_t)total_tiles), "alloc tile state");
  CK(ws().tile_src.ensure((size_t)total_tiles), "alloc tile flags");
  CK(ws().pend.ensure((size_t)total_tiles * eik::kPendWords), "alloc pending masks");

  // frontier capacity per bucket slot
  uint64_t want_cap = opts && opts->capacity > 0 ? (uint64_t)opts->capacity
                                                 : (uint64_t)total_tiles / 4 + 4096;
  want_cap = next_pow2(std::max<uint64_t>(want_cap, opts && opts->capacity > 0 ? 16 : 1024));
  while (want_cap * eik::kNumSlots > kMaxCapEntries && want_cap > 1024) want_cap >>= 1;
  // the ring layout depends on cap; storage only grows.  Entries need no
  // clearing: the sequence words (zeroed below) say which positions hold one.
  CK(ws().slots.ensure((size_t)(want_cap * eik::kNumSlots)), "alloc frontier");
  CK(ws().seq.ensure((size_t)(want_cap * eik::kNumSlots)), "alloc frontier sequence");
  ws().cap = want_cap;

  // uploads
  if (!all_src.empty()) {
    CK(cudaMemcpyAsync(ws().src_idx.p, all_src.data(), all_src.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice, stream), "upload sources");
    CK(cudaMemcpyAsync(ws().src_t.p, all_t0.data(), all_t0.size() * sizeof(double),
                       cudaMemcpyHostToDevice, stream), "upload source times");
    CK(cudaMemcpyAsync(ws().seeds.p, seeds.data(), seeds.size() * sizeof(SeedItem),
                       cudaMemcpyHostToDevice, stream), "upload seeds");
  }
  CK(cudaMemcpyAsync(ws().probs.p, probs.data(), probs.size() * sizeof(Prob),
                     cudaMemcpyHostToDevice, stream), "upload problems");
  CK(cudaMemsetAsync(ws().ctl.p, 0, sizeof(Ctl), stream), "clear control block");
  CK(cudaMemsetAsync(ws().state.p, 0, (size_t)total_tiles * sizeof(unsigned long long), stream),
     "clear tile states");
  CK(cudaMemsetAsync(ws().tile_src.p, 0, (size_t)total_tiles, stream), "clear tile flags");
  CK(cudaMemsetAsync(ws().pend.p, 0, (size_t)total_tiles * eik::kPendWords * sizeof(unsigned),
                     stream), "clear pending masks");
  CK(cudaMemsetAsync(ws().seq.p, 0, (size_t)(want_cap * eik::kNumSlots) * sizeof(unsigned), stream),
     "clear frontier sequence");

  // r = h / v (staging host speeds first)
  int64_t v_off = 0;
  for (size_t j = 0; j < speeds.size(); ++j) {
    const HostProblem *owner = nullptr;
    for (size_t i = 0; i < hps.size(); ++i) if (prob_speed[i] == (int)j) { owner = &hps[i]; break; }
    const double *vsrc = speeds[j];
    if (!owner->speed_dev) {
      // pinned host speeds: init_c reads them in place; else a staged copy
      const double *m = static_cast<const double *>(mapped_ptr(vsrc));
      if (m) {
        vsrc = m;
      } else {
        CK(cudaMemcpyAsync(ws().v_stage.p + v_off, vsrc, speed_n[j] * sizeof(double),
                           cudaMemcpyHostToDevice, stream), "upload speed");
        vsrc = ws().v_stage.p + v_off;
        v_off += speed_n[j];
      }
    }
    CK(eik::launch_init_c(vsrc, speed_h[j], ws().r.p + speed_off[j], speed_n[j], ws().ctl.p, stream,
                          form != 0, from_slowness(opts)), "init_c launch");
  }
  int64_t max_cells = 0;
  for (auto &P : probs) max_cells = std::max<int64_t>(max_cells, P.nx * P.ny * P.nz);
  CK(eik::launch_init_t_all(ws().probs.p, (int)probs.size(), max_cells, stream), "init_t launch");

  SolveParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.probs = ws().probs.p;
  sp.nprob = (int)probs.size();
  sp.ndim = ndim;
  sp.state = ws().state.p;
  sp.tile_src = ws().tile_src.p;
  sp.pend = ws().pend.p;
  const AutoCfg ac = auto_config(ndim, total_src, opts && opts->arith == 2);
  sp.window = (unsigned)(opts && opts->window > 0 ? opts->window : ac.window);
  sp.band = opts && opts->band > 0 ? opts->band : ac.band;
  sp.arith = opts && opts->arith == 2 ? eik::kArithInt : eik::kArithFp64;
  sp.gate_pending_only = opts && (opts->sched_flags & 1) ? 1 : 0;
  sp.tile_shape = shape;
  sp.update = form;
  sp.track_changes = opts && (opts->sched_flags & 32) ? 1 : 0;
  sp.visit_budget = sp.track_changes ? (unsigned long long)total_tiles * 256ull + 4096ull : 0ull;
  sp.trace = opts && opts->trace && opts->trace_cap > 0 ? static_cast<eik::TraceRec *>(opts->trace)
                                                        : nullptr;
  sp.trace_cap = sp.trace ? (unsigned long long)opts->trace_cap : 0ull;
  sp.slots = ws().slots.p;
  sp.seq = ws().seq.p;
  sp.cap_mask = (unsigned)(ws().cap - 1);
  sp.ctl = ws().ctl.p;
  const int64_t tmo_ms = opts && opts->timeout_ms > 0 ? opts->timeout_ms : 60000;
  sp.timeout_ns = tmo_ms * 1000000ll;
  sp.counters = opts ? opts->counters : 0;
  sp.test_stall = opts ? opts->test_stall : 0;
  const double k_delta = opts && opts->k_delta > 0 ? opts->k_delta : ac.k_delta;
  const double delta_fixed = opts && opts->delta > 0 ? opts->delta : 0.0;

  CK(eik::launch_seed(sp, ws().seeds.p, (int64_t)seeds.size(), k_delta, delta_fixed, stream),
     "seed launch");
  int dev_sms = 0;
  CK(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ws().device), "SM count");
  const int64_t grid = size_grid(sp, opts, ndim, shape, tx * ty * tz, total_src, total_tiles, dev_sms);

  eik_stats acc;
  std::memset(&acc, 0, sizeof(acc));
  unsigned status = 0;
  for (int attempt = 0;; ++attempt) {
    CK(cudaEventRecord(ws().ev0, stream), "event record");
    CK(eik::launch_persistent(sp, (int)grid, stream), "solve launch");
    CK(cudaEventRecord(ws().ev1, stream), "event record");
    CK(cudaMemcpyAsync(ws().ctl_host, ws().ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, stream),
       "read status");
    CK(cudaStreamSynchronize(stream), "solve");
    float kms = 0.f;
    CK(cudaEventElapsedTime(&kms, ws().ev0, ws().ev1), "event time");
    acc.solve_ms += kms;
    const Ctl &c = *ws().ctl_host;
    status = c.status;
    acc.evals += (int64_t)c.stats[eik::kStatEvals];
    acc.decreases += (int64_t)c.stats[eik::kStatDecreases];
    acc.visits += (int64_t)c.stats[eik::kStatVisits];
    acc.pushes += (int64_t)c.stats[eik::kStatPushes];
    acc.stale_pops += (int64_t)c.stats[eik::kStatStale];
    acc.rounds += (int64_t)c.stats[eik::kStatRounds];
    acc.max_queue = std::max<int64_t>(acc.max_queue, (int64_t)c.stats[eik::kStatMaxQueue]);
    acc.visit_ns += (int64_t)c.stats[eik::kStatVisitNs];
    acc.idle_ns += (int64_t)c.stats[eik::kStatIdleNs];
    acc.ctas = grid;
    acc.trace_n = (int64_t)c.trace_n;
    for (int k = 0; k < 9; ++k) acc.detail[k] += (int64_t)c.stats[eik::kStatCycLoad + k];
    if (status != eik::kEcapacity || attempt >= kMaxRetries ||
        ws().cap * 4 * eik::kNumSlots > kMaxCapEntries) break;
    // grow the frontier, clear the scheduler (keep delta) and resume
    const uint64_t ncap = ws().cap * 4;
    CK(ws().slots.ensure((size_t)(ncap * eik::kNumSlots)), "grow frontier");
    CK(ws().seq.ensure((size_t)(ncap * eik::kNumSlots)), "grow frontier sequence");
    ws().cap = ncap;
    sp.slots = ws().slots.p;
    sp.seq = ws().seq.p;
    sp.cap_mask = (unsigned)(ncap - 1);
    CK(cudaMemsetAsync(ws().seq.p, 0, (size_t)(ncap * eik::kNumSlots) * sizeof(unsigned), stream),
       "clear frontier sequence");
    CK(cudaMemsetAsync(ws().ctl.p, 0, offsetof(Ctl, rsum), stream), "clear scheduler");
    CK(cudaMemsetAsync(&ws().ctl.p->stats[0], 0, sizeof(Ctl) - offsetof(Ctl, stats), stream),
       "clear counters");
    CK(cudaMemsetAsync(ws().state.p, 0, (size_t)total_tiles * sizeof(unsigned long long), stream),
       "clear tile states");
    CK(eik::launch_reseed(sp, probs.data(), (int)probs.size(), stream), "reseed launch");
    acc.retries++;
  }
  if (status != 0) {
    const Ctl &c = *ws().ctl_host;
    if (status == eik::kEinval) {
      set_err("invalid input data (cell %llu: speed must be finite and > 0, h/v finite and > 0)",
              (unsigned long long)c.error_info[0]);
      return EIK_EINVAL;
    }
    if (status == eik::kEtimeout) {
      set_err("device wait timed out (site %llu)", (unsigned long long)c.error_info[0]);
      return EIK_ETIMEOUT;
    }
    if (status == eik::kEcapacity) {
      set_err("frontier capacity exhausted");
      return EIK_ECAPACITY;
    }
    set_err("device status %u", status);
    return EIK_ECUDA;
  }
  if (sp.counters) {
    CK(cudaMemsetAsync(ws().count.p, 0, sizeof(unsigned long long), stream), "clear count");
    CK(eik::launch_count_finite_all(ws().probs.p, (int)probs.size(), max_cells, ws().count.p,
                                    stream), "count");
    unsigned long long finite = 0;
    CK(cudaMemcpyAsync(&finite, ws().count.p, sizeof(finite), cudaMemcpyDeviceToHost, stream),
       "read count");
    CK(cudaStreamSynchronize(stream), "count");
    acc.good = (int64_t)finite - total_src;
  }
  // host outputs: written by one copy kernel into the mapped pinned buffers
  // (else a copy per problem)
  std::vector<eik::CopyItem> items;
  int64_t max_n = 0;
  for (size_t i = 0; i < hps.size(); ++i) {
    if (hps[i].out_dev) continue;
    double *m = static_cast<double *>(const_cast<void *>(mapped_ptr(hps[i].out)));
    if (m) {
      items.push_back(eik::CopyItem{probs[i].t, m, hps[i].n});
      max_n = std::max<int64_t>(max_n, hps[i].n);
    } else {
      CK(cudaMemcpyAsync(hps[i].out, probs[i].t, hps[i].n * sizeof(double), cudaMemcpyDeviceToHost,
                         stream), "download t");
    }
  }
  if (!items.empty()) {
    CK(ws().copies.ensure(items.size()), "alloc copy list");
    CK(cudaMemcpyAsync(ws().copies.p, items.data(), items.size() * sizeof(eik::CopyItem),
                       cudaMemcpyHostToDevice, stream), "upload copy list");
    CK(eik::launch_copy_items(ws().copies.p, (int)items.size(), max_n, stream), "copy launch");
  }
  CK(cudaStreamSynchronize(stream), "download");
  if (stats) *stats = acc;
  return EIK_OK;
}


}  // namespace

extern "C" {

eik_status eik_solve(const double *speed, double h, int ndim, const int64_t *dims,
                     const int64_t *src_idx, const double *src_t, int64_t nsrc, double *out_t,
                     const eik_opts *opts, eik_stats *stats, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<HostProblem> hps(1);
  eik_status st = check_problem(speed, h, ndim, dims, src_idx, src_t, nsrc, out_t, hps[0], s);
  if (st != EIK_OK) return st;
  return run(hps, opts, stats, s);
}

eik_status eik_solve_batched(const eik_problem *probs, int nprob, const eik_opts *opts,
                             eik_stats *stats, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nprob <= 0 || !probs) { set_err("empty batch"); return EIK_EINVAL; }
  std::vector<HostProblem> hps((size_t)nprob);
  for (int i = 0; i < nprob; ++i) {
    const eik_problem &q = probs[i];
    eik_status st = check_problem(q.speed, q.h, q.ndim, q.dims, q.src_idx, q.src_t, q.nsrc,
                                  q.out_t, hps[(size_t)i], s);
    if (st != EIK_OK) return st;
  }
  return run(hps, opts, stats, s);
}

// Autotuner: coordinate descent over the scheduling parameters, timing the
// persistent launch of the caller's own batch.  The fixed point does not
// depend on the schedule (Theorem 1), so every trial must reproduce the first
// trial's bits; a device digest of all outputs checks that.
eik_status eik_autotune(const eik_problem *probs, int nprob, const eik_opts *base, int repeats,
                        eik_opts *best, eik_tune_trial *trials, int max_trials, int *ntrials,
                        void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ntrials) *ntrials = 0;
  if (nprob <= 0 || !probs || !best) { set_err("bad autotune arguments"); return EIK_EINVAL; }
  if (repeats <= 0) repeats = 2;
  std::vector<HostProblem> hps((size_t)nprob);
  int64_t max_cells = 0;
  for (int i = 0; i < nprob; ++i) {
    const eik_problem &q = probs[i];
    eik_status st = check_problem(q.speed, q.h, q.ndim, q.dims, q.src_idx, q.src_t, q.nsrc,
                                  q.out_t, hps[(size_t)i], s);
    if (st != EIK_OK) return st;
    if (!hps[(size_t)i].speed_dev || !hps[(size_t)i].out_dev) {
      set_err("eik_autotune takes device pointers only (problem %d)", i);
      return EIK_EINVAL;
    }
    max_cells = std::max<int64_t>(max_cells, hps[(size_t)i].n);
  }
  const int ndim = hps[0].ndim;
  if (base && base->schedule != 0) {
    set_err("eik_autotune tunes the asynchronous schedule (opts.schedule 0)");
    return EIK_EINVAL;
  }
  if (base && base->update != 0) {
    set_err("eik_autotune needs the exact update (opts.update 0): only then are the bits "
            "independent of the schedule");
    return EIK_EINVAL;
  }
  eik_opts cur;
  std::memset(&cur, 0, sizeof(cur));
  if (base) cur = *base;
  cur.counters = 0;
  cur.test_stall = 0;
  cur.trace = nullptr;
  cur.trace_cap = 0;
  const bool int_arith = cur.arith == 2;
  {
    // start from the automatic choice, named explicitly
    const AutoCfg ac = auto_config(ndim, count_sources(hps), int_arith);
    if (cur.tile <= 0) cur.tile = ac.shape + 1;
    if (cur.k_delta <= 0) cur.k_delta = ac.k_delta;
    if (cur.window <= 0) cur.window = ac.window;
    if (cur.band <= 0) cur.band = ac.band;
  }

  unsigned long long ref[2] = {0, 0};
  bool have_ref = false;
  int n = 0;
  auto trial = [&](const eik_opts &o, double &ms) -> eik_status {
    ms = 1e300;
    eik_status st = EIK_OK;
    for (int r = 0; r < repeats && st == EIK_OK; ++r) {
      std::vector<HostProblem> h2 = hps;
      eik_stats stt;
      st = run(h2, &o, &stt, s);
      if (st != EIK_OK) break;
      ms = std::min(ms, stt.solve_ms);
      if (r == 0) {
        unsigned long long dig[2] = {0, 0};
        CK(ws().count.ensure(2), "autotune: digest buffer");
        CK(cudaMemsetAsync(ws().count.p, 0, 2 * sizeof(unsigned long long), s), "autotune: clear");
        CK(eik::launch_checksum_all(ws().probs.p, nprob, max_cells, ws().count.p, s), "digest");
        CK(cudaMemcpyAsync(dig, ws().count.p, sizeof(dig), cudaMemcpyDeviceToHost, s), "digest");
        CK(cudaStreamSynchronize(s), "digest");
        if (!have_ref) {
          ref[0] = dig[0];
          ref[1] = dig[1];
          have_ref = true;
        } else if (dig[0] != ref[0] || dig[1] != ref[1]) {
          set_err("autotune: trial %d (tile %d, k_delta %g, window %d, band %g, ctas/SM %d) "
                  "changed the result bits", n, o.tile, o.k_delta, o.window, o.band, o.ctas_per_sm);
          return EIK_ECUDA;
        }
      }
    }
    if (trials && n < max_trials) {
      trials[n].opts = o;
      trials[n].ms = st == EIK_OK ? ms : -1.0;
      trials[n].status = (int)st;
      trials[n].reserved = 0;
    }
    ++n;
    return st;
  };

  double best_ms = 0;
  eik_status st = trial(cur, best_ms);
  if (st != EIK_OK) { if (ntrials) *ntrials = std::min(n, max_trials); return st; }
  static const double kds[] = {0.25, 0.375, 0.5, 0.75, 1, 2, 4, 8, 16, 32};
  static const int wins[] = {1, 2, 4, 8, 16, 24, 31};
  static const double bands[] = {1, 2, 4, 6, 8, 12, 16};
  constexpr double kGain = 0.01;   // a change must save more than 1 %
  auto consider = [&](const eik_opts &o) -> eik_status {
    double ms = 0;
    eik_status e = trial(o, ms);
    if (e == EIK_ECUDA) return e;                  // changed bits or a CUDA failure
    if (e == EIK_OK && ms < best_ms * (1.0 - kGain)) { best_ms = ms; cur = o; }
    return EIK_OK;
  };
  for (int pass = 0; pass < 2; ++pass) {
    const eik_opts start = cur;
    if (!int_arith) {
      const int t0 = cur.tile;
      for (int t = 1; t <= eik::kNumTileShapes; ++t) {
        if (t == t0) continue;
        eik_opts o = cur;
        o.tile = t;
        o.ctas_per_sm = 0;
        if ((st = consider(o)) != EIK_OK) break;
      }
      if (st != EIK_OK) break;
    }
    if (cur.delta <= 0) {
      const double k0 = cur.k_delta;
      for (double k : kds) {
        if (k == k0) continue;
        eik_opts o = cur;
        o.k_delta = k;
        if ((st = consider(o)) != EIK_OK) break;
      }
      if (st != EIK_OK) break;
    }
    {
      const int w0 = cur.window;
      for (int w : wins) {
        if (w == w0) continue;
        eik_opts o = cur;
        o.window = w;
        if ((st = consider(o)) != EIK_OK) break;
      }
      if (st != EIK_OK) break;
    }
    {
      const double b0 = cur.band;
      for (double b : bands) {
        if (b == b0) continue;
        eik_opts o = cur;
        o.band = b;
        if ((st = consider(o)) != EIK_OK) break;
      }
      if (st != EIK_OK) break;
    }
    {
      const int ar = int_arith ? eik::kArithInt : eik::kArithFp64;
      const int occ = std::max(eik::persistent_blocks_per_sm(ndim, ar, cur.tile - 1),
                               eik::persistent_wide_blocks_per_sm(ndim, ar, cur.tile - 1));
      const int c0 = cur.ctas_per_sm;
      for (int c = 1; c <= occ; ++c) {
        if (c == c0) continue;
        eik_opts o = cur;
        o.ctas_per_sm = c;
        if ((st = consider(o)) != EIK_OK) break;
      }
      if (st != EIK_OK) break;
    }
    if (std::memcmp(&start, &cur, sizeof(cur)) == 0) break;   // no change in a whole pass
  }
  if (st != EIK_OK) { if (ntrials) *ntrials = std::min(n, max_trials); return st; }
  // frontier capacity from the deepest slot the chosen schedule reaches
  if (!base || base->capacity <= 0) {
    eik_opts o = cur;
    o.counters = 1;
    std::vector<HostProblem> h2 = hps;
    eik_stats stt;
    st = run(h2, &o, &stt, s);
    if (st != EIK_OK) { if (ntrials) *ntrials = std::min(n, max_trials); return st; }
    // the depth varies from run to run with the asynchronous schedule: a wide
    // margin keeps later solves from overflowing (a retry costs a relaunch)
    cur.capacity = (int64_t)next_pow2((uint64_t)std::max<int64_t>(1024, 16 * stt.max_queue));
  }
  *best = cur;
  if (ntrials) *ntrials = std::min(n, max_trials);
  return EIK_OK;
}

// Update-form ablation: one application of Algorithm 1 (or d-bar) per point.
eik_status eik_eval_update(int form, const double *speed, double h, const double *t_h,
                           const double *t_v, int64_t n, double *out, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (form < 0 || form > 3 || n < 0 || !(h > 0.0) || (n > 0 && (!speed || !t_h || !t_v || !out))) {
    set_err("bad eik_eval_update arguments");
    return EIK_EINVAL;
  }
  if (n == 0) return EIK_OK;
  if (!is_device_ptr(speed) || !is_device_ptr(t_h) || !is_device_ptr(t_v) || !is_device_ptr(out)) {
    set_err("eik_eval_update takes device pointers only");
    return EIK_EINVAL;
  }
  CK(eik::launch_eval_update(form, speed, h, t_h, t_v, n, out, s), "eval launch");
  CK(cudaStreamSynchronize(s), "eval");
  return EIK_OK;
}

// The fixed-point residual of Table 3 on the device.
eik_status eik_residual(const eik_problem *prob, int form, int64_t *bad, double *max_rel,
                        void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!prob || !bad || !max_rel) { set_err("bad eik_residual arguments"); return EIK_EINVAL; }
  HostProblem hp;
  eik_status st = check_problem(prob->speed, prob->h, prob->ndim, prob->dims, prob->src_idx,
                                prob->src_t, prob->nsrc, prob->out_t, hp, s);
  if (st != EIK_OK) return st;
  if (!hp.speed_dev || !hp.out_dev) { set_err("eik_residual takes device pointers only"); return EIK_EINVAL; }
  eik_opts o;
  std::memset(&o, 0, sizeof(o));
  o.update = form;
  int f = 0;
  st = update_form(&o, hp.ndim, f);
  if (st != EIK_OK) return st;
  st = ensure_device();
  if (st != EIK_OK) return st;
  const size_t ns = hp.src.size();
  CK(ws().src_idx.ensure(std::max<size_t>(ns, 1)), "residual: sources");
  CK(ws().src_t.ensure(std::max<size_t>(ns, 1)), "residual: source times");
  CK(ws().count.ensure(2), "residual: result");
  if (ns) {
    CK(cudaMemcpyAsync(ws().src_idx.p, hp.src.data(), ns * sizeof(int64_t), cudaMemcpyHostToDevice, s),
       "residual: upload sources");
    CK(cudaMemcpyAsync(ws().src_t.p, hp.t0.data(), ns * sizeof(double), cudaMemcpyHostToDevice, s),
       "residual: upload source times");
  }
  CK(cudaMemsetAsync(ws().count.p, 0, 2 * sizeof(unsigned long long), s), "residual: clear");
  CK(eik::launch_residual(f, hp.ndim, hp.speed, hp.h, hp.out, hp.dims[2], hp.dims[1], hp.dims[0],
                          ws().src_idx.p, ws().src_t.p, (int64_t)ns, ws().count.p, s),
     "residual launch");
  unsigned long long res[2] = {0, 0};
  CK(cudaMemcpyAsync(res, ws().count.p, sizeof(res), cudaMemcpyDeviceToHost, s), "residual: read");
  CK(cudaStreamSynchronize(s), "residual");
  *bad = (int64_t)res[0];
  std::memcpy(max_rel, &res[1], sizeof(double));
  return EIK_OK;
}

// The fixed-order sum of k arrays (the cross-source gradient of a sharded
// tomography step, gathered on one device).
eik_status eik_sum_ordered(const double *const *src, int k, double *dst, int64_t n, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (k < 0 || n < 0 || (k > 0 && !src) || (n > 0 && !dst)) {
    set_err("bad eik_sum_ordered arguments");
    return EIK_EINVAL;
  }
  if (n == 0) return EIK_OK;
  if (!is_device_ptr(dst)) { set_err("eik_sum_ordered takes device pointers only"); return EIK_EINVAL; }
  for (int j = 0; j < k; ++j) {
    if (!is_device_ptr(src[j])) { set_err("eik_sum_ordered: src[%d] is not a device pointer", j); return EIK_EINVAL; }
  }
  eik_status st = ensure_device();
  if (st != EIK_OK) return st;
  CK(ws().sum_ptr.ensure((size_t)std::max(k, 1)), "sum: pointer table");
  if (k > 0) {
    CK(cudaMemcpyAsync(ws().sum_ptr.p, src, (size_t)k * sizeof(const double *), cudaMemcpyHostToDevice, s),
       "sum: upload pointer table");
  }
  CK(eik::launch_sum_ordered(ws().sum_ptr.p, k, dst, n, s), "sum launch");
  CK(cudaStreamSynchronize(s), "sum");
  return EIK_OK;
}

// Slab decomposition of one grid (the domain decomposition the paper leaves
// to future work, Introduction): the outermost axis is split into nslabs
// slabs, each solved as one problem of a batch with a ghost row on each side
// it shares with a neighbour.  The ghost rows hold the neighbour's boundary
// values as fixed sources (finite ones); between epochs the boundary rows are
// copied into an exchange buffer on the device and the epochs repeat until
// no exchanged value changes.  Ghost values only decrease from epoch to epoch
// (the solve is monotone in its boundary values), so the loop ends; at the
// end every cell of every slab satisfies the update with its neighbours'
// final values across the slab boundaries, i.e. the union is the fixed point
// of the whole grid (unique, Theorem 1), bit for bit.  One device runs all
// slabs here; with one slab per GPU the exchange is a peer copy of one row
// into the neighbour's memory.
eik_status eik_solve_slabs(const double *speed, double h, int ndim, const int64_t *dims,
                           const int64_t *src_idx, const double *src_t, int64_t nsrc,
                           double *out_t, int nslabs, const eik_opts *opts, eik_stats *stats,
                           int *epochs, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (epochs) *epochs = 0;
  HostProblem hp;
  eik_status st = check_problem(speed, h, ndim, dims, src_idx, src_t, nsrc, out_t, hp, s);
  if (st != EIK_OK) return st;
  if (!hp.speed_dev || !hp.out_dev) { set_err("eik_solve_slabs takes device speed and out_t"); return EIK_EINVAL; }
  if (opts && (opts->update != 0 || opts->schedule != 0 || (opts->sched_flags & 32) || opts->test_stall)) {
    set_err("eik_solve_slabs runs the exact update (opts.update 0) on the asynchronous schedule");
    return EIK_EINVAL;
  }
  const int64_t L = hp.dims[3 - ndim];                  // outermost extent
  const int64_t plane = hp.n / L;
  if (nslabs < 1 || nslabs > L) { set_err("nslabs must be in 1..%lld", (long long)L); return EIK_EINVAL; }
  st = ensure_device();
  if (st != EIK_OK) return st;
  const int K = nslabs;
  std::vector<int64_t> lo(K + 1), glo(K), ghi(K), toff(K);
  for (int k = 0; k <= K; ++k) lo[k] = (int64_t)k * L / K;
  int64_t tcells = 0;
  for (int k = 0; k < K; ++k) {
    glo[k] = lo[k] > 0 ? lo[k] - 1 : 0;
    ghi[k] = lo[k + 1] < L ? lo[k + 1] + 1 : L;
    toff[k] = tcells;
    tcells += (ghi[k] - glo[k]) * plane;
  }
  // exchange buffer: for boundary b (between slabs b and b+1) two rows: slab b's
  // last own row (slab b+1's ghost) and slab b+1's first own row (slab b's ghost)
  const int64_t nx_rows = 2 * (int64_t)(K - 1);
  CK(ws().slab_t.ensure((size_t)std::max<int64_t>(tcells, 1)), "slabs: fields");
  CK(ws().slab_x.ensure((size_t)std::max<int64_t>(nx_rows * plane, 1)), "slabs: exchange");
  std::vector<double> xprev((size_t)(nx_rows * plane), INFINITY), xcur((size_t)(nx_rows * plane));
  const int max_epochs = 64 + 8 * K;
  eik_stats acc;
  std::memset(&acc, 0, sizeof(acc));
  bool done = false;
  int e = 0;
  for (; e < max_epochs && !done; ++e) {
    std::vector<HostProblem> hps((size_t)K);
    for (int k = 0; k < K; ++k) {
      HostProblem &q = hps[(size_t)k];
      q.speed = speed + glo[k] * plane;
      q.speed_dev = true;
      q.h = hp.h;
      q.ndim = ndim;
      q.dims[0] = q.dims[1] = q.dims[2] = 1;
      for (int a = 0; a < ndim; ++a) q.dims[3 - ndim + a] = hp.dims[3 - ndim + a];
      q.dims[3 - ndim] = ghi[k] - glo[k];
      q.n = q.dims[0] * q.dims[1] * q.dims[2];
      q.out = ws().slab_t.p + toff[k];
      q.out_dev = true;
      // ghost sources first (they precede or follow the own rows, so the list
      // stays sorted with the own sources in between)
      if (k > 0) {                                      // row glo[k] = slab k-1's last own row
        const double *g = xprev.data() + (size_t)(2 * (k - 1)) * plane;
        for (int64_t j = 0; j < plane; ++j)
          if (std::isfinite(g[j])) { q.src.push_back(j); q.t0.push_back(g[j]); }
      }
      for (size_t i = 0; i < hp.src.size(); ++i) {
        const int64_t row = hp.src[i] / plane;
        if (row >= lo[k] && row < lo[k + 1]) {
          q.src.push_back(hp.src[i] - glo[k] * plane);
          q.t0.push_back(hp.t0[i]);
        }
      }
      if (k + 1 < K) {                                  // row ghi[k]-1 = slab k+1's first own row
        const double *g = xprev.data() + (size_t)(2 * k + 1) * plane;
        const int64_t base = (ghi[k] - 1 - glo[k]) * plane;
        for (int64_t j = 0; j < plane; ++j)
          if (std::isfinite(g[j])) { q.src.push_back(base + j); q.t0.push_back(g[j]); }
      }
    }
    eik_stats es;
    st = run(hps, opts, &es, s);
    if (st != EIK_OK) return st;
    acc.evals += es.evals; acc.decreases += es.decreases; acc.visits += es.visits;
    acc.pushes += es.pushes; acc.stale_pops += es.stale_pops; acc.rounds += es.rounds;
    acc.retries += es.retries; acc.max_queue = std::max(acc.max_queue, es.max_queue);
    acc.visit_ns += es.visit_ns; acc.idle_ns += es.idle_ns; acc.ctas = es.ctas;
    acc.solve_ms += es.solve_ms;
    // exchange: each boundary row into the buffer slot of the slab that reads it
    for (int b = 0; b + 1 < K; ++b) {
      const double *last_b = ws().slab_t.p + toff[b] + (lo[b + 1] - 1 - glo[b]) * plane;
      const double *first_b1 = ws().slab_t.p + toff[b + 1] + (lo[b + 1] - glo[b + 1]) * plane;
      CK(cudaMemcpyAsync(ws().slab_x.p + (size_t)(2 * b) * plane, last_b, (size_t)plane * sizeof(double),
                         cudaMemcpyDeviceToDevice, s), "slabs: exchange");
      CK(cudaMemcpyAsync(ws().slab_x.p + (size_t)(2 * b + 1) * plane, first_b1,
                         (size_t)plane * sizeof(double), cudaMemcpyDeviceToDevice, s), "slabs: exchange");
    }
    if (nx_rows > 0)
      CK(cudaMemcpyAsync(xcur.data(), ws().slab_x.p, (size_t)(nx_rows * plane) * sizeof(double),
                         cudaMemcpyDeviceToHost, s), "slabs: read exchange");
    CK(cudaStreamSynchronize(s), "slabs: epoch");
    // global AND: done when no exchanged value changed
    done = std::memcmp(xcur.data(), xprev.data(), xcur.size() * sizeof(double)) == 0;
    xprev.swap(xcur);
  }
  if (!done) {
    set_err("eik_solve_slabs: exchanged values still changing after %d epochs", max_epochs);
    return EIK_ETIMEOUT;
  }
  for (int k = 0; k < K; ++k) {
    CK(cudaMemcpyAsync(out_t + lo[k] * plane, ws().slab_t.p + toff[k] + (lo[k] - glo[k]) * plane,
                       (size_t)((lo[k + 1] - lo[k]) * plane) * sizeof(double), cudaMemcpyDeviceToDevice, s),
       "slabs: assemble");
  }
  if (opts && opts->counters) {
    CK(cudaMemsetAsync(ws().count.p, 0, sizeof(unsigned long long), s), "slabs: count");
    Prob P;
    std::memset(&P, 0, sizeof(P));
    P.t = out_t;
    P.nx = hp.dims[2];
    P.ny = hp.dims[1];
    P.nz = hp.dims[0];
    CK(eik::launch_count_finite(&P, 1, ws().count.p, s), "slabs: count");
    unsigned long long finite = 0;
    CK(cudaMemcpyAsync(&finite, ws().count.p, sizeof(finite), cudaMemcpyDeviceToHost, s), "slabs: count");
    CK(cudaStreamSynchronize(s), "slabs: count");
    acc.good = (int64_t)finite - (int64_t)hp.src.size();
  }
  CK(cudaStreamSynchronize(s), "slabs");
  if (stats) *stats = acc;
  if (epochs) *epochs = e;
  return EIK_OK;
}

void eik_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (select_device() != EIK_OK) return;
  ws().release_all();
  adj().release_all();
  bsp().release_all();
}

const char *eik_status_str(eik_status s) {
  switch (s) {
    case EIK_OK: return "EIK_OK";
    case EIK_EINVAL: return "EIK_EINVAL";
    case EIK_ENOMEM: return "EIK_ENOMEM";
    case EIK_ECAPACITY: return "EIK_ECAPACITY";
    case EIK_ETIMEOUT: return "EIK_ETIMEOUT";
    case EIK_ECUDA: return "EIK_ECUDA";
  }
  return "EIK_UNKNOWN";
}

const char *eik_last_error(void) { return g_err; }

int eik_abi_version(void) { return 108; }

uint64_t eik_kernel_launches(void) { return (uint64_t)eik::kernel_launches(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Plans: a batch of problems prepared once (validation, sources, workspace),
// then solved any number of times by eik_plan_enqueue, which only enqueues
// device work on the stream (no allocation, no host synchronisation), so a
// CUDA graph can capture it.
// ---------------------------------------------------------------------------
struct eik_plan {
  int device = -1;
  int ndim = 2;
  std::vector<Prob> probs;                   // host copies of the device records
  std::vector<const double *> speeds;        // distinct speed arrays (device copies)
  std::vector<const double *> speed_host;    // pinned host sources to copy (NULL: device input,
                                             // or read in place through its mapping)
  std::vector<double *> out_host;            // per problem: pinned host output to copy (NULL:
                                             // device, or written by the copy kernel)
  DevBuf<double> v_stage, t_stage;           // device copies of pinned host inputs / outputs
  DevBuf<eik::CopyItem> copies;              // outputs written through their mapping
  int ncopies = 0;
  int64_t copy_max_n = 0;
  std::vector<int64_t> speed_off, speed_n;
  std::vector<double> speed_h;
  int64_t total_tiles = 0, nseeds = 0, total_src = 0, max_cells = 0;
  DevBuf<double> c;
  DevBuf<unsigned long long> state;
  DevBuf<unsigned char> tile_src;
  DevBuf<unsigned> pend;
  DevBuf<unsigned long long> slots;
  DevBuf<unsigned> seq;
  DevBuf<int64_t> src_idx;
  DevBuf<double> src_t;
  DevBuf<SeedItem> seeds;
  DevBuf<Prob> probs_d;
  DevBuf<Ctl> ctl;
  DevBuf<unsigned long long> count;
  Ctl *ctl_host = nullptr;
  SolveParams sp;
  int grid = 1;
  double k_delta = 0.0, delta_fixed = 0.0;
  int from_slowness = 0;
  uint64_t cap = 0;

  ~eik_plan() {
    v_stage.release(); t_stage.release(); copies.release();
    c.release(); state.release(); tile_src.release(); pend.release(); slots.release();
    seq.release(); src_idx.release(); src_t.release(); seeds.release(); probs_d.release(); ctl.release();
    count.release();
    if (ctl_host) cudaFreeHost(ctl_host);
  }
};

namespace {

eik_status plan_build(eik_plan &pl, std::vector<HostProblem> &hps, const eik_opts *opts,
                      cudaStream_t stream) {
  CK(cudaGetDevice(&pl.device), "cudaGetDevice");
  pl.ndim = hps[0].ndim;
  for (size_t i = 0; i < hps.size(); ++i) {
    const HostProblem &hp = hps[i];
    if (hp.ndim != pl.ndim) { set_err("all problems of a plan must have the same ndim"); return EIK_EINVAL; }
    if ((!hp.speed_dev && !is_pinned_host(hp.speed)) || (!hp.out_dev && !is_pinned_host(hp.out))) {
      set_err("plans take device or pinned host pointers (problem %d: pageable host memory)", (int)i);
      return EIK_EINVAL;
    }
  }
  int64_t tx, ty, tz;
  int shape = 0;
  eik_status tst = tile_shape(opts, pl.ndim, count_sources(hps), shape, tx, ty, tz);
  if (tst != EIK_OK) return tst;
  int form = 0;
  tst = update_form(opts, pl.ndim, form);
  if (tst != EIK_OK) return tst;
  if (opts && opts->schedule != 0) { set_err("plans run the asynchronous schedule (opts.schedule 0)"); return EIK_EINVAL; }
  std::vector<int> prob_speed(hps.size());
  int64_t c_total = 0;
  for (size_t i = 0; i < hps.size(); ++i) {
    int found = -1;
    for (size_t j = 0; j < pl.speeds.size(); ++j)
      if (pl.speeds[j] == hps[i].speed && pl.speed_n[j] == hps[i].n && pl.speed_h[j] == hps[i].h)
        found = (int)j;
    if (found < 0) {
      found = (int)pl.speeds.size();
      pl.speeds.push_back(hps[i].speed);
      pl.speed_host.push_back(hps[i].speed_dev ? nullptr : hps[i].speed);
      pl.speed_off.push_back(c_total);
      pl.speed_n.push_back(hps[i].n);
      pl.speed_h.push_back(hps[i].h);
      c_total += hps[i].n;
    }
    prob_speed[i] = found;
  }
  // pinned host speeds with a device mapping are read in place by init_c
  for (size_t j = 0; j < pl.speeds.size(); ++j) {
    if (!pl.speed_host[j]) continue;
    const double *m = static_cast<const double *>(mapped_ptr(pl.speed_host[j]));
    if (m) {
      pl.speeds[j] = m;
      pl.speed_host[j] = nullptr;
    }
  }
  for (auto &hp : hps) pl.total_src += (int64_t)hp.src.size();
  CK(pl.c.ensure((size_t)c_total), "plan: alloc c");
  {  // device copies of pinned host speeds and outputs
    int64_t v_cells = 0, t_cells = 0;
    for (size_t j = 0; j < pl.speeds.size(); ++j) if (pl.speed_host[j]) v_cells += pl.speed_n[j];
    for (auto &hp : hps) if (!hp.out_dev) t_cells += hp.n;
    if (v_cells) CK(pl.v_stage.ensure((size_t)v_cells), "plan: alloc speed copies");
    if (t_cells) CK(pl.t_stage.ensure((size_t)t_cells), "plan: alloc output copies");
    int64_t off = 0;
    for (size_t j = 0; j < pl.speeds.size(); ++j) {
      if (!pl.speed_host[j]) continue;
      pl.speeds[j] = pl.v_stage.p + off;
      off += pl.speed_n[j];
    }
  }
  int64_t t_off = 0;
  CK(pl.src_idx.ensure((size_t)std::max<int64_t>(pl.total_src, 1)), "plan: alloc src_idx");
  CK(pl.src_t.ensure((size_t)std::max<int64_t>(pl.total_src, 1)), "plan: alloc src_t");
  CK(pl.seeds.ensure((size_t)std::max<int64_t>(pl.total_src, 1)), "plan: alloc seeds");
  CK(pl.probs_d.ensure(hps.size()), "plan: alloc problems");
  CK(pl.ctl.ensure(1), "plan: alloc control block");
  CK(pl.count.ensure(1), "plan: alloc count");
  CK(cudaMallocHost(&pl.ctl_host, sizeof(Ctl)), "plan: pinned control block");
  std::vector<SeedItem> seeds;
  std::vector<int64_t> all_src;
  std::vector<double> all_t0;
  std::vector<eik::CopyItem> out_items;
  pl.probs.resize(hps.size());
  for (size_t i = 0; i < hps.size(); ++i) {
    HostProblem &hp = hps[i];
    Prob &P = pl.probs[i];
    std::memset(&P, 0, sizeof(P));
    P.nx = hp.dims[2];
    P.ny = hp.dims[1];
    P.nz = hp.dims[0];
    P.ntx = (P.nx + tx - 1) / tx;
    P.nty = (P.ny + ty - 1) / ty;
    P.ntz = (P.nz + tz - 1) / tz;
    P.tile_base = pl.total_tiles;
    pl.total_tiles += P.ntx * P.nty * P.ntz;
    pl.max_cells = std::max<int64_t>(pl.max_cells, P.nx * P.ny * P.nz);
    P.c = pl.c.p + pl.speed_off[prob_speed[i]];
    if (hp.out_dev) {
      P.t = hp.out;
      pl.out_host.push_back(nullptr);
    } else {
      P.t = pl.t_stage.p + t_off;
      t_off += hp.n;
      double *m = static_cast<double *>(const_cast<void *>(mapped_ptr(hp.out)));
      if (m) {
        out_items.push_back(eik::CopyItem{P.t, m, hp.n});
        pl.copy_max_n = std::max<int64_t>(pl.copy_max_n, hp.n);
      }
      pl.out_host.push_back(m ? nullptr : hp.out);
    }
    P.src_idx = pl.src_idx.p + all_src.size();
    P.src_t = pl.src_t.p + all_src.size();
    P.nsrc = (int64_t)hp.src.size();
    for (size_t k = 0; k < hp.src.size(); ++k) {
      seeds.push_back(SeedItem{(int64_t)i, hp.src[k], hp.t0[k]});
      all_src.push_back(hp.src[k]);
      all_t0.push_back(hp.t0[k]);
    }
  }
  pl.nseeds = (int64_t)seeds.size();
  if (pl.total_tiles >= (int64_t(1) << 32)) { set_err("too many tiles"); return EIK_EINVAL; }
  CK(pl.state.ensure((size_t)pl.total_tiles), "plan: alloc tile state");
  CK(pl.tile_src.ensure((size_t)pl.total_tiles), "plan: alloc tile flags");
  CK(pl.pend.ensure((size_t)pl.total_tiles * eik::kPendWords), "plan: alloc pending masks");
  uint64_t want_cap = opts && opts->capacity > 0 ? (uint64_t)opts->capacity
                                                 : (uint64_t)pl.total_tiles / 2 + 4096;
  want_cap = next_pow2(std::max<uint64_t>(want_cap, 16));
  while (want_cap * eik::kNumSlots > kMaxCapEntries && want_cap > 1024) want_cap >>= 1;
  pl.cap = want_cap;
  CK(pl.slots.ensure((size_t)(want_cap * eik::kNumSlots)), "plan: alloc frontier");
  CK(pl.seq.ensure((size_t)(want_cap * eik::kNumSlots)), "plan: alloc frontier sequence");
  if (!out_items.empty()) {
    pl.ncopies = (int)out_items.size();
    CK(pl.copies.ensure(out_items.size()), "plan: alloc copy list");
    CK(cudaMemcpyAsync(pl.copies.p, out_items.data(), out_items.size() * sizeof(eik::CopyItem),
                       cudaMemcpyHostToDevice, stream), "plan: upload copy list");
  }
  if (!all_src.empty()) {
    CK(cudaMemcpyAsync(pl.src_idx.p, all_src.data(), all_src.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice, stream), "plan: upload sources");
    CK(cudaMemcpyAsync(pl.src_t.p, all_t0.data(), all_t0.size() * sizeof(double),
                       cudaMemcpyHostToDevice, stream), "plan: upload source times");
    CK(cudaMemcpyAsync(pl.seeds.p, seeds.data(), seeds.size() * sizeof(SeedItem),
                       cudaMemcpyHostToDevice, stream), "plan: upload seeds");
  }
  CK(cudaMemcpyAsync(pl.probs_d.p, pl.probs.data(), pl.probs.size() * sizeof(Prob),
                     cudaMemcpyHostToDevice, stream), "plan: upload problems");
  CK(cudaStreamSynchronize(stream), "plan: uploads");

  SolveParams &sp = pl.sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.probs = pl.probs_d.p;
  sp.nprob = (int)pl.probs.size();
  sp.ndim = pl.ndim;
  sp.state = pl.state.p;
  sp.tile_src = pl.tile_src.p;
  sp.pend = pl.pend.p;
  sp.slots = pl.slots.p;
  sp.seq = pl.seq.p;
  sp.cap_mask = (unsigned)(pl.cap - 1);
  sp.ctl = pl.ctl.p;
  const int64_t tmo_ms = opts && opts->timeout_ms > 0 ? opts->timeout_ms : 60000;
  sp.timeout_ns = tmo_ms * 1000000ll;
  sp.counters = opts ? opts->counters : 0;
  sp.test_stall = 0;
  const AutoCfg ac = auto_config(pl.ndim, count_sources(hps), opts && opts->arith == 2);
  sp.window = (unsigned)(opts && opts->window > 0 ? opts->window : ac.window);
  sp.band = opts && opts->band > 0 ? opts->band : ac.band;
  sp.arith = opts && opts->arith == 2 ? eik::kArithInt : eik::kArithFp64;
  sp.gate_pending_only = opts && (opts->sched_flags & 1) ? 1 : 0;
  sp.tile_shape = shape;
  sp.update = form;
  sp.track_changes = opts && (opts->sched_flags & 32) ? 1 : 0;
  sp.visit_budget = sp.track_changes ? (unsigned long long)pl.total_tiles * 256ull + 4096ull : 0ull;
  sp.trace = nullptr;
  sp.trace_cap = 0;
  pl.k_delta = opts && opts->k_delta > 0 ? opts->k_delta : ac.k_delta;
  pl.delta_fixed = opts && opts->delta > 0 ? opts->delta : 0.0;
  pl.from_slowness = from_slowness(opts);
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl.device), "SM count");
  pl.grid = (int)size_grid(sp, opts, pl.ndim, shape, tx * ty * tz, pl.nseeds, pl.total_tiles, sms);
  return EIK_OK;
}

}  // namespace

extern "C" {

eik_status eik_plan_create(const eik_problem *probs, int nprob, const eik_opts *opts,
                           eik_plan **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!out || nprob <= 0 || !probs) { set_err("bad plan arguments"); return EIK_EINVAL; }
  *out = nullptr;
  std::vector<HostProblem> hps((size_t)nprob);
  for (int i = 0; i < nprob; ++i) {
    const eik_problem &q = probs[i];
    eik_status st = check_problem(q.speed, q.h, q.ndim, q.dims, q.src_idx, q.src_t, q.nsrc,
                                  q.out_t, hps[(size_t)i], nullptr);
    if (st != EIK_OK) return st;
  }
  eik_plan *pl = new (std::nothrow) eik_plan();
  if (!pl) return EIK_ENOMEM;
  eik_status st = plan_build(*pl, hps, opts, nullptr);
  if (st != EIK_OK) {
    delete pl;
    return st;
  }
  *out = pl;
  return EIK_OK;
}

eik_status eik_plan_enqueue(eik_plan *pl, void *stream) {
  if (!pl) return EIK_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(pl->ctl.p, 0, sizeof(Ctl), s), "clear control block");
  CK(cudaMemsetAsync(pl->state.p, 0, (size_t)pl->total_tiles * sizeof(unsigned long long), s),
     "clear tile states");
  CK(cudaMemsetAsync(pl->tile_src.p, 0, (size_t)pl->total_tiles, s), "clear tile flags");
  CK(cudaMemsetAsync(pl->pend.p, 0, (size_t)pl->total_tiles * eik::kPendWords * sizeof(unsigned), s),
     "clear pending masks");
  CK(cudaMemsetAsync(pl->seq.p, 0, (size_t)(pl->cap * eik::kNumSlots) * sizeof(unsigned), s),
     "clear frontier sequence");
  for (size_t j = 0; j < pl->speeds.size(); ++j) {
    if (pl->speed_host[j]) {
      CK(cudaMemcpyAsync(const_cast<double *>(pl->speeds[j]), pl->speed_host[j],
                         (size_t)pl->speed_n[j] * sizeof(double), cudaMemcpyHostToDevice, s),
         "plan: upload speed");
    }
    CK(eik::launch_init_c(pl->speeds[j], pl->speed_h[j], pl->c.p + pl->speed_off[j], pl->speed_n[j],
                          pl->ctl.p, s, pl->sp.update != 0, pl->from_slowness), "init_c launch");
  }
  CK(eik::launch_init_t_all(pl->sp.probs, (int)pl->probs.size(), pl->max_cells, s), "init_t launch");
  CK(eik::launch_seed(pl->sp, pl->seeds.p, pl->nseeds, pl->k_delta, pl->delta_fixed, s), "seed launch");
  CK(eik::launch_persistent(pl->sp, pl->grid, s), "solve launch");
  if (pl->ncopies)
    CK(eik::launch_copy_items(pl->copies.p, pl->ncopies, pl->copy_max_n, s), "plan: copy launch");
  for (size_t i = 0; i < pl->probs.size(); ++i) {
    if (!pl->out_host[i]) continue;
    const Prob &P = pl->probs[i];
    CK(cudaMemcpyAsync(pl->out_host[i], P.t, (size_t)(P.nx * P.ny * P.nz) * sizeof(double),
                       cudaMemcpyDeviceToHost, s), "plan: download t");
  }
  return EIK_OK;
}

eik_status eik_plan_status(eik_plan *pl, eik_stats *stats, void *stream) {
  if (!pl) return EIK_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(pl->ctl_host, pl->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, s), "read status");
  unsigned long long finite = 0;
  if (stats && pl->sp.counters) {
    CK(cudaMemsetAsync(pl->count.p, 0, sizeof(unsigned long long), s), "clear count");
    CK(eik::launch_count_finite_all(pl->sp.probs, (int)pl->probs.size(), pl->max_cells,
                                    pl->count.p, s), "count");
    CK(cudaMemcpyAsync(&finite, pl->count.p, sizeof(finite), cudaMemcpyDeviceToHost, s), "read count");
  }
  CK(cudaStreamSynchronize(s), "plan status");
  const Ctl &c = *pl->ctl_host;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->evals = (int64_t)c.stats[eik::kStatEvals];
    stats->decreases = (int64_t)c.stats[eik::kStatDecreases];
    stats->visits = (int64_t)c.stats[eik::kStatVisits];
    stats->pushes = (int64_t)c.stats[eik::kStatPushes];
    stats->stale_pops = (int64_t)c.stats[eik::kStatStale];
    stats->rounds = (int64_t)c.stats[eik::kStatRounds];
    stats->max_queue = (int64_t)c.stats[eik::kStatMaxQueue];
    stats->ctas = pl->grid;
    if (pl->sp.counters) stats->good = (int64_t)finite - pl->total_src;
  }
  switch (c.status) {
    case 0: return EIK_OK;
    case eik::kEinval: set_err("invalid input data"); return EIK_EINVAL;
    case eik::kEtimeout: set_err("device wait timed out"); return EIK_ETIMEOUT;
    case eik::kEcapacity: set_err("frontier capacity exhausted (create the plan with a larger capacity)");
      return EIK_ECAPACITY;
    default: return EIK_ECUDA;
  }
}

void eik_plan_destroy(eik_plan *pl) { delete pl; }

}  // extern "C"

// ---------------------------------------------------------------------------
// eik_adjoint: d(loss)/d(slowness) through the fixed points of a batch.
// ---------------------------------------------------------------------------

extern "C" eik_status eik_adjoint(const eik_problem *probs, int nprob, const double *const *dL_dt,
                                  double *const *dL_dslowness, const eik_opts *opts,
                                  eik_stats *stats, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nprob <= 0 || !probs || !dL_dslowness) { set_err("bad adjoint arguments"); return EIK_EINVAL; }
  if (nprob >= (1 << 23)) { set_err("adjoint: too many problems"); return EIK_EINVAL; }
  std::vector<HostProblem> hps((size_t)nprob);
  int64_t total = 0, total_src = 0;
  for (int i = 0; i < nprob; ++i) {
    const eik_problem &q = probs[i];
    eik_status st = check_problem(q.speed, q.h, q.ndim, q.dims, q.src_idx, q.src_t, q.nsrc,
                                  q.out_t, hps[(size_t)i], s);
    if (st != EIK_OK) return st;
    if (!hps[(size_t)i].speed_dev || !hps[(size_t)i].out_dev || !is_device_ptr(dL_dslowness[i]) ||
        (dL_dt && dL_dt[i] && !is_device_ptr(dL_dt[i]))) {
      set_err("eik_adjoint takes device pointers only (problem %d)", i);
      return EIK_EINVAL;
    }
    total += hps[(size_t)i].n;
    total_src += (int64_t)hps[(size_t)i].src.size();
  }
  {
    eik_status sd = select_device();
    if (sd != EIK_OK) return sd;
  }
  // schedule: sched_flags bits 3-4, 1 = levels, 2 = tiles, 0 = default (tiles
  // when every problem has the same ndim)
  const int adj_mode = opts ? (opts->sched_flags >> 3) & 3 : 0;
  if (adj_mode == 3) { set_err("adjoint: bad schedule flags"); return EIK_EINVAL; }
  bool same_ndim = true;
  for (int i = 1; i < nprob; ++i) same_ndim = same_ndim && hps[(size_t)i].ndim == hps[0].ndim;
  if (adj_mode == 2 && !same_ndim) {
    set_err("adjoint: the tile schedule needs one ndim per batch");
    return EIK_EINVAL;
  }
  const bool tiles = adj_mode == 2 || (adj_mode == 0 && same_ndim && kAdjTilesDefault);
  const int *tsh = hps[0].ndim == 3 ? eik::kAdjTile3 : eik::kAdjTile2;
  int64_t total_tiles = 0;
  std::vector<int64_t> ntile((size_t)nprob * 3);
  for (int i = 0; i < nprob; ++i) {
    const HostProblem &hp = hps[(size_t)i];
    const int64_t ext[3] = {hp.dims[2], hp.dims[1], hp.dims[0]};   // x, y, z
    for (int k = 0; k < 3; ++k) ntile[(size_t)i * 3 + k] = (ext[k] + tsh[k] - 1) / tsh[k];
    total_tiles += ntile[(size_t)i * 3] * ntile[(size_t)i * 3 + 1] * ntile[(size_t)i * 3 + 2];
  }
  if (tiles && total_tiles >= (int64_t(1) << 31)) { set_err("adjoint: too many tiles"); return EIK_EINVAL; }
  const uint64_t qcap = next_pow2((uint64_t)std::max<int64_t>(total_tiles, 2));
  if (!adj().ctl_host) CK(cudaMallocHost(&adj().ctl_host, sizeof(eik::AdjCtl)), "adjoint: pinned");
  CK(adj().cnt.ensure((size_t)total), "adjoint: alloc counts");
  if (tiles) {
    CK(adj().cnt_out.ensure((size_t)total), "adjoint: alloc counts");
    CK(adj().status.ensure((size_t)total), "adjoint: alloc status");
    CK(adj().tile_state.ensure((size_t)total_tiles), "adjoint: alloc tile states");
    CK(adj().ring.ensure((size_t)qcap), "adjoint: alloc tile queue");
  } else {
    CK(adj().front.ensure((size_t)total * 2), "adjoint: alloc frontiers");
  }
  CK(adj().W.ensure((size_t)total * 3), "adjoint: alloc weights");
  CK(adj().mask.ensure((size_t)total), "adjoint: alloc masks");
  if (!tiles) CK(adj().lam.ensure((size_t)total), "adjoint: alloc lambda");
  CK(adj().probs.ensure((size_t)nprob), "adjoint: alloc problems");
  CK(adj().ctl.ensure(1), "adjoint: alloc control");
  CK(adj().src.ensure((size_t)std::max<int64_t>(total_src, 1)), "adjoint: alloc sources");
  // summed outputs: problems that share a dL_dslowness array form a group (in
  // order of first appearance); each problem's gradient goes to the workspace
  // and the group's output receives +0 + g_first + ... + g_last in problem order
  const bool sum_shared = opts && (opts->sched_flags & kFlagSumShared);
  std::vector<double *> group_out;
  std::vector<std::vector<int>> group_of;
  if (sum_shared) {
    for (int i = 0; i < nprob; ++i) {
      size_t g = 0;
      while (g < group_out.size() && group_out[g] != dL_dslowness[i]) ++g;
      if (g == group_out.size()) {
        group_out.push_back(dL_dslowness[i]);
        group_of.emplace_back();
      } else if (hps[(size_t)group_of[g][0]].n != hps[(size_t)i].n) {
        set_err("adjoint: problems %d and %d share an output but differ in size", group_of[g][0], i);
        return EIK_EINVAL;
      }
      group_of[g].push_back(i);
    }
    CK(adj().gsum.ensure((size_t)total), "adjoint: alloc summed gradients");
    CK(adj().gptr.ensure((size_t)nprob), "adjoint: alloc gradient table");
  }
  std::vector<eik::AdjProb> ap((size_t)nprob);
  std::vector<int64_t> all_src;
  int64_t base = 0, tile_base = 0;
  for (int i = 0; i < nprob; ++i) {
    const HostProblem &hp = hps[(size_t)i];
    eik::AdjProb &A = ap[(size_t)i];
    A.cnt_out = tiles ? adj().cnt_out.p + base : nullptr;
    A.status = tiles ? adj().status.p + base : nullptr;
    A.ntx = ntile[(size_t)i * 3];
    A.nty = ntile[(size_t)i * 3 + 1];
    A.ntz = ntile[(size_t)i * 3 + 2];
    A.tile_base = tile_base;
    tile_base += A.ntx * A.nty * A.ntz;
    A.t = hp.out;
    A.v = hp.speed;
    A.v_is_slowness = from_slowness(opts);
    A.g = dL_dt ? dL_dt[i] : nullptr;
    A.grad = sum_shared ? adj().gsum.p + base : dL_dslowness[i];
    A.lam = tiles ? nullptr : adj().lam.p + base;
    for (int k = 0; k < 3; ++k) A.W[k] = adj().W.p + (size_t)k * (size_t)total + base;
    A.mask = adj().mask.p + base;
    A.cnt = adj().cnt.p + base;
    A.src_idx = adj().src.p + all_src.size();
    A.nsrc = (int64_t)hp.src.size();
    A.nx = hp.dims[2];
    A.ny = hp.dims[1];
    A.nz = hp.dims[0];
    A.ndim = hp.ndim;
    A.base = base;
    A.hh = hp.h * hp.h;
    all_src.insert(all_src.end(), hp.src.begin(), hp.src.end());
    base += hp.n;
  }
  if (!all_src.empty())
    CK(cudaMemcpyAsync(adj().src.p, all_src.data(), all_src.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice, s), "adjoint: upload sources");
  CK(cudaMemcpyAsync(adj().probs.p, ap.data(), ap.size() * sizeof(eik::AdjProb),
                     cudaMemcpyHostToDevice, s), "adjoint: upload problems");
  CK(cudaMemsetAsync(adj().cnt.p, 0, (size_t)total * sizeof(int), s), "adjoint: clear counts");
  if (tiles) {
    CK(cudaMemsetAsync(adj().cnt_out.p, 0, (size_t)total * sizeof(int), s), "adjoint: clear counts");
    CK(cudaMemsetAsync(adj().tile_state.p, 0, (size_t)total_tiles * sizeof(unsigned), s),
       "adjoint: clear tile states");
  }
  CK(cudaMemsetAsync(adj().ctl.p, 0, sizeof(eik::AdjCtl), s), "adjoint: clear control");
  const int64_t tmo_ms = opts && opts->timeout_ms > 0 ? opts->timeout_ms : 60000;
  if (!adj().ev0) {
    CK(cudaEventCreate(&adj().ev0), "adjoint: event");
    CK(cudaEventCreate(&adj().ev1), "adjoint: event");
  }
  CK(cudaEventRecord(adj().ev0, s), "adjoint: event record");
  if (tiles)
    CK(eik::launch_adjoint_tiles(adj().probs.p, nprob, total, total_tiles, hps[0].ndim, adj().ctl.p,
                                 adj().tile_state.p, adj().ring.p, qcap,
                                 opts ? opts->ctas_per_sm : 0, tmo_ms * 1000000ll,
                                 opts && opts->counters, s),
       "adjoint launch");
  else
    CK(eik::launch_adjoint(adj().probs.p, nprob, total, adj().ctl.p, adj().front.p,
                           tmo_ms * 1000000ll, s), "adjoint launch");
  if (sum_shared) {
    std::vector<const double *> table;
    std::vector<size_t> first;
    for (size_t g = 0; g < group_out.size(); ++g) {
      first.push_back(table.size());
      for (int i : group_of[g]) table.push_back(ap[(size_t)i].grad);
    }
    CK(cudaMemcpyAsync(adj().gptr.p, table.data(), table.size() * sizeof(const double *),
                       cudaMemcpyHostToDevice, s), "adjoint: upload gradient table");
    for (size_t g = 0; g < group_out.size(); ++g) {
      CK(eik::launch_sum_ordered(adj().gptr.p + first[g], (int)group_of[g].size(), group_out[g],
                                 hps[(size_t)group_of[g][0]].n, s), "adjoint: ordered sum");
    }
  }
  CK(cudaEventRecord(adj().ev1, s), "adjoint: event record");
  CK(cudaMemcpyAsync(adj().ctl_host, adj().ctl.p, sizeof(eik::AdjCtl), cudaMemcpyDeviceToHost, s),
     "adjoint: read status");
  CK(cudaStreamSynchronize(s), "adjoint");
  const eik::AdjCtl &c = *adj().ctl_host;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->good = (int64_t)c.done;
    stats->evals = (int64_t)c.reached;
    stats->visits = (int64_t)c.visits;
    stats->rounds = tiles ? (int64_t)c.rounds : (int64_t)c.levels;
    stats->visit_ns = (int64_t)c.visit_ns;
    stats->idle_ns = (int64_t)c.idle_ns;
    stats->ctas = (int64_t)c.ctas;
    for (int i = 0; i < 4; ++i) stats->detail[i] = (int64_t)c.cycles[i];
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, adj().ev0, adj().ev1) == cudaSuccess) stats->solve_ms = ms;
  }
  if (c.status == eik::kEtimeout) { set_err("adjoint: device wait timed out"); return EIK_ETIMEOUT; }
  if (c.status != 0) return EIK_ECUDA;
  if (c.done != c.reached) { set_err("adjoint: %llu of %llu cells processed",
                                     (unsigned long long)c.done, (unsigned long long)c.reached);
                             return EIK_ECUDA; }
  return EIK_OK;
}
