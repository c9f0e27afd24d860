// eik_solve_noalloc: the single-grid solve without any memory allocation.
//
// Some callers cannot allocate device memory: code whose device memory is
// owned by an arena or pool allocator that forbids outside cudaMalloc calls,
// and latency-sensitive loops where cudaMalloc / cudaFree would synchronise
// the whole device and stall other streams.  eik_solve grows a workspace on
// first use; this entry point instead runs the same kernels on a fixed
// scratch area that is a file-scope __device__ array, so it calls no
// cudaMalloc, cudaFree, cudaMallocHost or other allocating routine.
//
// The array (about 21 MB) exists on every GPU that loads this library, for
// as long as the library stays loaded.  Every call shares it: the call clears
// what must start at zero itself, and calls whose work overlaps on the GPU
// (different streams, or different host threads without ordering) race on it.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/eik.h"
#include "eik_internal.h"

namespace eik {
namespace na {

// Limits of the fixed scratch area.
constexpr int64_t kMaxCells = int64_t(1) << 20;
constexpr int64_t kMaxTiles = int64_t(1) << 15;
constexpr int64_t kMaxSources = 2048;
constexpr uint64_t kCap = 8192;                    // ring entries per bucket slot

constexpr size_t up256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCtl = 0;
constexpr size_t kOffProb = up256(kOffCtl + sizeof(Ctl));
constexpr size_t kOffCount = up256(kOffProb + sizeof(Prob));
constexpr size_t kOffC = up256(kOffCount + sizeof(unsigned long long));
constexpr size_t kOffState = up256(kOffC + sizeof(double) * kMaxCells);
constexpr size_t kOffTileSrc = up256(kOffState + sizeof(unsigned long long) * kMaxTiles);
constexpr size_t kOffPend = up256(kOffTileSrc + kMaxTiles);
constexpr size_t kOffSlots = up256(kOffPend + sizeof(unsigned) * kPendWords * kMaxTiles);
constexpr size_t kOffSeq = up256(kOffSlots + sizeof(unsigned long long) * kNumSlots * kCap);
constexpr size_t kOffSrcIdx = up256(kOffSeq + sizeof(unsigned) * kNumSlots * kCap);
constexpr size_t kOffSrcT = up256(kOffSrcIdx + sizeof(int64_t) * kMaxSources);
constexpr size_t kOffSeeds = up256(kOffSrcT + sizeof(double) * kMaxSources);
constexpr size_t kBytes = up256(kOffSeeds + sizeof(SeedItem) * kMaxSources);

__device__ __align__(256) unsigned char g_scratch[kBytes];

// Validate, sort and de-duplicate the sources (smallest time per cell), write
// the problem record and one seed item per input source (duplicates repeat
// the first unique source, which the seed kernel writes idempotently).
constexpr int kSortThreads = 1024;

__global__ void __launch_bounds__(kSortThreads)
sources_kernel(const int64_t *__restrict__ src_idx, const double *__restrict__ src_t, int64_t nsrc,
               Prob prob, int64_t ncells, unsigned char *base) {
  __shared__ unsigned long long key_idx[kMaxSources];
  __shared__ unsigned long long key_t[kMaxSources];
  __shared__ int s_bad, s_nuniq;
  Ctl *ctl = reinterpret_cast<Ctl *>(base + kOffCtl);
  const int tid = threadIdx.x;
  int n = static_cast<int>(nsrc);
  int np = 1;
  while (np < n) np <<= 1;
  if (tid == 0) { s_bad = 0; s_nuniq = 0; }
  __syncthreads();
  for (int i = tid; i < np; i += kSortThreads) {
    if (i < n) {
      const int64_t ix = src_idx[i];
      double t0 = src_t ? src_t[i] : 0.0;
      const unsigned long long tb = static_cast<unsigned long long>(__double_as_longlong(t0));
      const bool ok = ix >= 0 && ix < ncells && t0 >= 0.0 && tb < 0x7ff0000000000000ull;
      if (!ok) atomicExch(&s_bad, 1);
      if (t0 == 0.0) t0 = 0.0;     // -0 -> +0
      key_idx[i] = static_cast<unsigned long long>(ix);
      key_t[i] = static_cast<unsigned long long>(__double_as_longlong(t0));
    } else {
      key_idx[i] = ~0ull;
      key_t[i] = ~0ull;
    }
  }
  __syncthreads();
  int64_t *out_idx = reinterpret_cast<int64_t *>(base + kOffSrcIdx);
  double *out_t = reinterpret_cast<double *>(base + kOffSrcT);
  SeedItem *seeds = reinterpret_cast<SeedItem *>(base + kOffSeeds);
  if (s_bad) {
    // report EINVAL, and leave a problem record and seeds that stay in range
    // (the following launches run and return at once on the error status)
    for (int i = tid; i < n; i += kSortThreads) seeds[i] = SeedItem{0, 0, 0.0};
    if (tid == 0) {
      if (atomicCAS(&ctl->status, 0u, kEinval) == 0u) ctl->error_info[0] = ~0ull;
      prob.src_idx = out_idx;
      prob.src_t = out_t;
      prob.nsrc = 0;
      *reinterpret_cast<Prob *>(base + kOffProb) = prob;
    }
    return;
  }
  // bitonic sort of (index, time) pairs, ascending
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < np; i += kSortThreads) {
        const int l = i ^ j;
        if (l > i) {
          const bool asc = (i & k) == 0;
          const bool gt = key_idx[i] > key_idx[l] ||
                          (key_idx[i] == key_idx[l] && key_t[i] > key_t[l]);
          if (gt == asc) {
            const unsigned long long a = key_idx[i], b = key_t[i];
            key_idx[i] = key_idx[l];
            key_t[i] = key_t[l];
            key_idx[l] = a;
            key_t[l] = b;
          }
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) {   // compaction (n <= 2048, once per call)
    int u = 0;
    for (int i = 0; i < n; ++i) {
      if (i > 0 && key_idx[i] == key_idx[i - 1]) continue;
      out_idx[u] = static_cast<int64_t>(key_idx[i]);
      out_t[u] = __longlong_as_double(static_cast<long long>(key_t[i]));
      ++u;
    }
    s_nuniq = u;
    prob.src_idx = out_idx;
    prob.src_t = out_t;
    prob.nsrc = u;
    *reinterpret_cast<Prob *>(base + kOffProb) = prob;
  }
  __syncthreads();
  const int u = s_nuniq;
  for (int i = tid; i < n; i += kSortThreads) {
    const int j = i < u ? i : 0;
    seeds[i] = SeedItem{0, out_idx[j], out_t[j]};
  }
}

bool device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Every return path of eik_solve_noalloc leaves its reason for eik_last_error.
eik_status fail(eik_status st, const char *msg) {
  set_last_error("eik_solve_noalloc: %s", msg);
  return st;
}
eik_status cuda_fail(cudaError_t e, const char *what) {
  cudaGetLastError();
  set_last_error("eik_solve_noalloc: %s: %s", what, cudaGetErrorString(e));
  return EIK_ECUDA;
}

eik_status solve(const double *speed, double h, int ndim, const int64_t *dims,
                 const int64_t *src_idx, const double *src_t, int64_t nsrc, double *out_t,
                 const eik_opts *opts, eik_stats *stats, cudaStream_t s) {
  if (ndim != 2 && ndim != 3) return fail(EIK_EINVAL, "ndim must be 2 or 3");
  if (!dims) return fail(EIK_EINVAL, "dims is NULL");
  if (!(h > 0.0) || !(h < 1e308)) return fail(EIK_EINVAL, "h must be finite and > 0");
  int64_t n = 1;
  for (int k = 0; k < ndim; ++k) {
    if (dims[k] < 1) return fail(EIK_EINVAL, "every extent must be >= 1");
    if (dims[k] > kMaxCells) return fail(EIK_EINVAL, "more than 2^20 cells (the scratch limit)");
    n *= dims[k];
    if (n > kMaxCells) return fail(EIK_EINVAL, "more than 2^20 cells (the scratch limit)");
  }
  if (nsrc < 0) return fail(EIK_EINVAL, "nsrc must be >= 0");
  if (nsrc > kMaxSources) return fail(EIK_EINVAL, "more than 2048 sources (the scratch limit)");
  if (opts && (opts->update != 0 || opts->tile != 0 || opts->schedule != 0))
    return fail(EIK_EINVAL, "opts.update, opts.tile and opts.schedule must be 0");
  if (!device_ptr(speed) || !device_ptr(out_t))
    return fail(EIK_EINVAL, "speed and out_t must be device pointers");
  if (nsrc > 0 && !device_ptr(src_idx)) return fail(EIK_EINVAL, "src_idx must be a device pointer");
  if (src_t && !device_ptr(src_t)) return fail(EIK_EINVAL, "src_t must be a device pointer");
  const int64_t nx = dims[ndim - 1], ny = dims[ndim - 2], nz = ndim == 3 ? dims[0] : 1;
  const int64_t tx = ndim == 3 ? kTX3 : kTX2, ty = ndim == 3 ? kTY3 : kTY2, tz = ndim == 3 ? kTZ3 : 1;
  const int64_t ntx = (nx + tx - 1) / tx, nty = (ny + ty - 1) / ty, ntz = (nz + tz - 1) / tz;
  const int64_t ntiles = ntx * nty * ntz;
  if (ntiles > kMaxTiles) return fail(EIK_EINVAL, "more than 2^15 tiles (the scratch limit)");

  // The device address of the array on the current device.  In host code the
  // name g_scratch is a host-side stand-in, not a device address; the lookup
  // allocates nothing and is repeated on every call (no per-device cache).
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  void *ptr = nullptr;
  e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
  if (!ptr) return fail(EIK_ECUDA, "cudaGetSymbolAddress gave a null address");
  unsigned char *base = static_cast<unsigned char *>(ptr);
  Ctl *ctl = reinterpret_cast<Ctl *>(base + kOffCtl);
  Prob *prob_dev = reinterpret_cast<Prob *>(base + kOffProb);

  // clear what must start at zero (the array keeps the previous call's contents)
  if ((e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(base + kOffState, 0, sizeof(unsigned long long) * ntiles, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(base + kOffTileSrc, 0, ntiles, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(base + kOffPend, 0, sizeof(unsigned) * kPendWords * ntiles, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(base + kOffSeq, 0, sizeof(unsigned) * kNumSlots * kCap, s)) != cudaSuccess) {
    return cuda_fail(e, "clearing the scratch array");
  }
  Prob prob;
  std::memset(&prob, 0, sizeof(prob));
  prob.t = out_t;
  prob.c = reinterpret_cast<const double *>(base + kOffC);
  prob.nx = nx;
  prob.ny = ny;
  prob.nz = nz;
  prob.ntx = ntx;
  prob.nty = nty;
  prob.ntz = ntz;
  prob.tile_base = 0;
  prob.src_idx = reinterpret_cast<const int64_t *>(base + kOffSrcIdx);
  prob.src_t = reinterpret_cast<const double *>(base + kOffSrcT);
  prob.nsrc = 0;

  const int from_slowness = opts && (opts->sched_flags & (1 << 6)) ? 1 : 0;
  if ((e = launch_init_c(speed, h, reinterpret_cast<double *>(base + kOffC), n, ctl, s, 0,
                         from_slowness)) != cudaSuccess ||
      (e = launch_init_t(out_t, n, s)) != cudaSuccess) {
    return cuda_fail(e, "set-up launch");
  }
  sources_kernel<<<1, kSortThreads, 0, s>>>(src_idx, src_t, nsrc, prob, n, base);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sources launch");

  SolveParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.probs = prob_dev;
  sp.nprob = 1;
  sp.ndim = ndim;
  sp.state = reinterpret_cast<unsigned long long *>(base + kOffState);
  sp.tile_src = base + kOffTileSrc;
  sp.pend = reinterpret_cast<unsigned *>(base + kOffPend);
  sp.slots = reinterpret_cast<unsigned long long *>(base + kOffSlots);
  sp.seq = reinterpret_cast<unsigned *>(base + kOffSeq);
  sp.cap_mask = static_cast<unsigned>(kCap - 1);
  sp.ctl = ctl;
  sp.timeout_ns = (opts && opts->timeout_ms > 0 ? opts->timeout_ms : 60000) * 1000000ll;
  sp.counters = opts ? opts->counters : 0;
  sp.test_stall = 0;
  sp.window = static_cast<unsigned>(opts && opts->window > 0 ? opts->window : 16);
  sp.band = opts && opts->band > 0 ? opts->band : (ndim == 3 ? 8.0 : 16.0);
  sp.arith = opts && opts->arith == 2 ? kArithInt : kArithFp64;
  sp.gate_pending_only = opts && (opts->sched_flags & 1) ? 1 : 0;
  sp.trace = nullptr;
  sp.trace_cap = 0;
  const double k_delta = opts && opts->k_delta > 0 ? opts->k_delta : (ndim == 3 ? 2.0 : 16.0);
  const double delta_fixed = opts && opts->delta > 0 ? opts->delta : 0.0;
  if ((e = launch_seed(sp, reinterpret_cast<const SeedItem *>(base + kOffSeeds), nsrc, k_delta,
                       delta_fixed, s)) != cudaSuccess) {
    return cuda_fail(e, "seed launch");
  }
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = persistent_blocks_per_sm(ndim, sp.arith, 0);
  const int want = opts && opts->ctas_per_sm > 0 ? opts->ctas_per_sm : (ndim == 3 ? 2 : 1);
  if (want < per_sm) per_sm = want;
  int64_t grid = static_cast<int64_t>(sms) * per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  // lane-group d-bar when the solve has few tiles per CTA (as the main path)
  sp.lane_group_cells = ntiles < 8 * grid ? static_cast<int>(tx * ty * tz / 4) : 0;
  if ((e = launch_persistent(sp, static_cast<int>(grid), s)) != cudaSuccess)
    return cuda_fail(e, "solve launch");

  unsigned long long *count = reinterpret_cast<unsigned long long *>(base + kOffCount);
  if (stats) {
    if ((e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s)) != cudaSuccess ||
        (e = launch_count_finite(&prob, 1, count, s)) != cudaSuccess) {
      return cuda_fail(e, "count launch");
    }
  }
  // read back the status and counters into host stack memory
  unsigned status = 0;
  unsigned long long st[kNumStats];
  unsigned long long finite = 0;
  unsigned long long info = 0;
  if ((e = cudaMemcpyAsync(&status, &ctl->status, sizeof(status), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&info, &ctl->error_info[0], sizeof(info), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(st, ctl->stats, sizeof(st), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (stats && (e = cudaMemcpyAsync(&finite, count, sizeof(finite), cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    return cuda_fail(e, "status read-back");
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->evals = static_cast<int64_t>(st[kStatEvals]);
    stats->decreases = static_cast<int64_t>(st[kStatDecreases]);
    stats->visits = static_cast<int64_t>(st[kStatVisits]);
    stats->pushes = static_cast<int64_t>(st[kStatPushes]);
    stats->stale_pops = static_cast<int64_t>(st[kStatStale]);
    stats->rounds = static_cast<int64_t>(st[kStatRounds]);
    stats->ctas = grid;
  }
  if (status == kEinval) {
    if (info == ~0ull)
      return fail(EIK_EINVAL, "invalid sources (index out of range, or time negative, NaN or inf)");
    set_last_error("eik_solve_noalloc: invalid input data (cell %llu: speed must be finite and > 0, "
                   "h/v finite and > 0)", info);
    return EIK_EINVAL;
  }
  if (status == kEtimeout) return fail(EIK_ETIMEOUT, "a device wait reached its limit");
  if (status == kEcapacity)
    return fail(EIK_ECAPACITY, "frontier overflow (no capacity retry without allocation)");
  if (status != 0) return fail(EIK_ECUDA, "unexpected device status");
  if (stats) {
    // good = reached non-source cells; the number of unique sources is in the problem record
    Prob pr;
    if ((e = cudaMemcpyAsync(&pr, prob_dev, sizeof(pr), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      return cuda_fail(e, "problem record read-back");
    }
    stats->good = static_cast<int64_t>(finite) - pr.nsrc;
  }
  return EIK_OK;
}

}  // namespace na
}  // namespace eik

extern "C" eik_status eik_solve_noalloc(const double *speed, double h, int ndim,
                                        const int64_t *dims, const int64_t *src_idx,
                                        const double *src_t, int64_t nsrc, double *out_t,
                                        const eik_opts *opts, eik_stats *stats, void *stream) {
  std::lock_guard<std::mutex> lk(eik::api_mutex());
  return eik::na::solve(speed, h, ndim, dims, src_idx, src_t, nsrc, out_t, opts, stats,
                        static_cast<cudaStream_t>(stream));
}
