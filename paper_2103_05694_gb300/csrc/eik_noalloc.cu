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

constexpr int kMaxDevices = 64;
unsigned char *g_base[kMaxDevices] = {};           // device address of g_scratch, per device

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

}  // namespace na
}  // namespace eik

extern "C" eik_status eik_solve_noalloc(const double *speed, double h, int ndim,
                                        const int64_t *dims, const int64_t *src_idx,
                                        const double *src_t, int64_t nsrc, double *out_t,
                                        const eik_opts *opts, eik_stats *stats, void *stream) {
  using namespace eik;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((ndim != 2 && ndim != 3) || !dims || !(h > 0.0) || !(h < 1e308)) return EIK_EINVAL;
  int64_t n = 1;
  for (int k = 0; k < ndim; ++k) {
    if (dims[k] < 1 || dims[k] > na::kMaxCells) return EIK_EINVAL;
    n *= dims[k];
    if (n > na::kMaxCells) return EIK_EINVAL;                 // beyond the scratch limit
  }
  if (nsrc < 0 || nsrc > na::kMaxSources) return EIK_EINVAL;  // beyond the scratch limit
  if (opts && (opts->update != 0 || opts->tile != 0 || opts->schedule != 0))
    return EIK_EINVAL;   // default form, tile and schedule only
  if (!na::device_ptr(speed) || !na::device_ptr(out_t)) return EIK_EINVAL;
  if (nsrc > 0 && !na::device_ptr(src_idx)) return EIK_EINVAL;
  if (src_t && !na::device_ptr(src_t)) return EIK_EINVAL;
  const int64_t nx = dims[ndim - 1], ny = dims[ndim - 2], nz = ndim == 3 ? dims[0] : 1;
  const int64_t tx = ndim == 3 ? kTX3 : kTX2, ty = ndim == 3 ? kTY3 : kTY2, tz = ndim == 3 ? kTZ3 : 1;
  const int64_t ntx = (nx + tx - 1) / tx, nty = (ny + ty - 1) / ty, ntz = (nz + tz - 1) / tz;
  const int64_t ntiles = ntx * nty * ntz;
  if (ntiles > na::kMaxTiles) return EIK_EINVAL;              // beyond the scratch limit

  // once per device, with that device current: the device address of the array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= na::kMaxDevices) return EIK_ECUDA;
  if (!na::g_base[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, na::g_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return EIK_ECUDA;
    }
    na::g_base[dev] = static_cast<unsigned char *>(ptr);
  }
  unsigned char *base = na::g_base[dev];
  Ctl *ctl = reinterpret_cast<Ctl *>(base + na::kOffCtl);
  Prob *prob_dev = reinterpret_cast<Prob *>(base + na::kOffProb);

  // clear what must start at zero (the array keeps the previous call's contents)
  if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess ||
      cudaMemsetAsync(base + na::kOffState, 0, sizeof(unsigned long long) * ntiles, s) != cudaSuccess ||
      cudaMemsetAsync(base + na::kOffTileSrc, 0, ntiles, s) != cudaSuccess ||
      cudaMemsetAsync(base + na::kOffPend, 0, sizeof(unsigned) * kPendWords * ntiles, s) != cudaSuccess ||
      cudaMemsetAsync(base + na::kOffSeq, 0, sizeof(unsigned) * kNumSlots * na::kCap, s) !=
          cudaSuccess) {
    return EIK_ECUDA;
  }
  Prob prob;
  std::memset(&prob, 0, sizeof(prob));
  prob.t = out_t;
  prob.c = reinterpret_cast<const double *>(base + na::kOffC);
  prob.nx = nx;
  prob.ny = ny;
  prob.nz = nz;
  prob.ntx = ntx;
  prob.nty = nty;
  prob.ntz = ntz;
  prob.tile_base = 0;
  prob.src_idx = reinterpret_cast<const int64_t *>(base + na::kOffSrcIdx);
  prob.src_t = reinterpret_cast<const double *>(base + na::kOffSrcT);
  prob.nsrc = 0;

  if (launch_init_c(speed, h, reinterpret_cast<double *>(base + na::kOffC), n, ctl, s) != cudaSuccess ||
      launch_init_t(out_t, n, s) != cudaSuccess) {
    return EIK_ECUDA;
  }
  na::sources_kernel<<<1, na::kSortThreads, 0, s>>>(src_idx, src_t, nsrc, prob, n, base);
  note_launches(1);
  if (cudaGetLastError() != cudaSuccess) return EIK_ECUDA;

  SolveParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.probs = prob_dev;
  sp.nprob = 1;
  sp.ndim = ndim;
  sp.state = reinterpret_cast<unsigned long long *>(base + na::kOffState);
  sp.tile_src = base + na::kOffTileSrc;
  sp.pend = reinterpret_cast<unsigned *>(base + na::kOffPend);
  sp.slots = reinterpret_cast<unsigned long long *>(base + na::kOffSlots);
  sp.seq = reinterpret_cast<unsigned *>(base + na::kOffSeq);
  sp.cap_mask = static_cast<unsigned>(na::kCap - 1);
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
  if (launch_seed(sp, reinterpret_cast<const SeedItem *>(base + na::kOffSeeds), nsrc, k_delta,
                  delta_fixed, s) != cudaSuccess) {
    return EIK_ECUDA;
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
  if (launch_persistent(sp, static_cast<int>(grid), s) != cudaSuccess) return EIK_ECUDA;

  unsigned long long *count = reinterpret_cast<unsigned long long *>(base + na::kOffCount);
  if (stats) {
    if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess ||
        launch_count_finite(&prob, 1, count, s) != cudaSuccess) {
      return EIK_ECUDA;
    }
  }
  // read back the status and counters into host stack memory
  unsigned status = 0;
  unsigned long long st[kNumStats];
  unsigned long long finite = 0;
  if (cudaMemcpyAsync(&status, &ctl->status, sizeof(status), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(st, ctl->stats, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      (stats && cudaMemcpyAsync(&finite, count, sizeof(finite), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    return EIK_ECUDA;
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
  if (status == kEinval) return EIK_EINVAL;
  if (status == kEtimeout) return EIK_ETIMEOUT;
  if (status == kEcapacity) return EIK_ECAPACITY;
  if (status != 0) return EIK_ECUDA;
  if (stats) {
    // good = reached non-source cells; the number of unique sources is in the problem record
    Prob pr;
    if (cudaMemcpyAsync(&pr, prob_dev, sizeof(pr), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      return EIK_ECUDA;
    }
    stats->good = static_cast<int64_t>(finite) - pr.nsrc;
  }
  return EIK_OK;
}
