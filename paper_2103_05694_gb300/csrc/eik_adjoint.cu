// Adjoint of the exact fixed point: d(loss)/d(slowness) for traveltime
// tomography (not in the paper; implicit differentiation of the
// real-arithmetic local equations at the computed field).
//
// For a reached non-source cell n with axis minima a_k and active axes
// A(n) = {k : a_k < t_n}, the local equation sum_{k in A} (t_n - a_k)^2 =
// h^2 s_n^2 (s = 1/v) gives dt_n = [sum_A (t_n - a_k) da_k + h^2 s_n ds_n] / S_n
// with S_n = sum_A (t_n - a_k).  For g = dL/dt:
//   lambda_n = g_n + sum_{downwind m, order x-, x+, y-, y+, z-, z+} lambda_m w(m, n),
//   w(m, n)  = (t_m - t_n) / S_m, halved when m's two neighbours on that axis tie,
//   dL/ds_n  = lambda_n (h^2 s_n) / S_n   (0 for sources and unreached cells).
// Every operation is an explicit round-to-nearest intrinsic and the sum order
// is fixed, so the result equals the CPU oracle's bit for bit.
//
// Schedule: Kahn order, level by level.  cnt[n] = number of downwind cells
// that use n; cells with cnt 0 form the first frontier.  One cooperative
// persistent launch processes a frontier (pull lambda from the final downwind
// lambdas, decrement the counts of the cell's upwind cells, append those that
// reach zero to the next frontier), then meets at a grid barrier whose wait is
// bounded by %globaltimer, and moves to the next frontier.
#include <cstdint>
#include <cuda_runtime.h>

#include "eik_internal.h"

namespace eik {
namespace {

constexpr unsigned long long kInfB = 0x7ff0000000000000ull;
constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ unsigned long long ubits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}
__device__ __forceinline__ double ld_rlx_d(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_rlx_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rlx_d(double *p, double v) {
  asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ long long gtime() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int find_adj_prob(const AdjProb *probs, int nprob, int64_t q) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].base <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool adj_is_source(const AdjProb &P, int64_t n) {
  int64_t lo = 0, hi = P.nsrc - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int64_t v = P.src_idx[mid];
    if (v == n) return true;
    if (v < n) lo = mid + 1; else hi = mid - 1;
  }
  return false;
}

struct Nbrs {
  int64_t idx[6];      // neighbour index per (axis, side), -1 off-grid
  double t[6];
};

__device__ __forceinline__ void neighbours(const AdjProb &P, int64_t n, Nbrs &nb) {
  const int64_t x = n % P.nx, yz = n / P.nx, y = yz % P.ny, z = yz / P.ny;
  const int64_t c3[3] = {x, y, z};
  const int64_t n3[3] = {P.nx, P.ny, P.nz};
  const int64_t st[3] = {1, P.nx, P.nx * P.ny};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const bool lo_in = k < P.ndim && c3[k] > 0;
    const bool hi_in = k < P.ndim && c3[k] + 1 < n3[k];
    nb.idx[2 * k] = lo_in ? n - st[k] : -1;
    nb.idx[2 * k + 1] = hi_in ? n + st[k] : -1;
    nb.t[2 * k] = lo_in ? P.t[n - st[k]] : __longlong_as_double(kInfB);
    nb.t[2 * k + 1] = hi_in ? P.t[n + st[k]] : __longlong_as_double(kInfB);
  }
}

// S_n over the active axes (0 if none), terms summed in axis order.
__device__ __forceinline__ double upwind_sum(const Nbrs &nb, double tn, int ndim) {
  double S = 0.0;
  for (int k = 0; k < ndim; ++k) {
    const double ak = ubits(nb.t[2 * k]) < ubits(nb.t[2 * k + 1]) ? nb.t[2 * k] : nb.t[2 * k + 1];
    if (ak < tn) S = __dadd_rn(S, __dsub_rn(tn, ak));
  }
  return S;
}

// counts, S, zeroed outputs, number of reached cells
__global__ void adj_setup_kernel(const AdjProb *probs, int nprob, int64_t total, AdjCtl *ctl) {
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const AdjProb &P = probs[find_adj_prob(probs, nprob, q)];
    const int64_t n = q - P.base;
    P.grad[n] = 0.0;
    P.lam[n] = 0.0;
    const double tn = P.t[n];
    if (!(ubits(tn) < kInfB)) { P.S[n] = 0.0; continue; }
    atomicAdd(&ctl->reached, 1ull);
    if (P.nsrc > 0 && adj_is_source(P, n)) { P.S[n] = 0.0; continue; }
    Nbrs nb;
    neighbours(P, n, nb);
    P.S[n] = upwind_sum(nb, tn, P.ndim);
    for (int k = 0; k < P.ndim; ++k) {
      const unsigned long long lo = ubits(nb.t[2 * k]), hi = ubits(nb.t[2 * k + 1]);
      const unsigned long long ak = lo < hi ? lo : hi;
      if (!(ak < ubits(tn))) continue;                 // axis not active
      if (lo == ak) atomicAdd(P.cnt + nb.idx[2 * k], 1);
      if (hi == ak) atomicAdd(P.cnt + nb.idx[2 * k + 1], 1);
    }
  }
}

__device__ __forceinline__ unsigned ld_acq_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Warp-aggregated append of the lanes' ready entries to a frontier.  All 32
// lanes of the warp call it.
__device__ __forceinline__ void append_ready(unsigned long long *count, unsigned long long *front,
                                             bool ready, unsigned long long entry) {
  const unsigned bal = __ballot_sync(kFullMask, ready);
  if (!bal) return;
  const unsigned lane = threadIdx.x & 31u;
  const int leader = __ffs(bal) - 1;
  unsigned long long base = 0;
  if (lane == static_cast<unsigned>(leader)) base = atomicAdd(count, static_cast<unsigned long long>(__popc(bal)));
  base = __shfl_sync(kFullMask, base, leader);
  if (ready) front[base + __popc(bal & ((1u << lane) - 1u))] = entry;
}

__global__ void adj_seed_kernel(const AdjProb *probs, int nprob, int64_t total, AdjCtl *ctl,
                                unsigned long long *front) {
  const int64_t span = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t base = blockIdx.x * static_cast<int64_t>(blockDim.x); base < total; base += span) {
    const int64_t q = base + threadIdx.x;
    bool ready = false;
    if (q < total) {
      const AdjProb &P = probs[find_adj_prob(probs, nprob, q)];
      const int64_t n = q - P.base;
      ready = ubits(P.t[n]) < kInfB && P.cnt[n] == 0;
    }
    append_ready(&ctl->nfront[0], front, ready, static_cast<unsigned long long>(q));
  }
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident).  The wait
// is bounded: on expiry the status becomes EIK_ETIMEOUT and every block leaves.
// Returns false when the launch must stop.
__device__ bool grid_barrier(AdjCtl *ctl, long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acq_u32(&ctl->bar_gen);
    __threadfence();
    if (atomicAdd(&ctl->bar_count, 1u) + 1u == gridDim.x) {
      ctl->bar_count = 0u;
      __threadfence();
      st_rel_u32(&ctl->bar_gen, gen + 1u);
    } else {
      const long long t0 = gtime();
      while (ld_acq_u32(&ctl->bar_gen) == gen) {
        if (ld_acq_u32(&ctl->status) != 0u) break;
        if (gtime() - t0 > timeout_ns) { atomicCAS(&ctl->status, 0u, kEtimeout); break; }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ld_acq_u32(&ctl->status) == 0u;
}

// lambda and dL/ds of one ready cell, then release its upwind cells; the ones
// that become ready are appended to the next frontier.  All 32 lanes call it.
__device__ void adj_process(const AdjProb &P, int64_t n, AdjCtl *ctl, unsigned long long *count,
                            unsigned long long *front, bool live) {
  unsigned long long ready_entry[6];
  bool ready[6] = {false, false, false, false, false, false};
  if (live) {
    const double tn = P.t[n];
    Nbrs nb;
    neighbours(P, n, nb);
    double lam = P.g ? P.g[n] : 0.0;
    // pull: downwind neighbours m for which n holds m's axis minimum (active);
    // S_m = 0 marks a source or an unreached cell, whose time does not depend on n
    for (int j = 0; j < 2 * P.ndim; ++j) {
      const int64_t m = nb.idx[j];
      if (m < 0) continue;
      const double tm = nb.t[j];
      if (!(ubits(tm) > ubits(tn)) || !(ubits(tm) < kInfB)) continue;
      const double Sm = P.S[m];
      if (!(Sm > 0.0)) continue;
      const int k = j >> 1;
      // m's other neighbour on axis k, beyond m, away from n
      const int64_t other = (j & 1) ? m + (m - n) : m - (n - m);
      const int64_t mx = m % P.nx, myz = m / P.nx, my = myz % P.ny, mz = myz / P.ny;
      const int64_t mc[3] = {mx, my, mz};
      const int64_t mn[3] = {P.nx, P.ny, P.nz};
      const bool other_in = (j & 1) ? (mc[k] + 1 < mn[k]) : (mc[k] > 0);
      const double to = other_in ? P.t[other] : __longlong_as_double(kInfB);
      if (ubits(to) < ubits(tn)) continue;             // the other neighbour holds the minimum
      double w = __ddiv_rn(__dsub_rn(tm, tn), Sm);
      if (ubits(to) == ubits(tn)) w = __dmul_rn(w, 0.5);
      const double lm = ld_rlx_d(P.lam + m);           // written by another SM
      lam = __dadd_rn(lam, __dmul_rn(lm, w));
    }
    st_rlx_d(P.lam + n, lam);
    const double Sn = P.S[n];
    if (Sn > 0.0) {                                    // not a source
      const double s = __ddiv_rn(1.0, P.v[n]);
      P.grad[n] = __dmul_rn(lam, __ddiv_rn(__dmul_rn(P.hh, s), Sn));
      for (int k = 0; k < P.ndim; ++k) {
        const unsigned long long lo = ubits(nb.t[2 * k]), hi = ubits(nb.t[2 * k + 1]);
        const unsigned long long ak = lo < hi ? lo : hi;
        if (!(ak < ubits(tn))) continue;
        for (int side = 0; side < 2; ++side) {
          if ((side ? hi : lo) != ak) continue;
          const int64_t u = nb.idx[2 * k + side];
          if (atomicSub(P.cnt + u, 1) == 1) {
            ready[2 * k + side] = true;
            ready_entry[2 * k + side] = static_cast<unsigned long long>(P.base + u);
          }
        }
      }
    }
  }
  const unsigned nlive = __popc(__ballot_sync(kFullMask, live));
  if ((threadIdx.x & 31u) == 0 && nlive) atomicAdd(&ctl->done, static_cast<unsigned long long>(nlive));
  for (int j = 0; j < 6; ++j) append_ready(count, front, ready[j], ready[j] ? ready_entry[j] : 0ull);
}

__global__ void adj_levels_kernel(const AdjProb *probs, int nprob, int64_t total, AdjCtl *ctl,
                                  unsigned long long *front, long long timeout_ns) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t warp0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + (threadIdx.x & ~31u);
  const unsigned lane = threadIdx.x & 31u;
  for (unsigned long long level = 0;; ++level) {
    const int cur = static_cast<int>(level % 3ull);
    const int nxt = static_cast<int>((level + 1ull) % 3ull);
    const unsigned long long n_cur = ld_rlx_u64(&ctl->nfront[cur]);
    if (n_cur == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->levels = level;
      return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nfront[(level + 2ull) % 3ull] = 0ull;
    const unsigned long long *in = front + (level & 1ull) * static_cast<unsigned long long>(total);
    unsigned long long *out = front + ((level + 1ull) & 1ull) * static_cast<unsigned long long>(total);
    for (int64_t b = warp0; b < static_cast<int64_t>(n_cur); b += stride) {
      const int64_t i = b + lane;
      const bool live = i < static_cast<int64_t>(n_cur);
      int pi = 0;
      int64_t n = 0;
      if (live) {
        const int64_t e = static_cast<int64_t>(in[i]);
        pi = find_adj_prob(probs, nprob, e);
        n = e - probs[pi].base;
      }
      adj_process(probs[pi], n, ctl, &ctl->nfront[nxt], out, live);
    }
    if (!grid_barrier(ctl, timeout_ns)) return;
  }
}

int g_sms = 0;

int sms() {
  if (!g_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

}  // namespace

cudaError_t launch_adjoint(const AdjProb *probs_dev, int nprob, int64_t total, AdjCtl *ctl,
                           unsigned long long *front, long long timeout_ns, cudaStream_t stream) {
  int64_t g = (total + 255) / 256;
  if (g > 8 * sms()) g = 8 * sms();
  if (g < 1) g = 1;
  adj_setup_kernel<<<static_cast<int>(g), 256, 0, stream>>>(probs_dev, nprob, total, ctl);
  adj_seed_kernel<<<static_cast<int>(g), 256, 0, stream>>>(probs_dev, nprob, total, ctl, front);
  note_launches(2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // co-resident blocks only: the levels meet at a grid barrier
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_levels_kernel, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm > 4) per_sm = 4;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  int blocks = sms() * per_sm;
  void *args[] = {const_cast<AdjProb **>(&probs_dev), &nprob, &total, &ctl, &front, &timeout_ns};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(adj_levels_kernel), dim3(blocks),
                                  dim3(256), args, 0, stream);
  note_launches(1);
  return e;
}

}  // namespace eik
