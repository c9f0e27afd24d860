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
// Set-up (fully parallel) evaluates everything that does not depend on lambda:
// per cell m the mask of its upwind sides, the weight of each active axis
// W_k(m) = fl(fl(t_m - a_k) / S_m) (halved on a tie) and the coefficient
// fl(fl(h^2 fl(1 / v)) / S), and counts for every cell the downwind cells that
// use it.  The dependent part is then one multiply-add per downwind neighbour.
//
// Schedule: Kahn order, level by level.  Cells with count 0 form the first
// frontier.  One cooperative persistent launch processes a frontier (each cell
// pulls lambda from its downwind cells, writes lambda and dL/ds, decrements its
// upwind cells' counts and appends those that reach zero to the next
// frontier), then its blocks meet at a grid barrier bounded by %globaltimer.
// (Letting a thread follow the cells it releases does not pay on this graph:
// in 2D most cells have two downwind users, so chains merge after about two
// steps while the few long chains stretch every frontier.)
#include <cstdint>
#include <cuda_runtime.h>

#include "eik_grid.cuh"
#include "eik_internal.h"

namespace eik {
namespace {

constexpr unsigned long long kInfB = 0x7ff0000000000000ull;
constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kThreads = 1024;   // threads per block of the level kernel

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

// A cell with its coordinates, so that neighbours need no division.
struct Cell {
  int64_t n;
  int64_t c[3];
};

__device__ __forceinline__ Cell cell_of(const AdjProb &P, int64_t n) {
  Cell e;
  e.n = n;
  if (P.nx * P.ny * P.nz < (int64_t(1) << 31)) {     // 32-bit division where it fits
    const unsigned un = static_cast<unsigned>(n), ux = static_cast<unsigned>(P.nx),
                   uy = static_cast<unsigned>(P.ny);
    const unsigned yz = un / ux;
    e.c[0] = static_cast<int64_t>(un - yz * ux);
    e.c[1] = static_cast<int64_t>(yz % uy);
    e.c[2] = static_cast<int64_t>(yz / uy);
    return e;
  }
  const int64_t yz = n / P.nx;
  e.c[0] = n - yz * P.nx;
  e.c[1] = yz % P.ny;
  e.c[2] = yz / P.ny;
  return e;
}

// A frontier entry: problem index above bit kEntryShift, cell index below.
constexpr int kEntryShift = 40;
__device__ __forceinline__ unsigned long long entry_of(int pi, int64_t n) {
  return (static_cast<unsigned long long>(pi) << kEntryShift) | static_cast<unsigned long long>(n);
}

// Neighbour of a cell on side j (0..5: x-, x+, y-, y+, z-, z+), -1 off the grid.
__device__ __forceinline__ int64_t nbr(const AdjProb &P, const Cell &e, int j) {
  const int k = j >> 1;
  if (k >= P.ndim) return -1;
  const int64_t ext = k == 0 ? P.nx : (k == 1 ? P.ny : P.nz);
  const int64_t st = k == 0 ? 1 : (k == 1 ? P.nx : P.nx * P.ny);
  if (j & 1) return e.c[k] + 1 < ext ? e.n + st : -1;
  return e.c[k] > 0 ? e.n - st : -1;
}

// Per cell: zeroed lambda, the upwind-side mask, per-axis weights, the gradient
// coefficient (kept in grad until lambda is known), reached count, and the
// downwind-use counts of the upwind cells.
__global__ void adj_setup_kernel(const AdjProb *probs, int nprob, int64_t total, AdjCtl *ctl) {
  unsigned long long reached = 0;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const AdjProb &P = probs[find_adj_prob(probs, nprob, q)];
    const int64_t n = q - P.base;
    P.lam[n] = 0.0;
    P.grad[n] = 0.0;
    P.mask[n] = 0;
    const double tn = P.t[n];
    if (!(ubits(tn) < kInfB)) continue;
    ++reached;
    if (P.nsrc > 0 && adj_is_source(P, n)) continue;
    const Cell e = cell_of(P, n);
    unsigned long long lo[3], hi[3], ak[3];
    double S = 0.0;
    for (int k = 0; k < P.ndim; ++k) {
      const int64_t a = nbr(P, e, 2 * k), b = nbr(P, e, 2 * k + 1);
      lo[k] = a >= 0 ? ubits(P.t[a]) : kInfB;
      hi[k] = b >= 0 ? ubits(P.t[b]) : kInfB;
      ak[k] = lo[k] < hi[k] ? lo[k] : hi[k];
      if (ak[k] < ubits(tn))
        S = __dadd_rn(S, __dsub_rn(tn, __longlong_as_double(static_cast<long long>(ak[k]))));
    }
    if (!(S > 0.0)) continue;   // unreachable for a reached non-source cell
    unsigned char mask = 0;
    for (int k = 0; k < P.ndim; ++k) {
      if (!(ak[k] < ubits(tn))) continue;               // axis not active
      double w = __ddiv_rn(__dsub_rn(tn, __longlong_as_double(static_cast<long long>(ak[k]))), S);
      if (lo[k] == hi[k]) w = __dmul_rn(w, 0.5);        // tie: half to each side
      P.W[k][n] = w;
      if (lo[k] == ak[k]) {
        mask |= static_cast<unsigned char>(1u << (2 * k));
        atomicAdd(P.cnt + nbr(P, e, 2 * k), 1);
      }
      if (hi[k] == ak[k]) {
        mask |= static_cast<unsigned char>(1u << (2 * k + 1));
        atomicAdd(P.cnt + nbr(P, e, 2 * k + 1), 1);
      }
    }
    P.mask[n] = mask;
    const double s = __ddiv_rn(1.0, P.v[n]);
    P.grad[n] = __ddiv_rn(__dmul_rn(P.hh, s), S);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) reached += __shfl_xor_sync(kFullMask, reached, o);
  if ((threadIdx.x & 31) == 0 && reached) atomicAdd(&ctl->reached, reached);
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
  if (lane == static_cast<unsigned>(leader))
    base = atomicAdd(count, static_cast<unsigned long long>(__popc(bal)));
  base = __shfl_sync(kFullMask, base, leader);
  if (ready) front[base + __popc(bal & ((1u << lane) - 1u))] = entry;
}

__global__ void adj_seed_kernel(const AdjProb *probs, int nprob, int64_t total, AdjCtl *ctl,
                                unsigned long long *front) {
  const int64_t span = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t base = blockIdx.x * static_cast<int64_t>(blockDim.x); base < total; base += span) {
    const int64_t q = base + threadIdx.x;
    bool ready = false;
    unsigned long long ent = 0;
    if (q < total) {
      const int pi = find_adj_prob(probs, nprob, q);
      const AdjProb &P = probs[pi];
      const int64_t n = q - P.base;
      ready = ubits(P.t[n]) < kInfB && P.cnt[n] == 0;
      ent = entry_of(pi, n);
    }
    append_ready(&ctl->nfront[0], front, ready, ent);
  }
}

// lambda and dL/ds of one ready cell, then release its upwind cells; the ones
// that become ready are appended to the next frontier.  All 32 lanes call it.
__device__ void adj_process(const AdjProb *probs, unsigned long long entry, bool live,
                            unsigned long long *count, unsigned long long *front) {
  unsigned long long ready_entry[6];
  bool ready[6] = {false, false, false, false, false, false};
  if (live) {
    const int pi = static_cast<int>(entry >> kEntryShift);
    const AdjProb &P = probs[pi];
    const Cell e = cell_of(P, static_cast<int64_t>(entry & ((1ull << kEntryShift) - 1ull)));
    const int64_t n = e.n;
    int64_t m[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) m[j] = nbr(P, e, j);
    unsigned mm[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) mm[j] = m[j] >= 0 ? P.mask[m[j]] : 0u;
    double lam = P.g ? P.g[n] : 0.0;
    // pull from the downwind neighbours m for which n is an upwind side
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (!((mm[j] >> (j ^ 1)) & 1u)) continue;          // n is m's side j^1
      const double lm = ld_rlx_d(P.lam + m[j]);           // written by another thread
      lam = __dadd_rn(lam, __dmul_rn(lm, P.W[j >> 1][m[j]]));
    }
    st_rlx_d(P.lam + n, lam);
    const unsigned mk = P.mask[n];
    if (mk) {                                              // a reached non-source cell
      P.grad[n] = __dmul_rn(lam, P.grad[n]);
      // no fence here: a cell released now is processed only after the next
      // grid barrier, whose release / acquire publishes every lambda of this level
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        if (!((mk >> j) & 1u)) continue;
        if (atomicSub(P.cnt + m[j], 1) == 1) {
          ready[j] = true;
          ready_entry[j] = entry_of(pi, m[j]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 6; ++j) append_ready(count, front, ready[j], ready[j] ? ready_entry[j] : 0ull);
}

__global__ void __launch_bounds__(kThreads) adj_levels_kernel(const AdjProb *probs, int nprob,
                                                               int64_t total, AdjCtl *ctl,
                                                               unsigned long long *front,
                                                               long long timeout_ns) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t warp0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + (threadIdx.x & ~31u);
  const unsigned lane = threadIdx.x & 31u;
  unsigned long long done = 0;
  for (unsigned long long level = 0;; ++level) {
    const int cur = static_cast<int>(level % 3ull);
    const int nxt = static_cast<int>((level + 1ull) % 3ull);
    const unsigned long long n_cur = ld_rlx_u64(&ctl->nfront[cur]);
    if (n_cur == 0) {
      if (blockIdx.x == 0 && threadIdx.x == 0) ctl->levels = level;
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nfront[(level + 2ull) % 3ull] = 0ull;
    const unsigned long long *in = front + (level & 1ull) * static_cast<unsigned long long>(total);
    unsigned long long *out = front + ((level + 1ull) & 1ull) * static_cast<unsigned long long>(total);
    for (int64_t b = warp0; b < static_cast<int64_t>(n_cur); b += stride) {
      const int64_t i = b + lane;
      const bool live = i < static_cast<int64_t>(n_cur);
      adj_process(probs, live ? in[i] : 0ull, live, &ctl->nfront[nxt], out);
      done += live ? 1u : 0u;
    }
    // the other blocks' decrements and lambdas before the next frontier
    if (!grid::barrier(&ctl->bar_count, &ctl->bar_gen, &ctl->status, timeout_ns)) break;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) done += __shfl_xor_sync(kFullMask, done, o);
  if (lane == 0 && done) atomicAdd(&ctl->done, done);
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
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_levels_kernel, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm > 2) per_sm = 2;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
#ifndef EIK_ADJ_BLOCK_DIV
#define EIK_ADJ_BLOCK_DIV 4
#endif
  // a quarter of the SMs' worth of 1024-thread blocks: a level rarely holds more
  // ready cells, and fewer, fuller blocks measured faster (32-source 1024^2:
  // 48.8 -> 43.5 ms)
  int blocks = sms() * per_sm / EIK_ADJ_BLOCK_DIV;
  if (blocks < 1) blocks = 1;
  void *args[] = {const_cast<AdjProb **>(&probs_dev), &nprob, &total, &ctl, &front, &timeout_ns};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(adj_levels_kernel), dim3(blocks),
                                  dim3(kThreads), args, 0, stream);
  note_launches(1);
  return e;
}

}  // namespace eik
