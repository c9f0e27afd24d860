// Other schedules for the same exactly monotone update (d-bar), as ablations
// of the scheduling question the paper studies (section "TAO analysis of
// existing Eikonal solvers"): every schedule reaches the same bits
// (Theorem 1); they differ in the work they do (good / bad / empty updates,
// Figure 3's measure) and in time.
//
//  * Fast iterative method, Algorithm 3 with epsilon = 0, in bulk-synchronous
//    rounds: the cells of worklist w are updated; a cell whose value did not
//    decrease updates those of its neighbours that are not in w and pushes the
//    ones that decreased onto w'; a cell that decreased is pushed onto w'.
//  * Topology-driven schedule, Algorithm 4: every cell is updated in every
//    iteration until an iteration changes nothing.
//  * Fast sweeping method, Algorithm 5: sweeps in the 2^D axis directions,
//    each sweep's cells in hyperplane order (the cells of one hyperplane
//    x' + y' (+ z') = k in sweep coordinates are independent and run in
//    parallel; hyperplanes follow one another), until a full set of sweeps
//    changes nothing.
//
// One cooperative persistent launch per solve; rounds are separated by a grid
// barrier bounded by %globaltimer.  One thread per cell update, no tiles: the
// point is the schedule, not the speed.
#include <cstdint>
#include <cuda_runtime.h>

#include "eik_exact.cuh"
#include "eik_grid.cuh"
#include "eik_internal.h"

namespace eik {
namespace {

constexpr unsigned long long kInfB = 0x7ff0000000000000ull;
constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ unsigned long long ld_rlx_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// The update of cell n at the current field (relaxed loads: other threads
// commit meanwhile); commits a decrease with atomicMin.  Returns true if the
// value decreased.
template <int D>
__device__ __forceinline__ bool update_cell(const BspParams &p, int64_t n, unsigned long long &evals,
                                            unsigned long long &decs) {
  if (p.fixed[n]) return false;
  ++evals;
  const int64_t x = n % p.nx, yz = n / p.nx, y = yz % p.ny, z = yz / p.ny;
  unsigned long long *T = reinterpret_cast<unsigned long long *>(p.t);
  unsigned long long a[D];
  {
    const unsigned long long l = x > 0 ? ld_rlx_u64(T + n - 1) : kInfB;
    const unsigned long long r = x + 1 < p.nx ? ld_rlx_u64(T + n + 1) : kInfB;
    a[0] = l < r ? l : r;
  }
  {
    const unsigned long long l = y > 0 ? ld_rlx_u64(T + n - p.nx) : kInfB;
    const unsigned long long r = y + 1 < p.ny ? ld_rlx_u64(T + n + p.nx) : kInfB;
    a[1] = l < r ? l : r;
  }
  if constexpr (D == 3) {
    const int64_t s = p.nx * p.ny;
    const unsigned long long l = z > 0 ? ld_rlx_u64(T + n - s) : kInfB;
    const unsigned long long r = z + 1 < p.nz ? ld_rlx_u64(T + n + s) : kInfB;
    a[2] = l < r ? l : r;
  }
  const unsigned long long cur = ld_rlx_u64(T + n);
  unsigned long long nv;
  if (!hw::relax<D>(cur, a, static_cast<unsigned long long>(__double_as_longlong(p.c[n])), nv))
    return false;
  const unsigned long long old = atomicMin(T + n, nv);
  if (nv < old) { ++decs; return true; }
  return false;
}

__device__ __forceinline__ int64_t neighbour(const BspParams &p, int64_t n, int j) {
  const int k = j >> 1;
  if (k >= p.ndim) return -1;
  const int64_t x = n % p.nx, yz = n / p.nx, y = yz % p.ny, z = yz / p.ny;
  const int64_t c = k == 0 ? x : (k == 1 ? y : z);
  const int64_t ext = k == 0 ? p.nx : (k == 1 ? p.ny : p.nz);
  const int64_t st = k == 0 ? 1 : (k == 1 ? p.nx : p.nx * p.ny);
  if (j & 1) return c + 1 < ext ? n + st : -1;
  return c > 0 ? n - st : -1;
}

// Append n to w_{r+1} once (marks only grow).
__device__ __forceinline__ void push_next(const BspParams &p, unsigned r, int64_t n, int nxt) {
  unsigned *mk = p.mark[(r + 1u) & 1u];
  if (atomicMax(mk + n, r + 1u) < r + 1u) {
    const unsigned long long slot = atomicAdd(&p.ctl->nfront[nxt], 1ull);
    p.front[(r + 1u) & 1u][slot] = static_cast<unsigned long long>(n);
  }
}

__device__ __forceinline__ void add_counts(BspCtl *ctl, unsigned long long evals,
                                           unsigned long long decs) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    evals += __shfl_xor_sync(kFullMask, evals, o);
    decs += __shfl_xor_sync(kFullMask, decs, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (evals) atomicAdd(&ctl->evals, evals);
    if (decs) atomicAdd(&ctl->decreases, decs);
  }
}

// Sources: t = t0, fixed, and (for the worklist schedule) w_1 = the sources.
__global__ void bsp_seed_kernel(BspParams p, const int64_t *src_idx, const double *src_t, int64_t nsrc) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < nsrc;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t n = src_idx[i];
    p.t[n] = src_t[i];
    p.fixed[n] = 1;
    p.mark[1][n] = 1u;
    p.front[1][i] = static_cast<unsigned long long>(n);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) p.ctl->nfront[1] = static_cast<unsigned long long>(nsrc);
}

template <int D>
__global__ void fim_kernel(BspParams p) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t gtid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  unsigned long long evals = 0, decs = 0;
  for (unsigned r = 1;; ++r) {
    const int cur = static_cast<int>(r % 3u), nxt = static_cast<int>((r + 1u) % 3u);
    const unsigned long long n_cur = ld_rlx_u64(&p.ctl->nfront[cur]);
    if (n_cur == 0) {
      if (gtid == 0) p.ctl->rounds = r - 1u;
      break;
    }
    if (gtid == 0) p.ctl->nfront[(r + 2u) % 3u] = 0ull;
    const unsigned long long *w = p.front[r & 1u];
    const unsigned *in_w = p.mark[r & 1u];
    for (int64_t i = gtid; i < static_cast<int64_t>(n_cur); i += stride) {
      const int64_t n = static_cast<int64_t>(w[i]);
      if (update_cell<D>(p, n, evals, decs)) {
        push_next(p, r, n, nxt);                        // not converged: again next round
        continue;
      }
      for (int j = 0; j < 2 * D; ++j) {                 // converged: update the neighbours
        const int64_t m = neighbour(p, n, j);
        if (m < 0 || in_w[m] == r) continue;            // m is in w: its own update follows
        if (update_cell<D>(p, m, evals, decs)) push_next(p, r, m, nxt);
      }
    }
    if (!grid::barrier(&p.ctl->bar_count, &p.ctl->bar_gen, &p.ctl->status, p.timeout_ns)) break;
  }
  add_counts(p.ctl, evals, decs);
}

template <int D>
__global__ void topo_kernel(BspParams p) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t gtid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t n_all = p.nx * p.ny * p.nz;
  unsigned long long evals = 0, decs = 0;
  for (unsigned it = 0;; ++it) {
    if (gtid == 0) p.ctl->nfront[(it + 1u) % 3u] = 0ull;   // change count of the next iteration
    unsigned long long changed = 0;
    for (int64_t n = gtid; n < n_all; n += stride) changed += update_cell<D>(p, n, evals, decs) ? 1u : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) changed += __shfl_xor_sync(kFullMask, changed, o);
    if ((threadIdx.x & 31) == 0 && changed) atomicAdd(&p.ctl->nfront[it % 3u], changed);
    if (!grid::barrier(&p.ctl->bar_count, &p.ctl->bar_gen, &p.ctl->status, p.timeout_ns)) break;
    if (ld_rlx_u64(&p.ctl->nfront[it % 3u]) == 0) {
      if (gtid == 0) p.ctl->rounds = it + 1u;
      break;
    }
  }
  add_counts(p.ctl, evals, decs);
}

template <int D>
__global__ void fsm_kernel(BspParams p) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t gtid = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const int64_t nx = p.nx, ny = p.ny, nz = D == 3 ? p.nz : 1;
  const int64_t planes = nx + ny + nz - 2;
  unsigned long long evals = 0, decs = 0;
  for (unsigned it = 0;; ++it) {
    if (gtid == 0) p.ctl->nfront[(it + 1u) % 3u] = 0ull;   // change count of the next iteration
    unsigned long long changed = 0;
    bool ok = true;
    for (int d = 0; d < (1 << D) && ok; ++d) {
      for (int64_t k = 0; k < planes; ++k) {
        if (D == 2) {
          const int64_t lo = k - (ny - 1) > 0 ? k - (ny - 1) : 0;
          const int64_t hi = k < nx - 1 ? k : nx - 1;
          for (int64_t xs = lo + gtid; xs <= hi; xs += stride) {
            const int64_t ys = k - xs;
            const int64_t x = (d & 1) ? nx - 1 - xs : xs, y = (d & 2) ? ny - 1 - ys : ys;
            changed += update_cell<D>(p, y * nx + x, evals, decs) ? 1u : 0u;
          }
        } else {
          for (int64_t q = gtid; q < nx * ny; q += stride) {
            const int64_t xs = q % nx, ys = q / nx, zs = k - xs - ys;
            if (zs < 0 || zs >= nz) continue;
            const int64_t x = (d & 1) ? nx - 1 - xs : xs, y = (d & 2) ? ny - 1 - ys : ys;
            const int64_t z = (d & 4) ? nz - 1 - zs : zs;
            changed += update_cell<D>(p, (z * ny + y) * nx + x, evals, decs) ? 1u : 0u;
          }
        }
        if (!grid::barrier(&p.ctl->bar_count, &p.ctl->bar_gen, &p.ctl->status, p.timeout_ns)) {
          ok = false;
          break;
        }
      }
    }
    if (!ok) break;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) changed += __shfl_xor_sync(kFullMask, changed, o);
    if ((threadIdx.x & 31) == 0 && changed) atomicAdd(&p.ctl->nfront[it % 3u], changed);
    if (!grid::barrier(&p.ctl->bar_count, &p.ctl->bar_gen, &p.ctl->status, p.timeout_ns)) break;
    if (ld_rlx_u64(&p.ctl->nfront[it % 3u]) == 0) {
      if (gtid == 0) p.ctl->rounds = it + 1u;
      break;
    }
  }
  add_counts(p.ctl, evals, decs);
}

int sm_count() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <typename K>
cudaError_t launch_coop(K kernel, BspParams &p, cudaStream_t stream, int max_per_sm = 4) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm > max_per_sm) per_sm = max_per_sm;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  void *args[] = {&p};
  e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(kernel), dim3(sm_count() * per_sm),
                                  dim3(256), args, 0, stream);
  note_launches(1);
  return e;
}

}  // namespace

cudaError_t launch_bsp_seed(const BspParams &p, const int64_t *src_idx, const double *src_t,
                            int64_t nsrc, cudaStream_t stream) {
  int64_t g = (nsrc + 255) / 256;
  if (g < 1) g = 1;
  if (g > 1024) g = 1024;
  bsp_seed_kernel<<<static_cast<int>(g), 256, 0, stream>>>(p, src_idx, src_t, nsrc);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_schedule(int schedule, BspParams p, cudaStream_t stream) {
  if (schedule == kScheduleFim)
    return p.ndim == 3 ? launch_coop(fim_kernel<3>, p, stream) : launch_coop(fim_kernel<2>, p, stream);
  if (schedule == kScheduleTopo)
    return p.ndim == 3 ? launch_coop(topo_kernel<3>, p, stream) : launch_coop(topo_kernel<2>, p, stream);
  if (schedule == kScheduleFsm)   // short hyperplanes, many barriers: one block per SM
    return p.ndim == 3 ? launch_coop(fsm_kernel<3>, p, stream, 1) : launch_coop(fsm_kernel<2>, p, stream, 1);
  return cudaErrorInvalidValue;
}

}  // namespace eik
