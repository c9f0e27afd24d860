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
// Two schedules process the cells in dependency (Kahn) order with the same
// operations in the same order, so their results are identical:
//  * tiles (the default; see "Tile schedule" below): persistent CTAs take
//    tiles from a queue and run the order inside a tile in shared memory,
//    handing cross-tile dependencies over through counts and the queue;
//  * levels: cells with count 0 form the first frontier; one cooperative
//    persistent launch processes a frontier (each cell pulls lambda from its
//    downwind cells, writes lambda and dL/ds, decrements its upwind cells'
//    counts and appends those that reach zero to the next frontier), then its
//    blocks meet at a grid barrier bounded by %globaltimer.  (Letting a thread
//    follow the cells it releases does not pay on this graph: in 2D most cells
//    have two downwind users, so chains merge after about two steps while the
//    few long chains stretch every frontier.)
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
__global__ void adj_setup_kernel(const AdjProb *probs, int nprob, int64_t total, AdjCtl *ctl,
                                 int tx, int ty, int tz) {
  // tx > 0: tile schedule with tiles tx x ty x tz: a downwind user in another
  // tile counts in cnt_out
  const int tdim[3] = {tx, ty, tz};
  unsigned long long reached = 0;
  for (int64_t q = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; q < total;
       q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const AdjProb &P = probs[find_adj_prob(probs, nprob, q)];
    const int64_t n = q - P.base;
    if (P.lam) P.lam[n] = 0.0;   // the tile schedule does not store lambda
    P.grad[n] = 0.0;
    P.mask[n] = 0;
    const double tn = P.t[n];
    const bool is_reached = ubits(tn) < kInfB;
    if (tx > 0) P.status[n] = is_reached ? 1 : 0;
    if (!is_reached) continue;
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
      // the upwind neighbour on the low side is in another tile when this cell
      // starts its tile along axis k; on the high side when it ends it
      const bool lo_out = tx > 0 && e.c[k] % tdim[k] == 0;
      const bool hi_out = tx > 0 && (e.c[k] + 1) % tdim[k] == 0;
      if (lo[k] == ak[k]) {
        mask |= static_cast<unsigned char>(1u << (2 * k));
        atomicAdd((lo_out ? P.cnt_out : P.cnt) + nbr(P, e, 2 * k), 1);
      }
      if (hi[k] == ak[k]) {
        mask |= static_cast<unsigned char>(1u << (2 * k + 1));
        atomicAdd((hi_out ? P.cnt_out : P.cnt) + nbr(P, e, 2 * k + 1), 1);
      }
    }
    P.mask[n] = mask;
    // slowness input: v = fl(1/s_in) as the forward used, then s = fl(1/v)
    const double vn = P.v_is_slowness ? __ddiv_rn(1.0, P.v[n]) : P.v[n];
    const double s = __ddiv_rn(1.0, vn);
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

// ---------------------------------------------------------------------------
// Tile schedule.  The same per-cell work in the same order as above, but the
// unit of scheduling is a tile of cells held in shared memory.  A cell's users
// are split into those in its own tile (cnt, decremented in shared memory while
// the tile is visited) and those in other tiles (cnt_out, decremented with a
// global atomic after the user's lambda is published).  A tile is visited when
// one of its cells may have become ready; a visit runs Kahn rounds in shared
// memory until none of its cells is ready, so the critical path costs a block
// barrier per level instead of a grid barrier.
//
// Tile state word: bit 0 = activated (queued, or to be queued again), bit 1 =
// being visited.  Activation is one atomicOr, so it is ordered against the
// visitor's claim and finish.  The queue is a bounded ring of sequence-tagged
// slots: a slot holds FREE(i) when index i may be pushed into it, FULL(i, tile)
// once pushed.
// ---------------------------------------------------------------------------
constexpr unsigned kTActive = 1u, kTRunning = 2u;
constexpr unsigned kNoTile = 0xffffffffu;

__device__ __forceinline__ unsigned long long slot_free(unsigned long long i) {
  return (i << 32) | kNoTile;
}
__device__ __forceinline__ unsigned long long slot_full(unsigned long long i, unsigned tile) {
  return (i << 32) | tile;
}
__device__ __forceinline__ unsigned long long ld_rlx_slot(const unsigned long long *p) {
  return ld_rlx_u64(p);
}
__device__ __forceinline__ void st_rlx_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_acq_s32(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_rlx_s32(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_rlx_u8(const unsigned char *p) {
  unsigned short v;
  asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return v;
}

struct TileQueue {
  unsigned *state;
  unsigned long long *ring;
  unsigned long long mask;   // ring slots - 1
  AdjCtl *ctl;
  long long timeout_ns;
};

__device__ __forceinline__ void tq_fail(const TileQueue &q) { atomicCAS(&q.ctl->status, 0u, kEtimeout); }

__device__ void tq_push(const TileQueue &q, unsigned tile) {
  const unsigned long long i = atomicAdd(&q.ctl->tail, 1ull);
  unsigned long long *slot = q.ring + (i & q.mask);
  const long long t0 = grid::now_ns();
  // at most total_tiles tiles are queued and the ring has at least that many
  // slots, so the slot's previous index has a taker, which frees it
  while (ld_rlx_slot(slot) != slot_free(i & 0xffffffffull)) {
    if (grid::now_ns() - t0 > q.timeout_ns) { tq_fail(q); return; }
  }
  st_rlx_u64(slot, slot_full(i & 0xffffffffull, tile));
}

// A cell of `tile` may have become ready (called after the release it follows
// and a fence).
__device__ void tq_activate(const TileQueue &q, unsigned tile) {
  if (atomicOr(q.state + tile, kTActive) == 0u) tq_push(q, tile);   // was idle
}

// Take the next queued tile; -1 when every reached cell is done or on error.
// The taker draws a ticket (fetch-and-add, no retry under contention) and
// waits on that slot alone until its tile is pushed.  The wait gives up when
// no cell has been processed anywhere for timeout_ns.
__device__ long long tq_pop(const TileQueue &q, unsigned long long reached) {
  const unsigned long long h = atomicAdd(&q.ctl->head, 1ull);
  unsigned long long *slot = q.ring + (h & q.mask);
  const unsigned long long tag = (h & 0xffffffffull) << 32;
  unsigned long long last_done = ~0ull;
  long long since = 0;
#pragma unroll 1
  for (;;) {
    const unsigned long long v = ld_rlx_slot(slot);
    if ((v & ~0xffffffffull) == tag && static_cast<unsigned>(v) != kNoTile) {
      st_rlx_u64(slot, slot_free((h + q.mask + 1ull) & 0xffffffffull));
      return static_cast<long long>(static_cast<unsigned>(v));
    }
    if (grid::ld_acq(&q.ctl->status) != 0u) return -1;
    const unsigned long long d = ld_rlx_u64(&q.ctl->done);
    if (d >= reached) return -1;
    const long long now = grid::now_ns();
    if (d != last_done) {
      last_done = d;
      since = now;
    } else if (now - since > q.timeout_ns) {
      tq_fail(q);
      return -1;
    }
    __nanosleep(128);
  }
}

__device__ __forceinline__ int find_tile_prob(const AdjProb *probs, int nprob, long long tile) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <int TX, int TY, int TZ>
__device__ __forceinline__ unsigned tile_of_cell(const AdjProb &P, int64_t x, int64_t y, int64_t z) {
  return static_cast<unsigned>(P.tile_base + ((z / TZ) * P.nty + (y / TY)) * P.ntx + (x / TX));
}

__global__ void adj_ring_init_kernel(unsigned long long *ring, unsigned long long slots) {
  for (unsigned long long i = blockIdx.x * static_cast<unsigned long long>(blockDim.x) + threadIdx.x;
       i < slots; i += static_cast<unsigned long long>(gridDim.x) * blockDim.x)
    ring[i] = slot_free(i);
}

// Queue the tiles holding a cell that is ready from the start.
template <int TX, int TY, int TZ>
__global__ void adj_tile_seed_kernel(const AdjProb *probs, int nprob, int64_t total, TileQueue q) {
  for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < total;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const AdjProb &P = probs[find_adj_prob(probs, nprob, g)];
    const int64_t n = g - P.base;
    if (P.status[n] != 1 || P.cnt[n] != 0 || P.cnt_out[n] != 0) continue;
    const Cell e = cell_of(P, n);
    tq_activate(q, tile_of_cell<TX, TY, TZ>(P, e.c[0], e.c[1], e.c[2]));
  }
}

// Persistent CTAs, one thread per cell of a tile.  In this schedule a
// processed cell m publishes the products p_k(m) = fl(lambda_m * W_k(m)) in
// place of its weights W_k(m) (its upwind cells need nothing else from it) and
// dL/ds; lambda itself is not stored.
//
// A visit takes a snapshot: a pending cell may be processed in this visit only
// if its cross-tile count read 0 (acquire) when the visit started; the products
// of its downwind neighbours across the tile edge are then final and are read
// once.  The visit is a Kahn queue in shared memory with one block barrier per
// round: the cells of the round's list, packed into the first threads so that
// a round's FP64 work occupies as few warps as possible, sum g and the
// products of their downwind neighbours in the fixed order (x-, x+, y-, y+,
// z-, z+), form their own products, and release their upwind cells in the tile;
// a cell whose in-tile count reaches zero joins the next round's list.  After
// the last round each thread publishes its own cell if it was processed, the
// tile is handed back, and the cross-tile releases follow (after a fence),
// queueing a tile whose cell's count reaches zero.  A cross-tile count that
// reaches zero during a visit marks the tile for another visit.
#ifndef EIK_ADJ_TILE_MINB
#define EIK_ADJ_TILE_MINB 4
#endif
// TIMING: per-CTA clocks of the visit phases and of the waits for work (the
// eik_stats timing fields); without it those reads compile out.
template <int D, int TX, int TY, int TZ, bool TIMING>
__global__ void __launch_bounds__(TX * TY * TZ, (EIK_ADJ_TILE_MINB * 256 + TX * TY * TZ - 1) /
                                                     (TX * TY * TZ)) adj_tiles_kernel(
    const AdjProb *probs, int nprob, TileQueue q) {
  constexpr int NT = TX * TY * TZ;
  constexpr unsigned kClear = 0x40u, kDid = 0x80u;   // s_flags; bits 0..2D-1: halo sides
  __shared__ double s_pw[D][NT];           // W_k, replaced by p_k once processed
  __shared__ double s_halo[2 * D][NT];     // product of the neighbour across the tile edge
  __shared__ double s_g[NT];
  __shared__ double s_lam[NT];
  __shared__ double s_coef[NT];
  __shared__ int s_cnt[NT];
  __shared__ unsigned char s_mask[NT];
  __shared__ unsigned char s_flags[NT];
  __shared__ unsigned short s_list[2][NT];
  __shared__ int s_n[3];
  __shared__ long long s_tile;
  __shared__ int s_prob;
  const int tid = threadIdx.x;
  const unsigned lane = threadIdx.x & 31u;
  const int lc[3] = {tid % TX, (tid / TX) % TY, tid / (TX * TY)};
  constexpr int tdim[3] = {TX, TY, TZ};
  constexpr int lstride[3] = {1, TX, TX * TY};
  const unsigned long long reached = ld_rlx_u64(&q.ctl->reached);
  unsigned long long visits = 0, rounds = 0, visit_ns = 0, idle_ns = 0, cyc[4] = {0, 0, 0, 0};
  long long t_claim = 0, c0 = 0;
#pragma unroll 1
  for (;;) {
    if (tid == 0) {
      long long t_wait = 0;
      if constexpr (TIMING) {
        c0 = clock64();
        t_wait = grid::now_ns();
      }
      long long tile = tq_pop(q, reached);
      if constexpr (TIMING) {
        t_claim = grid::now_ns();
        idle_ns += static_cast<unsigned long long>(t_claim - t_wait);
      }
      int pi = 0;
      if (tile >= 0) {
        // queued -> being visited; activations from now on set bit 0 again
        if (atomicExch(q.state + tile, kTRunning) != kTActive) {
          tq_fail(q);                                 // a queued tile is claimed once
          tile = -1;
        } else {
          __threadfence();                            // the claim before the tile's loads
          pi = find_tile_prob(probs, nprob, tile);
        }
      }
      s_tile = tile;
      s_prob = pi;
      s_n[0] = s_n[1] = s_n[2] = 0;
      if constexpr (TIMING) {
        const long long c1 = clock64();
        cyc[0] += static_cast<unsigned long long>(c1 - c0);
        c0 = c1;
      }
    }
    __syncthreads();
    const long long tile = s_tile;
    if (tile < 0) break;
    {
    const AdjProb &P = probs[s_prob];
    const int64_t lt = tile - P.tile_base;
    const int64_t tx = lt % P.ntx, rest = lt / P.ntx;
    const int64_t gc[3] = {tx * TX + lc[0], (rest % P.nty) * TY + lc[1], (rest / P.nty) * TZ + lc[2]};
    const int64_t ext[3] = {P.nx, P.ny, P.nz};
    const int64_t gstride[3] = {1, P.nx, P.nx * P.ny};
    const bool present = gc[0] < P.nx && gc[1] < P.ny && gc[2] < P.nz;
    const int64_t n = present ? (gc[2] * P.ny + gc[1]) * P.nx + gc[0] : 0;
    // loads that do not depend on the cross-tile counts first, so that they are
    // in flight together with the acquire below
    unsigned st = 0u, mk = 0u, hm_out = 0u;
    double g = 0.0, coef = 0.0, pw[D];
    int cnt0 = 0;
    if (present) {
      st = ld_rlx_u8(P.status + n);
      mk = P.mask[n];
      cnt0 = ld_rlx_s32(P.cnt + n);
      g = P.g ? P.g[n] : 0.0;
      coef = P.grad[n];
    }
#pragma unroll
    for (int k = 0; k < D; ++k) pw[k] = present ? ld_rlx_d(P.W[k] + n) : 0.0;
#pragma unroll
    for (int j = 0; j < 2 * D; ++j) {
      const int k = j >> 1;
      const bool up = j & 1;
      const int l = lc[k] + (up ? 1 : -1);
      const int64_t c = gc[k] + (up ? 1 : -1);
      if (!present || (l >= 0 && l < tdim[k]) || c < 0 || c >= ext[k]) continue;
      const int64_t m = n + (up ? gstride[k] : -gstride[k]);
      if ((P.mask[m] >> (j ^ 1)) & 1u) hm_out |= 1u << j;   // this cell is m's side j^1
    }
    const bool pending = st == 1u;
    const bool out_clear = pending && ld_acq_s32(P.cnt_out + n) == 0;
    unsigned flags = out_clear ? kClear : 0u;
#pragma unroll
    for (int j = 0; j < 2 * D; ++j) {
      if (!out_clear || !((hm_out >> j) & 1u)) continue;
      const int k = j >> 1;
      const int64_t m = n + ((j & 1) ? gstride[k] : -gstride[k]);
      s_halo[j][tid] = ld_rlx_d(P.W[k] + m);                 // m's product, final
      flags |= 1u << j;
    }
    s_g[tid] = g;
    s_coef[tid] = coef;
    s_cnt[tid] = pending ? cnt0 : -1;             // -1: no release ever targets it
    s_mask[tid] = static_cast<unsigned char>(mk);
    s_flags[tid] = static_cast<unsigned char>(flags);
#pragma unroll
    for (int k = 0; k < D; ++k) s_pw[k][tid] = pw[k];
    if (out_clear && cnt0 == 0) s_list[0][atomicAdd(&s_n[0], 1)] = static_cast<unsigned short>(tid);
    }
    __syncthreads();
    if (TIMING && tid == 0) {
      const long long c1 = clock64();
      cyc[1] += static_cast<unsigned long long>(c1 - c0);
      c0 = c1;
    }
    unsigned long long processed = 0;
    int round = 0;
#pragma unroll 1
    for (; round <= NT; ++round) {
      // the entry is read together with the count (an unused slot holds some
      // earlier cell index, masked into the tile)
      const int n_cur = s_n[round % 3];
      const int c_any = s_list[round & 1][tid] & (NT - 1);
      if (n_cur == 0) break;
      processed += static_cast<unsigned long long>(n_cur);
      if (tid == 0) s_n[(round + 2) % 3] = 0;       // last read in the previous round
      if ((tid & ~31) < n_cur) {                    // warp-uniform
        const bool live = tid < n_cur;
        const int c = live ? c_any : 0;
        const int cc[3] = {c % TX, (c / TX) % TY, c / (TX * TY)};
        // every shared load of the round first (addresses depend on c only), so
        // that their latencies overlap; then the FP64 chain; then the releases
        int nb[2 * D];
        bool inb[2 * D];
#pragma unroll
        for (int j = 0; j < 2 * D; ++j) {
          const int k = j >> 1;
          const int l = cc[k] + ((j & 1) ? 1 : -1);
          inb[j] = l >= 0 && l < tdim[k];
          nb[j] = inb[j] ? c + ((j & 1) ? lstride[k] : -lstride[k]) : c;
        }
        const unsigned fc = s_flags[c];
        const unsigned mc = s_mask[c];
        double lam = s_g[c];
        unsigned mn[2 * D], fu[2 * D];
        double tv[2 * D], th[2 * D];
#pragma unroll
        for (int j = 0; j < 2 * D; ++j) {
          mn[j] = s_mask[nb[j]];
          fu[j] = s_flags[nb[j]];
          tv[j] = s_pw[j >> 1][nb[j]];
          th[j] = s_halo[j][c];                        // used only where flagged
        }
        unsigned fresh = 0u;                          // sides whose upwind cell became ready
        if (live) {
#pragma unroll
          for (int j = 0; j < 2 * D; ++j) {
            const bool halo = (fc >> j) & 1u;
            if (halo || (inb[j] && ((mn[j] >> (j ^ 1)) & 1u))) lam = __dadd_rn(lam, halo ? th[j] : tv[j]);
          }
          s_lam[c] = lam;
#pragma unroll
          for (int k = 0; k < D; ++k)
            if ((mc >> (2 * k)) & 3u) s_pw[k][c] = __dmul_rn(lam, s_pw[k][c]);
          s_flags[c] = static_cast<unsigned char>(fc | kDid);
          int old[2 * D];
#pragma unroll
          for (int j = 0; j < 2 * D; ++j)
            old[j] = (((mc >> j) & 1u) && inb[j]) ? atomicSub(&s_cnt[nb[j]], 1) : 0;
#pragma unroll
          for (int j = 0; j < 2 * D; ++j)
            if (old[j] == 1 && (fu[j] & kClear)) fresh |= 1u << j;
        }
        // append the cells made ready, one shared atomic per warp
        unsigned total = 0u, below = 0u;
        const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
        for (int j = 0; j < 2 * D; ++j) {
          const unsigned b = __ballot_sync(kFullMask, (fresh >> j) & 1u);
          below += __popc(b & lt_mask);
          total += __popc(b);
        }
        int base = 0;
        if (n_cur <= 32) {                           // warp 0 alone appends this round
          if (lane == 0) s_n[(round + 1) % 3] = static_cast<int>(total);
        } else {
          if (lane == 0 && total) base = atomicAdd(&s_n[(round + 1) % 3], static_cast<int>(total));
          base = __shfl_sync(kFullMask, base, 0);
        }
        if (fresh) {
          int pos = base + static_cast<int>(below);
          // below counts the lower lanes' entries of every side; this lane's own
          // entries take the next slots in side order
          unsigned short *out = s_list[(round + 1) & 1];
#pragma unroll
          for (int j = 0; j < 2 * D; ++j)
            if ((fresh >> j) & 1u) out[pos++] = static_cast<unsigned short>(nb[j]);
        }
      }
      __syncthreads();
    }
    if (TIMING && tid == 0) {
      const long long c1 = clock64();
      cyc[2] += static_cast<unsigned long long>(c1 - c0);
      c0 = c1;
    }
    // the cell of this thread again (not kept in registers over the rounds)
    const AdjProb &P = probs[s_prob];
    const int64_t lt = tile - P.tile_base;
    const int64_t tx = lt % P.ntx, rest = lt / P.ntx;
    const int64_t gc[3] = {tx * TX + lc[0], (rest % P.nty) * TY + lc[1], (rest / P.nty) * TZ + lc[2]};
    const int64_t gstride[3] = {1, P.nx, P.nx * P.ny};
    const bool present = gc[0] < P.nx && gc[1] < P.ny && gc[2] < P.nz;
    const int64_t n = present ? (gc[2] * P.ny + gc[1]) * P.nx + gc[0] : 0;
    const unsigned fl = s_flags[tid];
    const unsigned mk = s_mask[tid];
    const bool did = (fl & kDid) != 0u;
    if (did) {
      if (mk) P.grad[n] = __dmul_rn(s_lam[tid], s_coef[tid]);
#pragma unroll
      for (int k = 0; k < D; ++k)
        if ((mk >> (2 * k)) & 3u) st_rlx_d(P.W[k] + n, s_pw[k][tid]);
      P.status[n] = 2;
    } else if (s_cnt[tid] >= 0) {
      P.cnt[n] = s_cnt[tid];                               // the in-tile releases of this visit
    }
    __threadfence();                                       // results before hand-back and releases
    __syncthreads();
    if (tid == 0) {
      if (processed) atomicAdd(&q.ctl->done, processed);
      ++visits;
      rounds += static_cast<unsigned long long>(round);
      // end of the visit: back to idle, or queued again when activated meanwhile
      if (atomicCAS(q.state + tile, kTRunning, 0u) != kTRunning) {
        atomicExch(q.state + tile, kTActive);
        tq_push(q, static_cast<unsigned>(tile));
      }
    }
    if (did) {
#pragma unroll
      for (int j = 0; j < 2 * D; ++j) {
        if (!((mk >> j) & 1u)) continue;
        const int k = j >> 1;
        const bool up = j & 1;
        const int l = lc[k] + (up ? 1 : -1);
        if (l >= 0 && l < tdim[k]) continue;
        if (atomicSub(P.cnt_out + n + (up ? gstride[k] : -gstride[k]), 1) == 1) {
          __threadfence();                                 // the release before the activation
          int64_t uc[3] = {gc[0], gc[1], gc[2]};
          uc[k] += up ? 1 : -1;
          tq_activate(q, tile_of_cell<TX, TY, TZ>(P, uc[0], uc[1], uc[2]));
        }
      }
    }
    if (TIMING && tid == 0) {
      visit_ns += static_cast<unsigned long long>(grid::now_ns() - t_claim);
      cyc[3] += static_cast<unsigned long long>(clock64() - c0);
    }
  }
  if (tid == 0) {
    atomicAdd(&q.ctl->visits, visits);
    atomicAdd(&q.ctl->rounds, rounds);
    atomicAdd(&q.ctl->ctas, 1ull);
    if constexpr (TIMING) {
      atomicAdd(&q.ctl->visit_ns, visit_ns);
      atomicAdd(&q.ctl->idle_ns, idle_ns);
#pragma unroll
      for (int i = 0; i < 4; ++i) atomicAdd(&q.ctl->cycles[i], cyc[i]);
    }
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
  adj_setup_kernel<<<static_cast<int>(g), 256, 0, stream>>>(probs_dev, nprob, total, ctl, 0, 0, 0);
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

namespace {

template <int D, int TX, int TY, int TZ>
cudaError_t run_tiles(const AdjProb *probs_dev, int nprob, int64_t total, int64_t total_tiles,
                      TileQueue q, unsigned long long qcap, int ctas_per_sm, bool timing,
                      cudaStream_t stream) {
  int64_t g = (total + 255) / 256;
  if (g > 8 * sms()) g = 8 * sms();
  if (g < 1) g = 1;
  int64_t gr = (static_cast<int64_t>(qcap) + 255) / 256;
  if (gr > 8 * sms()) gr = 8 * sms();
  adj_ring_init_kernel<<<static_cast<int>(gr), 256, 0, stream>>>(q.ring, qcap);
  adj_setup_kernel<<<static_cast<int>(g), 256, 0, stream>>>(probs_dev, nprob, total, q.ctl, TX, TY, TZ);
  adj_tile_seed_kernel<TX, TY, TZ><<<static_cast<int>(g), 256, 0, stream>>>(probs_dev, nprob, total, q);
  note_launches(3);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // persistent CTAs, all resident (a cooperative launch guarantees it): an idle
  // CTA waits for tiles that running CTAs queue
  constexpr int NT = TX * TY * TZ;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_tiles_kernel<D, TX, TY, TZ, true>, NT, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  if (ctas_per_sm > 0 && per_sm > ctas_per_sm) per_sm = ctas_per_sm;
  int64_t blocks = static_cast<int64_t>(sms()) * per_sm;
  if (blocks > total_tiles) blocks = total_tiles;
  if (blocks < 1) blocks = 1;
  void *args[] = {const_cast<AdjProb **>(&probs_dev), &nprob, &q};
  const void *fn = timing ? reinterpret_cast<const void *>(adj_tiles_kernel<D, TX, TY, TZ, true>)
                          : reinterpret_cast<const void *>(adj_tiles_kernel<D, TX, TY, TZ, false>);
  e = cudaLaunchCooperativeKernel(fn, dim3(static_cast<unsigned>(blocks)), dim3(NT), args, 0, stream);
  note_launches(1);
  return e;
}

}  // namespace

cudaError_t launch_adjoint_tiles(const AdjProb *probs_dev, int nprob, int64_t total,
                                 int64_t total_tiles, int ndim, AdjCtl *ctl, unsigned *tile_state,
                                 unsigned long long *queue, unsigned long long qcap,
                                 int ctas_per_sm, long long timeout_ns, bool timing,
                                 cudaStream_t stream) {
  if (total_tiles < 1 || qcap < static_cast<unsigned long long>(total_tiles) || (qcap & (qcap - 1)))
    return cudaErrorInvalidValue;
  TileQueue q;
  q.state = tile_state;
  q.ring = queue;
  q.mask = qcap - 1ull;
  q.ctl = ctl;
  q.timeout_ns = timeout_ns;
  if (ndim == 3)
    return run_tiles<3, kAdjTile3[0], kAdjTile3[1], kAdjTile3[2]>(probs_dev, nprob, total, total_tiles,
                                                                  q, qcap, ctas_per_sm, timing, stream);
  return run_tiles<2, kAdjTile2[0], kAdjTile2[1], kAdjTile2[2]>(probs_dev, nprob, total, total_tiles,
                                                                q, qcap, ctas_per_sm, timing, stream);
}

}  // namespace eik
