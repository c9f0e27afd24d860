// Kernels of the exactly monotone Eikonal solver for sm_103a.
//
// Method (arXiv 2103.05694): the first-order upwind update (Algorithm 1,
// Eq. finite_difference) evaluated with the exactly monotone rounding d-bar
// (section "Achieving Exact Monotonicity with Finite Precision Arithmetic"),
// applied under asynchronous relaxed-priority scheduling with integer buckets
// floor(t / delta) (Algorithm 6, the "Asynchronous Marching Method").  Because
// d-bar is monotone and causal, every schedule reaches the same bits
// (Theorem 1).
//
// GB300 design:
//  * Work item = a tile of cells (by default 16x16 for one 2D front, 16x8 for 2D
//    batches of 8 or more sources, 8x4x4 in 3D; other shapes by option), one CTA
//    (one thread per cell) relaxes it in shared memory: tile plus a one-cell
//    halo staged with coalesced relaxed loads, x-neighbours by warp shuffles,
//    y/z neighbours from shared memory, rounds of Jacobi relaxation driven by
//    double-buffered tile values until the tile is locally converged.
//  * Commits are 64-bit atomicMin on the bit pattern of the (non-negative)
//    arrival time; the minimum committed time on each tile face activates the
//    neighbour tile across that face (one aggregated push per face).
//  * Scheduler: persistent kernel; kNumSlots bucket slots, each a ring of
//    64-bit entries (tile | bucket << 32) with a sequence word per position;
//    warp 0 of a CTA scans 32 slots per step from the lowest-bucket hint,
//    reserves a written entry of a slot and takes the slot's next index (two
//    fetch-and-adds: hundreds of idle CTAs never serialise on a retried CAS),
//    then claims the tile through its state word (idle / queued(b) / running
//    / dirty(b)); a stale entry is dropped.  Termination: the count of
//    unfinished entries reaches zero.
//  * FP64 is scarce on this part (about 1.6 DFMA per SM per clock), so every
//    comparison, min, max and sign test runs on integer bit patterns, and a
//    cell is evaluated only when a neighbour changed.
//  * Every wait is bounded by %globaltimer; on expiry the kernel records
//    EIK_ETIMEOUT in the control block and returns (no trap).
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "eik_exact.cuh"
#include "eik_forms.cuh"
#include "eik_internal.h"

namespace eik {
namespace {

constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;
constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kMaxRounds = 1u << 20;   // per tile visit; never reached in practice

__device__ __forceinline__ unsigned long long bits_of(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}
__device__ __forceinline__ double from_bits(unsigned long long u) {
  return __longlong_as_double(static_cast<long long>(u));
}
__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) {
  return a < b ? a : b;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a < b ? b : a;
}

// Minimum of a 64-bit value over the full warp with two warp-reduce
// instructions (high words first, then the low words of the lanes that hold
// the smallest high word).
__device__ __forceinline__ unsigned long long warp_min64(unsigned long long v) {
  const unsigned hi = __reduce_min_sync(0xffffffffu, static_cast<unsigned>(v >> 32));
  const unsigned lo = __reduce_min_sync(
      0xffffffffu, static_cast<unsigned>(v >> 32) == hi ? static_cast<unsigned>(v) : 0xffffffffu);
  return (static_cast<unsigned long long>(hi) << 32) | lo;
}

// Phase timing (counters >= 2, thread 0): add the cycles since the last lap
// to slot k of the CTA's statistics (slot 12 holds the last lap's clock).
__device__ __forceinline__ void lap(long long *st, int k) {
  const long long c1 = clock64();
  st[k] += c1 - st[12];
  st[12] = c1;
}

// One axis of a cell after an acceptance step: sides (left/right) with their
// values after the step and whether they changed (decreased).  True when the
// axis minimum decreased and is now below `best`: the smallest changed value
// lies below every unchanged side's value and below `best`.
__device__ __forceinline__ bool axis_fell(bool c1, unsigned long long v1, bool c2,
                                          unsigned long long v2, unsigned long long best) {
  const unsigned long long lowered = umin64(c1 ? v1 : kInfBits, c2 ? v2 : kInfBits);
  const unsigned long long kept = umin64(c1 ? kInfBits : v1, c2 ? kInfBits : v2);
  return lowered < kept && lowered < best;
}

// A cell's candidate is pending while it differs from the cell's value
// (+inf: none); accepting it sets the value to it.
__device__ __forceinline__ bool is_pending(unsigned long long pv, unsigned long long t) {
  return pv != t && pv != kInfBits;
}

// Relaxed, GPU-scope accesses (never served from a stale L1 line).
__device__ __forceinline__ unsigned ld_rlx(const unsigned *p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_rlx(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_rlx(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_time(const double *p) {
  double v;
  asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rlx(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_rlx(unsigned *p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acq(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long now_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ void raise_status(Ctl *ctl, unsigned code, unsigned long long info) {
  if (atomicCAS(&ctl->status, 0u, code) == 0u) {
    ctl->error_info[0] = info;
  }
}

// ---------------------------------------------------------------------------
// Scheduler.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long make_state(unsigned long long st, unsigned bucket,
                                                         unsigned faces) {
  return (st << 40) | (static_cast<unsigned long long>(faces) << 32) | bucket;
}
__device__ __forceinline__ unsigned long long state_of(unsigned long long s) { return (s >> 40) & 3ull; }
__device__ __forceinline__ unsigned bucket_of(unsigned long long s) {
  return static_cast<unsigned>(s & 0x3fffffffull);
}
__device__ __forceinline__ unsigned faces_of(unsigned long long s) {
  return static_cast<unsigned>((s >> 32) & 0x7full);
}

__device__ __forceinline__ unsigned bucket_of_time(unsigned long long tb, float inv_delta) {
  const float q = __double2float_rn(from_bits(tb)) * inv_delta;
  if (!(q < static_cast<float>(kMaxBucket))) return kMaxBucket;
  return static_cast<unsigned>(q);
}

// Append (tile, b) to bucket b's slot.  The caller already owns the right to
// push (it moved the tile's state to queued(b)).
__device__ bool push_entry(const SolveParams &p, unsigned long long tile, unsigned b) {
  Ctl *ctl = p.ctl;
  atomicAdd(&ctl->work, 1);
  const unsigned s = b & (kNumSlots - 1);
  const unsigned cap = p.cap_mask + 1u;
  const unsigned idx = atomicAdd(&ctl->push[s * kCounterPad], 1u);
  // depth as a signed difference: a popper may already have taken index idx
  const int depth = static_cast<int>(idx - ld_rlx(&ctl->pop[s * kCounterPad]));
  if (depth >= static_cast<int>(cap)) {
    raise_status(ctl, kEcapacity, (static_cast<unsigned long long>(s) << 32) | idx);
    return false;
  }
  const size_t pos = static_cast<size_t>(s) * cap + (idx & p.cap_mask);
  const unsigned lap = idx & ~p.cap_mask;
  const unsigned long long e = (static_cast<unsigned long long>(b) << 32) | tile;
  long long t0 = 0;
  while (ld_acq(p.seq + pos) != lap) {   // the previous lap's entry not taken yet
    const long long now = now_ns();
    if (t0 == 0) t0 = now;
    else if (now - t0 > p.timeout_ns) { raise_status(ctl, kEcapacity, 1ull << 63); return false; }
    if (ld_rlx(&ctl->status)) return false;
    __nanosleep(64);
  }
  st_rlx(p.slots + pos, e);
  st_rel(p.seq + pos, lap + 1u);
  // the entry is written: one more for poppers to reserve
  atomicAdd(&ctl->avail[s * kCounterPad], 1);
  // A scanner may have moved the lowest-bucket hint past this slot between
  // the caller's read of the hint and the push: pull the hint back.  A
  // scanner's forward CAS from a stale value then fails.
  atomicMin(&ctl->cur, b);
  if (p.counters) {
    atomicAdd(&ctl->stats[kStatPushes], 1ull);
    if (depth > 0) atomicMax(&ctl->stats[kStatMaxQueue], static_cast<unsigned long long>(depth));
  }
  return true;
}

// A face of `tile` has new lower halo values (the smallest in bucket
// `bucket`): make sure the tile is (re)processed after this point.
__device__ void activate(const SolveParams &p, unsigned long long tile, unsigned face_bits,
                         unsigned bucket) {
  Ctl *ctl = p.ctl;
  const unsigned cur = ld_rlx(&ctl->cur);
  unsigned b = bucket;
  if (b < cur) b = cur;
  else if (b - cur >= kNumSlots) b = cur + kNumSlots - 1;
  if (b > kMaxBucket) b = kMaxBucket;
  unsigned long long old = ld_rlx(&p.state[tile]);
#pragma unroll 1
  for (int it = 0; it < (1 << 22); ++it) {
    const unsigned long long st = state_of(old);
    const unsigned ob = bucket_of(old), of = faces_of(old);
    unsigned long long nw;
    bool need_push = false;
    if (st == kStIdle) {
      nw = make_state(kStQueued, b, face_bits);
      need_push = true;
    } else if (st == kStQueued) {
      nw = make_state(kStQueued, b < ob ? b : ob, of | face_bits);
      need_push = b < ob;
    } else if (st == kStRunning) {
      nw = make_state(kStDirty, b, face_bits);
    } else {
      nw = make_state(kStDirty, b < ob ? b : ob, of | face_bits);
    }
    if (nw == old) return;
    const unsigned long long prev = atomicCAS(&p.state[tile], old, nw);
    if (prev == old) {
      if (need_push) push_entry(p, tile, b);
      return;
    }
    old = prev;
  }
  raise_status(ctl, kEtimeout, 3);
}

// Claim a popped entry: queued(b) -> running.  Returns the face mask, or -1
// if the entry is stale (the tile was re-queued elsewhere or is done).
__device__ int try_claim(const SolveParams &p, unsigned long long tile, unsigned b) {
  unsigned long long old = ld_rlx(&p.state[tile]);
#pragma unroll 1
  for (int it = 0; it < (1 << 22); ++it) {
    if (state_of(old) != kStQueued || bucket_of(old) != b) return -1;
    const unsigned long long prev = atomicCAS(&p.state[tile], old, make_state(kStRunning, 0, 0));
    if (prev == old) return static_cast<int>(faces_of(old));
    old = prev;
  }
  raise_status(p.ctl, kEtimeout, 4);
  return -1;
}

// End of a visit: running -> idle, or dirty(b) -> queued(b) plus a push.
__device__ void finish_tile(const SolveParams &p, unsigned long long tile) {
  unsigned long long old = ld_rlx(&p.state[tile]);
#pragma unroll 1
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned long long nw;
    const bool dirty = state_of(old) == kStDirty;
    nw = dirty ? make_state(kStQueued, bucket_of(old), faces_of(old)) : 0ull;
    const unsigned long long prev = atomicCAS(&p.state[tile], old, nw);
    if (prev == old) {
      if (dirty) push_entry(p, tile, bucket_of(old));
      return;
    }
    old = prev;
  }
  raise_status(p.ctl, kEtimeout, 5);
}

// The entry of index q of slot s (reserved by the caller): wait until its
// pusher has written it, take it and free the position for the next lap.
__device__ unsigned long long take_slot(const SolveParams &p, unsigned s, unsigned q) {
  const size_t pos = static_cast<size_t>(s) * (p.cap_mask + 1u) + (q & p.cap_mask);
  const unsigned lap = q & ~p.cap_mask;
  long long t0 = 0;
#pragma unroll 1
  for (;;) {
    if (ld_acq(p.seq + pos) == lap + 1u) {
      const unsigned long long e = ld_rlx(p.slots + pos);
      st_rel(p.seq + pos, lap + p.cap_mask + 1u);     // after the read of the entry
      return e;
    }
    const long long now = now_ns();
    if (t0 == 0) t0 = now;
    else if (now - t0 > p.timeout_ns) { raise_status(p.ctl, kEtimeout, 6); return kEmpty; }
    if (ld_rlx(&p.ctl->status)) return kEmpty;
    __nanosleep(32);
  }
}

// Warp 0: take one entry from the lowest active bucket slots.  A slot is
// active while it holds entries or tiles claimed from it are still running;
// the hint `cur` moves up to the lowest active slot, and only slots within
// `window` buckets of it are popped (bounded look-ahead, the soft priority of
// OBIM).  On success the slot's run counter has been incremented for the
// caller, `slot_out` is the slot and `lo_out` the lowest active bucket.
// Returns kEmpty when the solve is over (done or error).
__device__ unsigned long long pop_entry(const SolveParams &p, long long &idle_since,
                                        unsigned &slot_out, unsigned &lo_out) {
  Ctl *ctl = p.ctl;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned win = p.window < 31u ? p.window : 31u;
#pragma unroll 1
  for (;;) {
    unsigned stop = 0, cur = 0;
    if (lane == 0) {
      stop = ld_rlx(&ctl->status) | ld_rlx(&ctl->done);
      cur = ld_rlx(&ctl->cur);
    }
    stop = __shfl_sync(kFull, stop, 0);
    if (stop) return kEmpty;
    cur = __shfl_sync(kFull, cur, 0);
    // find the lowest active slot at or above the hint (whole ring if needed)
    unsigned first = 0xffffffffu;
    unsigned q = 0, pp = 0, s = 0;
    bool pend = false;
#pragma unroll 1
    for (unsigned base = 0; base < kNumSlots; base += 32) {
      s = (cur + base + lane) & (kNumSlots - 1);
      q = ld_rlx(&ctl->pop[s * kCounterPad]);
      pp = ld_rlx(&ctl->push[s * kCounterPad]);
      const unsigned rn = p.gate_pending_only ? 0u : ld_rlx(&ctl->run[s * kCounterPad]);
      pend = static_cast<int>(pp - q) > 0;
      const unsigned act = __ballot_sync(kFull, pend || rn > 0u);
      if (act) {
        first = base + static_cast<unsigned>(__ffs(act) - 1);
        break;
      }
    }
    if (first == 0xffffffffu) {
      int w = 0;
      if (lane == 0) w = ld_rlx(&ctl->work);
      w = __shfl_sync(kFull, w, 0);
      if (w == 0) {
        if (lane == 0) st_rlx(&ctl->done, 1u);
        return kEmpty;
      }
    } else {
      if (first > 0 && lane == 0 && cur + first <= kMaxBucket) atomicCAS(&ctl->cur, cur, cur + first);
      if (first >= 32) continue;   // re-read the 32 slots from the new hint
      const unsigned lo = cur + first;
      unsigned cand = __ballot_sync(kFull, pend && lane >= first && lane <= first + win);
#pragma unroll 1
      while (cand) {
        const int l = __ffs(cand) - 1;
        unsigned long long e = kEmpty;
        int got = 0;
        if (lane == static_cast<unsigned>(l)) {
          atomicAdd(&ctl->run[s * kCounterPad], 1u);   // keep the slot active meanwhile
          // reserve one written entry, then take the next index: two
          // fetch-and-adds, so many idle CTAs never serialise on a retried CAS.
          // Reservations never exceed the entries written, so pop <= push.  Only
          // a popper that has just seen an entry to reserve tries (a failed try
          // holds the count down until it is undone).
          int *av = &ctl->avail[s * kCounterPad];
          if (ld_rlx(av) > 0) {
            if (atomicAdd(av, -1) > 0) {
              got = 1;
              e = take_slot(p, s, atomicAdd(&ctl->pop[s * kCounterPad], 1u));
            } else {
              atomicAdd(av, 1);                           // nothing left: undo the try
            }
          }
          if (!got) atomicAdd(&ctl->run[s * kCounterPad], 0xffffffffu);
        }
        got = __shfl_sync(kFull, got, l);
        if (got) {
          e = __shfl_sync(kFull, e, l);
          slot_out = __shfl_sync(kFull, s, l);
          lo_out = lo;
          return e;  // kEmpty here means the solve is being aborted
        }
        cand &= ~(1u << l);
      }
    }
    if (lane == 0) {
      const long long now = now_ns();
      if (idle_since == 0) idle_since = now;
      else if (now - idle_since > p.timeout_ns) raise_status(ctl, kEtimeout, 2);
    }
    __nanosleep(128);
  }
}

__device__ __forceinline__ int find_prob(const SolveParams &p, unsigned long long tile) {
  int lo = 0, hi = p.nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (static_cast<unsigned long long>(p.probs[mid].tile_base) <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool is_source(const Prob &P, int64_t idx) {
  int64_t lo = 0, hi = P.nsrc - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int64_t v = P.src_idx[mid];
    if (v == idx) return true;
    if (v < idx) lo = mid + 1; else hi = mid - 1;
  }
  return false;
}

// ---------------------------------------------------------------------------
// Persistent kernel: pop a tile, relax it in shared memory, commit, activate
// neighbour tiles, repeat until no work is left anywhere.
//
// A visit relaxes cells in roughly increasing order of time (delta-stepping
// inside the tile): every round accepts the pending candidates within `band`
// cell travel times of their CTA-wide minimum m and evaluates the cells whose
// neighbours changed.  Within one travel time of m candidates cannot improve
// each other; the default, wider band also accepts provisional values, which
// later decreases correct (fewer rounds, more updates).
// Candidates at or above the visit limit V = (lowest active bucket + window
// + 1) * delta are deferred: recorded in the tile's pending mask and the tile
// re-queued at their bucket.  Only accepted values are written to memory.
// ---------------------------------------------------------------------------
// Register budget: resident_ctas(tile cells) CTAs per SM; the wide build of a
// lean 64-cell kernel, EIK_WIDE_CTAS_64.
template <int D, int TX, int TY, int TZ, int ARITH, bool LEAN, bool WIDE = false>
__global__ void __launch_bounds__(TX * TY * TZ, WIDE ? EIK_WIDE_CTAS_64 : resident_ctas(TX * TY * TZ))
    persistent_kernel(SolveParams p) {
  static_assert(!WIDE || (LEAN && TX * TY * TZ == 64), "wide builds: lean 64-cell kernels only");
  // LEAN: the instantiation for plain d-bar solves without counters, traces,
  // lane groups or change tracking (the timed path); those features compile
  // out of it.
  const int counters = LEAN ? 0 : p.counters;
  const int update = LEAN ? 0 : p.update;
  const int track_changes = LEAN ? 0 : p.track_changes;
  const bool tracing = !LEAN && p.trace != nullptr;
  const int lane_group_cells = LEAN ? 0 : p.lane_group_cells;
  const unsigned long long visit_budget = LEAN ? 0ull : p.visit_budget;
  constexpr int NT = TX * TY * TZ;
  static_assert(NT % 32 == 0 && NT <= 32 * kPendWords, "whole warps, one pending bit per cell");
  constexpr int HZ = (D == 3) ? 1 : 0;
  constexpr int SX = TX + 2, SY = TY + 2, SZ = TZ + 2 * HZ;
  static_assert(32 % TX == 0 || TX == 32, "a tile row must not straddle warps");
  __shared__ double s_t[2][SZ][SY][SX];     // values at the start of round R: s_t[R & 1]
  __shared__ unsigned long long s_a[D][NT];  // axis minima of the cells on the list
  __shared__ unsigned long long s_c[NT];     // c = fl(fl(h/v)^2) of each cell of the tile
  __shared__ unsigned long long s_best[NT];  // value a candidate must beat
  __shared__ unsigned long long s_pv[NT];    // pending candidate of each cell (owner-indexed)
  __shared__ unsigned short s_list[NT];    // cells whose update needs FP64 this round
  __shared__ int s_cnt[2];
  __shared__ unsigned long long s_facemin[6];
  __shared__ unsigned long long s_min[3];
  __shared__ unsigned long long s_cmin;
  __shared__ unsigned long long s_vlim;
  __shared__ float s_band_f;
  __shared__ long long s_tile;
  __shared__ int s_prob, s_faces;
  __shared__ unsigned s_slot, s_lo;
  __shared__ int s_cont;
  // statistics, kept in shared memory so that no thread carries them in
  // registers through the persistent loop: [0] evaluations, [1] acceptances,
  // [2] commits, [3] visits, [4] rounds, [5] visit ns, [6] idle ns, [7..11]
  // cycles per phase (counters >= 2), [12] phase clock, [13] idle since,
  // [14] claim time; s_path: d-bar path counts (counters >= 2)
  __shared__ long long s_stat[15];
  __shared__ unsigned s_path[4];
  // the claimed tile's geometry (thread 0 writes it with the claim) and the
  // solve's bucket and band scalars, in shared memory so that no thread
  // carries them in registers through the rounds: the grid's time array,
  // extents, tiles per axis, the tile's coordinates and the problem's first
  // global tile id
  __shared__ double *s_T;
  __shared__ long long s_n[3], s_nt[3], s_tc[3], s_tbase;
  __shared__ double s_delta;
  __shared__ float s_inv_delta, s_band_scale;

  const int tid = threadIdx.x;
  const unsigned lane = tid & 31;
  const int warp = tid >> 5;
  const int lx = tid % TX, ly = (tid / TX) % TY, lz = tid / (TX * TY);
  const int xc = lx + 1, yc = ly + 1, zc = lz + HZ;
  s_pv[tid] = kInfBits;
  if (tid == 0) { s_cmin = kInfBits; s_min[0] = s_min[1] = s_min[2] = kInfBits; s_cnt[0] = s_cnt[1] = 0; }
  if (tid < 15) s_stat[tid] = 0;
  if (tid < 4) s_path[tid] = 0u;
  if (tid == 0) {
    s_delta = p.ctl->delta;
    s_inv_delta = static_cast<float>(p.ctl->inv_delta);
    s_band_scale = static_cast<float>(p.band) * rsqrtf(static_cast<float>(D));
  }
  if (p.test_stall && tid == 0) {   // testing aid: wait on a flag nothing sets
    const long long t0 = now_ns();
    while (ld_rlx(&p.ctl->never_set) == 0u) {
      if (now_ns() - t0 > p.timeout_ns) { raise_status(p.ctl, kEtimeout, 8); break; }
      __nanosleep(1000);
    }
  }
  unsigned R = 1;
  __syncthreads();

#pragma unroll 1
  for (;;) {
    if (tid < 32) {
      long long tile = -1;
      int faces = 0;
      unsigned slot = 0, lo = 0;
      const long long t_pop = (counters || tracing) ? now_ns() : 0;
#pragma unroll 1
      for (;;) {
        const unsigned long long e = pop_entry(p, s_stat[13], slot, lo);
        if (e == kEmpty) break;
        const unsigned long long tl = e & 0xffffffffull;
        const unsigned b = static_cast<unsigned>(e >> 32);
        int f = -1;
        if (tid == 0) f = try_claim(p, tl, b);
        f = __shfl_sync(kFull, f, 0);
        if (f >= 0) { tile = static_cast<long long>(tl); faces = f; break; }
        if (tid == 0) {
          atomicAdd(&p.ctl->run[slot * kCounterPad], 0xffffffffu);
          atomicAdd(&p.ctl->work, -1);
          if (counters) atomicAdd(&p.ctl->stats[kStatStale], 1ull);
        }
      }
      if (tid == 0) {
        s_stat[13] = 0;
        if (counters || tracing) {
          s_stat[14] = now_ns();
          s_stat[6] += s_stat[14] - t_pop;
        }
        int prob = 0;
        if (tile >= 0) {
          __threadfence();  // the claim is ordered before the tile's loads
          prob = find_prob(p, static_cast<unsigned long long>(tile));
          if (visit_budget && atomicAdd(&p.ctl->visits_total, 1ull) >= visit_budget)
            raise_status(p.ctl, kEtimeout, 9);   // this visit runs; then every CTA stops
          const double vlim = static_cast<double>(lo + p.window + 1u) * s_delta;
          s_vlim = bits_of(vlim);
          const Prob &P = p.probs[prob];
          const long long lt = tile - P.tile_base;
          const long long rest = lt / P.ntx;
          s_T = P.t;
          s_n[0] = P.nx; s_n[1] = P.ny; s_n[2] = P.nz;
          s_nt[0] = P.ntx; s_nt[1] = P.nty; s_nt[2] = P.ntz;
          s_tc[0] = lt % P.ntx; s_tc[1] = rest % P.nty; s_tc[2] = rest / P.nty;
          s_tbase = P.tile_base;
        }
        s_tile = tile;
        s_faces = faces;
        s_prob = prob;
        s_slot = slot;
        s_lo = lo;
      }
    }
    __syncthreads();
    const long long tile = s_tile;
    if (tile < 0) break;
    const bool timing = counters >= 2 && tid == 0;
    if (timing) s_stat[12] = clock64();
    const int faces = s_faces;
    // this thread's cell from the tile's geometry: its global index, and
    // whether it lies inside the grid
    auto cell_of = [&](int64_t &gidx) -> bool {
      const int64_t gx = s_tc[0] * TX + lx, gy = s_tc[1] * TY + ly, gz = s_tc[2] * TZ + lz;
      gidx = (gz * s_n[1] + gy) * s_n[0] + gx;
      return gx < s_n[0] && gy < s_n[1] && gz < s_n[2];
    };
    double tv;
    unsigned long long cv;
    bool active;
    {
      int64_t gidx;
      const bool present = cell_of(gidx);
      const Prob &P = p.probs[s_prob];
      tv = present ? ld_time(s_T + gidx) : from_bits(kInfBits);
      cv = present ? static_cast<unsigned long long>(__ldg(reinterpret_cast<const long long *>(P.c) + gidx))
                   : kInfBits;
      active = present && !(p.tile_src[tile] && is_source(P, gidx));
    }
    s_c[tid] = cv;
    unsigned pword = 0;
    if (lane == 0) pword = ld_rlx(p.pend + static_cast<size_t>(tile) * kPendWords + warp);
    pword = __shfl_sync(kFull, pword, 0);
    {  // smallest c of the tile's active cells -> acceptance band
      const unsigned long long cb = warp_min64(active ? cv : kInfBits);
      if (lane == 0 && cb < kInfBits) atomicMin(&s_cmin, cb);
    }
    // A claimed tile is worked on until it has nothing left inside the window:
    // after each commit, a tile that neighbours re-activated meanwhile (dirty)
    // or whose deferred cells came inside the moved window continues here
    // with a fresh halo instead of going back through the queue.
    int faces_now = faces;
    bool first = true;
    unsigned long long m = kInfBits;
    unsigned rounds = 0;
    unsigned long long vlim = 0;
#pragma unroll 1
    for (;;) {
    // halo faces: -x, +x, -y, +y (, -z, +z)
    {
      constexpr int FX = TY * TZ, FY = TX * TZ, FZ = (D == 3) ? TX * TY : 0;
      constexpr int H = 2 * FX + 2 * FY + 2 * FZ;
      const double *const T = s_T;
      const int64_t nx = s_n[0], ny = s_n[1], nz = s_n[2];
      const int64_t x0 = s_tc[0] * TX, y0 = s_tc[1] * TY, z0 = s_tc[2] * TZ;
#pragma unroll 1
      for (int i = tid; i < H; i += NT) {
        int64_t hx, hy, hz;
        int sx, sy, sz;
        if (i < 2 * FY) {              // y faces, x fastest: coalesced
          const int side = i / FY, j = i % FY;
          const int ix = j % TX, iz = j / TX;
          hx = x0 + ix; hy = side ? y0 + TY : y0 - 1; hz = z0 + iz;
          sx = ix + 1; sy = side ? TY + 1 : 0; sz = iz + HZ;
        } else if (i < 2 * FY + 2 * FZ) {   // z faces
          const int k = i - 2 * FY;
          const int side = k / (FZ > 0 ? FZ : 1), j = k % (FZ > 0 ? FZ : 1);
          const int ix = j % TX, iy = j / TX;
          hx = x0 + ix; hy = y0 + iy; hz = side ? z0 + TZ : z0 - 1;
          sx = ix + 1; sy = iy + 1; sz = side ? TZ + 1 : 0;
        } else {                        // x faces
          const int k = i - 2 * FY - 2 * FZ;
          const int side = k / FX, j = k % FX;
          const int iy = j % TY, iz = j / TY;
          hx = side ? x0 + TX : x0 - 1; hy = y0 + iy; hz = z0 + iz;
          sx = side ? TX + 1 : 0; sy = iy + 1; sz = iz + HZ;
        }
        const bool in = hx >= 0 && hx < nx && hy >= 0 && hy < ny && hz >= 0 && hz < nz;
        const double hv = in ? ld_time(T + (hz * ny + hy) * nx + hx) : from_bits(kInfBits);
        s_t[0][sz][sy][sx] = hv;     // the halo is the same in both buffers
        s_t[1][sz][sy][sx] = hv;
      }
    }
    s_t[R & 1u][zc][yc][xc] = tv;    // this cell at the start of the pass's first round
    if (tid < 6) s_facemin[tid] = kInfBits;
    if (tid == 0) { s_min[0] = s_min[1] = s_min[2] = kInfBits; s_cnt[0] = 0; s_cnt[1] = 0; }
    __syncthreads();
    if (timing) lap(s_stat, 7);
    if (first && tid == 0) {   // band = k * sqrt(c_min) / sqrt(D): one cell's travel time
      const float cm = s_cmin < kInfBits ? xf::to_f(s_cmin) : 0.0f;
      // s_cmin is the smallest c (or r for the explicit roots): one cell's travel time
      s_band_f = (update ? cm : sqrtf(cm)) * s_band_scale;
      s_cmin = kInfBits;
    }
    vlim = s_vlim;

    const double tv0 = tv;
    // cells to evaluate in the pass's first round: every cell (a seeded tile),
    // cells with a deferred candidate, and cells on a face whose halo changed
    // (bit k of face_need: the neighbour across face k)
    const bool full_pass = (faces_now & (1 << kFaceFull)) != 0;
    const bool pend_cell = first ? ((pword >> lane) & 1u) != 0u : is_pending(s_pv[tid], bits_of(tv));
    const unsigned face_need =
        (((faces_now & 1) && lx == 0) ? 1u : 0u) | (((faces_now & 2) && lx == TX - 1) ? 2u : 0u) |
        (((faces_now & 4) && ly == 0) ? 4u : 0u) | (((faces_now & 8) && ly == TY - 1) ? 8u : 0u) |
        ((D == 3 && (faces_now & 16) && lz == 0) ? 16u : 0u) |
        ((D == 3 && (faces_now & 32) && lz == TZ - 1) ? 32u : 0u);
    bool need = active && (full_pass || pend_cell || face_need != 0u);
    // Pending candidates live in s_pv (owner-indexed); a candidate is pending
    // while it differs from the cell's value, so accepting it needs no clearing.
    // The values at the start of round R are in s_t[R & 1].  Accepting round
    // R-1's candidates and evaluating round R form one phase: each thread
    // derives its neighbours' acceptance from their candidates and s_t[(R-1) & 1]
    // (x neighbours by shuffles), and writes its own new value to s_t[R & 1].
    // Two barriers per round.  The minimum over the candidates pending after
    // round R accumulates in s_min[R % 3].
    m = kInfBits;
    unsigned pass_round = 0;
#pragma unroll 1
    for (;;) {
      const unsigned b = R & 1u, bo = b ^ 1u;
      const bool accept = pass_round > 0;
      unsigned long long lim = 0;
      if (accept) {
        // (C) accept round R-1's pending candidates within the band above their minimum
        m = s_min[(R - 1u) % 3u];
        ++rounds;
        if (m >= vlim) break;   // nothing pending below the visit limit (uniform)
        // m + band on the FP32 pipe (every thread gets the same value; the band is
        // a scheduling heuristic), never below m so the smallest candidate is
        // always accepted
        const float lf = __fadd_rn(xf::to_f(m), s_band_f);
        lim = umin64(umax64(xf::from_f(lf), m), vlim - 1);
      }
      bool acc = false;
      const unsigned long long pv = s_pv[tid];
      if (accept && is_pending(pv, bits_of(tv)) && pv <= lim) {
        tv = from_bits(pv);
        acc = true;
      }
      {  // what stays pending takes part in this round's minimum
        const unsigned long long keep = warp_min64(is_pending(pv, bits_of(tv)) ? pv : kInfBits);
        if (lane == 0 && keep < kInfBits) atomicMin(&s_min[R % 3u], keep);
      }
      if (accept) s_t[b][zc][yc][xc] = tv;
      // (A) neighbour values after the acceptance, which of them changed, and the
      //     exact integer filters; the cells that may decrease go on a dense list
      //     for the FP64 phase
      double xl = __shfl_up_sync(kFull, tv, 1, TX);
      double xr = __shfl_down_sync(kFull, tv, 1, TX);
      const unsigned accbits = __ballot_sync(kFull, acc);
      const bool cxl = lx > 0 && ((accbits >> (lane - 1)) & 1u);
      const bool cxr = lx < TX - 1 && ((accbits >> (lane + 1)) & 1u);
      if (lx == 0) xl = s_t[bo][zc][yc][0];
      if (lx == TX - 1) xr = s_t[bo][zc][yc][TX + 1];
      // a neighbour in another warp (or the halo) at offset (dz, dy) and tile
      // thread offset dt: its value after the acceptance, and whether it changed
      auto across = [&](int dz, int dy, int dt, bool inside, bool &chg) -> double {
        chg = false;
        const double old = s_t[accept ? bo : b][zc + dz][yc + dy][xc];
        if (!accept || !inside) return old;
        const unsigned long long q = s_pv[tid + dt];
        if (is_pending(q, bits_of(old)) && q <= lim) {
          chg = true;
          return from_bits(q);
        }
        return old;
      };
      bool cyl, cyr, czl = false, czr = false;
      double yl, yr;
      if constexpr (D == 3 && TX * TY <= 32) {
        // whole xy-slices per warp: the y neighbours inside the tile are lanes
        // +-TX of this warp (their values after the acceptance, and whether they
        // changed), the others the halo
        const double ys_l = __shfl_up_sync(kFull, tv, TX), ys_r = __shfl_down_sync(kFull, tv, TX);
        cyl = ly > 0 && ((accbits >> (lane - TX)) & 1u);
        cyr = ly < TY - 1 && ((accbits >> (lane + TX)) & 1u);
        yl = ly > 0 ? ys_l : s_t[accept ? bo : b][zc][yc - 1][xc];
        yr = ly < TY - 1 ? ys_r : s_t[accept ? bo : b][zc][yc + 1][xc];
      } else {
        yl = across(0, -1, -TX, ly > 0, cyl);
        yr = across(0, 1, TX, ly < TY - 1, cyr);
      }
      double zl = 0.0, zr = 0.0;
      if constexpr (D == 3) {
        zl = across(-1, 0, -TX * TY, lz > 0, czl);
        zr = across(1, 0, TX * TY, lz < TZ - 1, czr);
      }
      // change tracking compares with the cell's value (a recomputed value may
      // also be larger); otherwise a candidate must beat value and pending
      const unsigned long long best =
          track_changes ? bits_of(tv) : umin64(bits_of(tv), is_pending(pv, bits_of(tv)) ? pv : kInfBits);
      if (update) {
        // the explicit forms (not monotone): any neighbour change re-evaluates
        if (accept) need = active && (cxl || cxr || cyl || cyr || czl || czr);
      } else if (accept) {
        // d-bar (monotone, causal): the cell can decrease only if an axis
        // minimum fell below `best` -- for tau < best, G(tau) is unchanged when
        // every axis minimum that moved is still >= best, so d-bar < best iff it
        // was before (and it was not, or the cell would hold that value)
        need = active && (axis_fell(cxl, bits_of(xl), cxr, bits_of(xr), best) ||
                          axis_fell(cyl, bits_of(yl), cyr, bits_of(yr), best) ||
                          (D == 3 && axis_fell(czl, bits_of(zl), czr, bits_of(zr), best)));
      } else if (need && !full_pass && !pend_cell) {
        // first round: a changed halo value matters only below `best`
        need = ((face_need & 1u) && bits_of(xl) < best) || ((face_need & 2u) && bits_of(xr) < best) ||
               ((face_need & 4u) && bits_of(yl) < best) || ((face_need & 8u) && bits_of(yr) < best) ||
               ((face_need & 16u) && bits_of(zl) < best) || ((face_need & 32u) && bits_of(zr) < best);
      }
      bool go = false;
      if (need) {
        unsigned long long a[D];
        a[0] = umin64(bits_of(xl), bits_of(xr));
        a[1] = umin64(bits_of(yl), bits_of(yr));
        if constexpr (D == 3) a[D - 1] = umin64(bits_of(zl), bits_of(zr));
        unsigned long long amin = a[0];
#pragma unroll
        for (int k = 1; k < D; ++k) amin = umin64(amin, a[k]);
        go = amin < kInfBits && (track_changes || best > amin);
        if (go) {
#pragma unroll
          for (int k = 0; k < D; ++k) s_a[k][tid] = a[k];
          s_best[tid] = best;
        }
      }
      if (counters) {   // evaluations and acceptances of this round (warp-aggregated)
        const unsigned ev = __ballot_sync(kFull, need);
        if (lane == 0 && (ev | accbits)) {
          atomicAdd(reinterpret_cast<unsigned long long *>(&s_stat[0]), static_cast<unsigned long long>(__popc(ev)));
          atomicAdd(reinterpret_cast<unsigned long long *>(&s_stat[1]), static_cast<unsigned long long>(__popc(accbits)));
        }
      }
      ++pass_round;
      {
        const unsigned bal = __ballot_sync(kFull, go);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&s_cnt[b], __popc(bal));
        base = __shfl_sync(kFull, base, 0);
        if (go) s_list[base + __popc(bal & ((1u << lane) - 1u))] = static_cast<unsigned short>(tid);
      }
      __syncthreads();                                              // barrier 1
      if (timing) lap(s_stat, 8);
      // (B) dense arithmetic phase.  Few cells (at most lane_group_cells): a
      //     group of 8 (or 4) lanes per cell evaluates d-bar (guess + one G
      //     pass over a window of points); else one lane per cell.  Only warps
      //     holding work take part.
      {
        const int cnt = s_cnt[b];
        if (tid == 0) {
          s_cnt[bo] = 0;                          // the list of round R+1
          s_min[(R + 1u) % 3u] = kInfBits;        // the minimum after round R+1
        }
        unsigned long long nv = kInfBits;
        bool part = false;
        if (ARITH == kArithFp64 && cnt <= lane_group_cells && cnt * 4 <= NT && !update) {
          const int L = cnt * 8 <= NT ? 8 : 4;
          if (warp < (cnt * L + 31) / 32) {
            part = true;
            const int g = tid / L;
            const bool valid = g < cnt;
            const int c = valid ? s_list[g] : 0;
            unsigned long long a[D];
#pragma unroll
            for (int k = 0; k < D; ++k) a[k] = valid ? s_a[k][c] : kInfBits;
            const unsigned long long best = valid ? s_best[c] : kInfBits;
            const unsigned long long cb = valid ? s_c[c] : 0ull;
            unsigned long long out;
            const bool dec = L == 8 ? hw::relax_group<D, 8>(best, a, cb, valid, out)
                                    : hw::relax_group<D, 4>(best, a, cb, valid, out);
            if (dec) {
              nv = out;
              if ((tid & (L - 1)) == 0) s_pv[c] = out;
            }
          }
        } else if (tid < ((cnt + 31) & ~31)) {
          part = true;
          if (tid < cnt) {
            const int c = s_list[tid];
            unsigned long long a[D];
#pragma unroll
            for (int k = 0; k < D; ++k) a[k] = s_a[k][c];
            bool dec;
            if (D == 2 && update) {   // explicit roots: s_c holds r = fl(h/v)
              nv = forms::explicit_update(update, a[0], a[D - 1], from_bits(s_c[c]));
              if (track_changes) {    // the latest value replaces any pending one
                dec = nv != s_best[c];
                if (!dec) s_pv[c] = kInfBits;
              } else {
                dec = nv < s_best[c];
              }
            } else {
              dec = ARITH == kArithInt ? xf::relax<D>(s_best[c], a, s_c[c], nv)
                                       : hw::relax<D>(s_best[c], a, s_c[c], nv,
                                                      counters >= 2 ? s_path : nullptr);
            }
            if (dec) s_pv[c] = nv; else nv = kInfBits;
          }
        }
        if (part) {   // warp-uniform
          nv = warp_min64(nv);
          if (lane == 0 && nv < kInfBits) atomicMin(&s_min[R % 3u], nv);
        }
      }
      __syncthreads();                                              // barrier 2
      if (timing) lap(s_stat, 9);
      ++R;
      if (rounds >= kMaxRounds) {   // uniform across the CTA
        if (tid == 0) raise_status(p.ctl, kEtimeout, 7);
        break;
      }
    }
    ++R;

    // commit and collect the smallest committed time per tile face
    const bool track = track_changes != 0;
    const bool commit = track ? bits_of(tv) != bits_of(tv0) : bits_of(tv) < bits_of(tv0);
    if (counters) {
      const unsigned cm = __ballot_sync(kFull, commit);
      if (lane == 0 && cm)
        atomicAdd(reinterpret_cast<unsigned long long *>(&s_stat[2]), static_cast<unsigned long long>(__popc(cm)));
    }
    if (commit) {   // a committed cell lies inside the grid
      const unsigned long long tb = bits_of(tv);
      int64_t gidx;
      cell_of(gidx);
      if (track)   // a value may rise: only this tile's visit writes its cells
        st_rlx(reinterpret_cast<unsigned long long *>(s_T + gidx), tb);
      else
        atomicMin(reinterpret_cast<unsigned long long *>(s_T + gidx), tb);
      // a face value can change the cell across the face only if it is below
      // that cell's value (causality; the loaded halo value is an upper bound).
      // Change tracking activates on any change.
      const auto &H = s_t[0];   // halo entries (both buffers hold them)
      if (lx == 0 && (track || tb < bits_of(H[zc][yc][xc - 1]))) atomicMin(&s_facemin[0], tb);
      if (lx == TX - 1 && (track || tb < bits_of(H[zc][yc][xc + 1]))) atomicMin(&s_facemin[1], tb);
      if (ly == 0 && (track || tb < bits_of(H[zc][yc - 1][xc]))) atomicMin(&s_facemin[2], tb);
      if (ly == TY - 1 && (track || tb < bits_of(H[zc][yc + 1][xc]))) atomicMin(&s_facemin[3], tb);
      if constexpr (D == 3) {
        if (lz == 0 && (track || tb < bits_of(H[zc - 1][yc][xc]))) atomicMin(&s_facemin[4], tb);
        if (lz == TZ - 1 && (track || tb < bits_of(H[zc + 1][yc][xc]))) atomicMin(&s_facemin[5], tb);
      }
    }
    __threadfence();
    __syncthreads();
    if (tid < 2 * D) {
      const unsigned long long fm = s_facemin[tid];
      if (fm != kInfBits) {
        const int k = tid >> 1, side = tid & 1;
        const int64_t tx = s_tc[0], ty = s_tc[1], tz = s_tc[2];
        int64_t ntx = tx, nty = ty, ntz = tz;
        bool exists;
        if (k == 0) { ntx = side ? tx + 1 : tx - 1; exists = side ? (tx + 1 < s_nt[0]) : (tx > 0); }
        else if (k == 1) { nty = side ? ty + 1 : ty - 1; exists = side ? (ty + 1 < s_nt[1]) : (ty > 0); }
        else { ntz = side ? tz + 1 : tz - 1; exists = side ? (tz + 1 < s_nt[2]) : (tz > 0); }
        if (exists) {
          const unsigned long long nt =
              static_cast<unsigned long long>(s_tbase + (ntz * s_nt[1] + nty) * s_nt[0] + ntx);
          activate(p, nt, 1u << (tid ^ 1), bucket_of_time(fm, s_inv_delta));
        }
      }
      __threadfence();
    }
    // continue on this tile?  (dirty: take the new faces; deferred cells now
    // inside the moved window: take no faces)
    if (tid == 0) {
      int cont = 0;
      unsigned long long old = ld_rlx(&p.state[tile]);
      if (state_of(old) == kStDirty) {
        const unsigned long long prev = atomicCAS(&p.state[tile], old, make_state(kStRunning, 0, 0));
        if (prev == old) {
          cont = 1;
          s_faces = static_cast<int>(faces_of(old));
        }
      }
      if (!cont && m < kInfBits) {
        const unsigned lo2 = ld_rlx(&p.ctl->cur);
        const unsigned long long v2 = bits_of(static_cast<double>(lo2 + p.window + 1u) * s_delta);
        if (m < v2) {
          cont = 2;
          s_faces = 0;
          s_vlim = v2;
          s_lo = lo2;
        }
      }
      if (cont) __threadfence();   // the claim of the new work is ordered before the halo loads
      s_cont = cont;
    }
    __syncthreads();
    if (!s_cont) break;
    faces_now = s_faces;
    first = false;
    if (tid < 6) s_facemin[tid] = kInfBits;
    }   // continuation loop

    // cells still pending are deferred to a later visit
    {
      const bool deferred = is_pending(s_pv[tid], bits_of(tv));
      s_pv[tid] = kInfBits;
      const unsigned pend_bits = __ballot_sync(kFull, deferred);
      if (lane == 0) {
        unsigned *pw = p.pend + static_cast<size_t>(tile) * kPendWords + warp;
        asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(pw), "r"(pend_bits) : "memory");
      }
      __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
      if (timing) lap(s_stat, 11);
      if (m < kInfBits) {   // deferred cells: come back at their bucket, beyond this window
        unsigned b = bucket_of_time(m, s_inv_delta);
        const unsigned bmin = s_lo + p.window + 1u;
        if (b < bmin) b = bmin;
        activate(p, static_cast<unsigned long long>(tile), 0u, b);
      }
      finish_tile(p, static_cast<unsigned long long>(tile));
      __threadfence();
      atomicAdd(&p.ctl->run[s_slot * kCounterPad], 0xffffffffu);
      atomicAdd(&p.ctl->work, -1);
      s_stat[3] += 1;
      s_stat[4] += rounds;
      if (counters) s_stat[5] += now_ns() - s_stat[14];
      if (tracing) {
        const unsigned long long k = atomicAdd(&p.ctl->trace_n, 1ull);
        if (k < p.trace_cap) {
          TraceRec rec;
          rec.t_claim = s_stat[14];
          rec.t_end = now_ns();
          rec.tile = static_cast<unsigned>(tile);
          rec.lo = s_lo;
          rec.rounds = rounds;
          rec.flags = (m < kInfBits ? 1u : 0u) | (static_cast<unsigned>(blockIdx.x) << 8);
          p.trace[k] = rec;
        }
      }
    }
  }

  if (counters) {
    __syncthreads();
    if (tid == 0) {
      const unsigned long long *st = reinterpret_cast<const unsigned long long *>(s_stat);
      atomicAdd(&p.ctl->stats[kStatEvals], st[0]);
      atomicAdd(&p.ctl->stats[kStatDecreases], st[1]);
      atomicAdd(&p.ctl->stats[kStatCommits], st[2]);
      atomicAdd(&p.ctl->stats[kStatVisits], st[3]);
      atomicAdd(&p.ctl->stats[kStatRounds], st[4]);
      atomicAdd(&p.ctl->stats[kStatVisitNs], st[5]);
      atomicAdd(&p.ctl->stats[kStatIdleNs], st[6]);
      if (counters >= 2) {
#pragma unroll
        for (int k = 0; k < 5; ++k) atomicAdd(&p.ctl->stats[kStatCycLoad + k], st[7 + k]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (s_path[k]) atomicAdd(&p.ctl->stats[kStatNewton + k], static_cast<unsigned long long>(s_path[k]));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Set-up kernels.
// ---------------------------------------------------------------------------

// Per-cell constant of the update, c = fl(fl(h / v)^2) (the right-hand side
// (h/v)^2 of Eq. difference_as_root); checks v > 0 finite and r, c finite and
// positive; sums r = fl(h / v) for the auto bucket width.
__global__ void init_c_kernel(const double *__restrict__ speed, double h, double *__restrict__ c_out,
                              int64_t n, Ctl *ctl, int store_r, int from_slowness) {
  double sum = 0.0;
  unsigned long long cnt = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    // slowness input: the speed is v = fl(1/s), correctly rounded
    const double v = from_slowness ? __ddiv_rn(1.0, speed[i]) : speed[i];
    const double ri = __ddiv_rn(h, v);
    const double c = __dmul_rn(ri, ri);
    const bool ok = v > 0.0 && bits_of(v) < kInfBits && ri > 0.0 && bits_of(ri) < kInfBits &&
                    c > 0.0 && bits_of(c) < kInfBits;
    if (!ok) raise_status(ctl, kEinval, static_cast<unsigned long long>(i));
    c_out[i] = store_r ? ri : c;
    sum += ri;
    ++cnt;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(kFull, sum, o);
    cnt += __shfl_xor_sync(kFull, cnt, o);
  }
  if ((threadIdx.x & 31) == 0 && cnt) {
    atomicAdd(&ctl->rsum, sum);
    atomicAdd(&ctl->rcount, cnt);
  }
}

// Sum of k arrays in a fixed order (the cross-source gradient of a
// tomography batch): starting from +0, src[0], src[1], ... are added one
// after the other, each addition rounded to nearest.  Streams k + 1 arrays:
// 8 (k + 1) bytes per element, HBM-bound.
__global__ void sum_ordered_kernel(const double *const *__restrict__ src, int k,
                                   double *__restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = __dadd_rn(acc, __ldcs(src[j] + i));
    dst[i] = acc;
  }
}

__global__ void init_t_kernel(double *__restrict__ t, int64_t n) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    t[i] = from_bits(kInfBits);
  }
}

__device__ __forceinline__ unsigned long long tile_of(const Prob &P, int64_t x, int64_t y, int64_t z,
                                                      int tx_, int ty_, int tz_) {
  return static_cast<unsigned long long>(P.tile_base +
                                         ((z / tz_) * P.nty + (y / ty_)) * P.ntx + (x / tx_));
}

// Boundary nodes: t := t0 and activate, with every cell to be evaluated, the
// tile of the source and the tiles of its in-grid neighbours.
__global__ void seed_kernel(SolveParams p, const SeedItem *__restrict__ items, int64_t n,
                            double k_delta, double delta_fixed, int tx_, int ty_, int tz_) {
  Ctl *ctl = p.ctl;
  double delta = delta_fixed > 0.0 ? delta_fixed
                                   : k_delta * (ctl->rsum / static_cast<double>(ctl->rcount));
  if (!(delta > 0.0) || !(bits_of(delta) < kInfBits)) delta = 1.0;
  const double inv = 1.0 / delta;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->delta = delta;
    ctl->inv_delta = inv;
  }
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const SeedItem it = items[i];
    const Prob &P = p.probs[it.prob];
    P.t[it.idx] = it.t0;
    const int64_t x = it.idx % P.nx, yz = it.idx / P.nx;
    const int64_t y = yz % P.ny, z = yz / P.ny;
    const unsigned long long own = tile_of(P, x, y, z, tx_, ty_, tz_);
    p.tile_src[own] = 1;
    const unsigned b = bucket_of_time(bits_of(it.t0), static_cast<float>(inv));
    activate(p, own, 1u << kFaceFull, b);
    const int64_t c3[3] = {x, y, z};
    const int64_t n3[3] = {P.nx, P.ny, P.nz};
    for (int k = 0; k < 3; ++k) {
      for (int side = 0; side < 2; ++side) {
        int64_t q[3] = {c3[0], c3[1], c3[2]};
        q[k] += side ? 1 : -1;
        if (q[k] < 0 || q[k] >= n3[k]) continue;
        const unsigned long long nt = tile_of(P, q[0], q[1], q[2], tx_, ty_, tz_);
        if (nt != own) activate(p, nt, 1u << kFaceFull, b);
      }
    }
  }
}

// Capacity retry: every tile holding a finite value is re-queued with a full
// evaluation (Theorem 1: any state reached by valid updates is a valid start).
__global__ void reseed_kernel(SolveParams p, int tx_, int ty_, int tz_, int64_t total_tiles) {
  const float inv = static_cast<float>(p.ctl->inv_delta);
  for (int64_t g = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; g < total_tiles;
       g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int pi = find_prob(p, static_cast<unsigned long long>(g));
    const Prob &P = p.probs[pi];
    const int64_t lt = g - P.tile_base;
    const int64_t tx = lt % P.ntx, rest = lt / P.ntx;
    const int64_t ty = rest % P.nty, tz = rest / P.nty;
    // the tile and its one-cell halo: a tile that is still all +inf but borders a
    // finite cell may have lost the activation its neighbour pushed when the
    // frontier overflowed, so it is activated too
    unsigned long long best = kInfBits;
    const int64_t z0 = tz * tz_ > 0 ? tz * tz_ - 1 : 0, z1 = (tz + 1) * tz_ + 1 < P.nz ? (tz + 1) * tz_ + 1 : P.nz;
    const int64_t y0 = ty * ty_ > 0 ? ty * ty_ - 1 : 0, y1 = (ty + 1) * ty_ + 1 < P.ny ? (ty + 1) * ty_ + 1 : P.ny;
    const int64_t x0 = tx * tx_ > 0 ? tx * tx_ - 1 : 0, x1 = (tx + 1) * tx_ + 1 < P.nx ? (tx + 1) * tx_ + 1 : P.nx;
    for (int64_t z = z0; z < z1; ++z)
      for (int64_t y = y0; y < y1; ++y)
        for (int64_t x = x0; x < x1; ++x)
          best = umin64(best, bits_of(ld_time(P.t + (z * P.ny + y) * P.nx + x)));
    if (best < kInfBits) activate(p, static_cast<unsigned long long>(g), 1u << kFaceFull,
                                  bucket_of_time(best, inv));
  }
}

// Batched forms: blockIdx.y selects the problem (first + y), blockIdx.x strides
// over its cells.
__global__ void init_t_all_kernel(const Prob *__restrict__ probs, int first) {
  const Prob &P = probs[first + blockIdx.y];
  const int64_t n = P.nx * P.ny * P.nz;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    P.t[i] = from_bits(kInfBits);
  }
}

__global__ void count_finite_all_kernel(const Prob *__restrict__ probs, int first,
                                        unsigned long long *out) {
  const Prob &P = probs[first + blockIdx.y];
  const int64_t n = P.nx * P.ny * P.nz;
  unsigned long long cnt = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    cnt += bits_of(P.t[i]) < kInfBits ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

// Order-dependent 64-bit digest of every problem's times (sum of bit patterns
// times odd per-cell multipliers, and an xor of mixed patterns): equal
// digests of two solves of the same batch mean identical bits, short of a
// collision.
__global__ void checksum_all_kernel(const Prob *__restrict__ probs, int first,
                                    unsigned long long *out) {
  const int pi = first + static_cast<int>(blockIdx.y);
  const Prob &P = probs[pi];
  const int64_t n = P.nx * P.ny * P.nz;
  unsigned long long sum = 0, x = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const unsigned long long b = bits_of(P.t[i]);
    const unsigned long long k = (static_cast<unsigned long long>(pi) << 40) ^ static_cast<unsigned long long>(i);
    sum += b * (2ull * k + 1ull);
    x ^= (b + 0x9e3779b97f4a7c15ull * (k + 1ull)) * 0xbf58476d1ce4e5b9ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_xor_sync(kFull, sum, o);
    x ^= __shfl_xor_sync(kFull, x, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, sum);
    atomicXor(out + 1, x);
  }
}

__global__ void count_finite_kernel(const double *__restrict__ t, int64_t n,
                                    unsigned long long *out) {
  unsigned long long cnt = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    cnt += bits_of(t[i]) < kInfBits ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

std::atomic<unsigned long long> g_launches{0};

int grid_for(int64_t n, int per_sm) {
  int64_t g = (n + 255) / 256;
  const int64_t cap = static_cast<int64_t>(num_sms()) * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

}  // namespace

void note_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long kernel_launches() { return g_launches.load(std::memory_order_relaxed); }

cudaError_t launch_init_c(const double *speed, double h, double *c, int64_t n, Ctl *ctl,
                          cudaStream_t stream, int store_r, int from_slowness) {
  if (n <= 0) return cudaSuccess;
  init_c_kernel<<<grid_for(n, 8), 256, 0, stream>>>(speed, h, c, n, ctl, store_r, from_slowness);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_sum_ordered(const double *const *src, int k, double *dst, int64_t n,
                               cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  sum_ordered_kernel<<<grid_for(n, 8), 256, 0, stream>>>(src, k, dst, n);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_init_t(double *t, int64_t n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  init_t_kernel<<<grid_for(n, 8), 256, 0, stream>>>(t, n);
  note_launches(1);
  return cudaGetLastError();
}

// blocks per problem for the batched element-wise kernels: about 8 per SM in
// total, at least one per problem
static int per_prob_blocks(int nprob, int64_t max_cells) {
  int64_t g = (max_cells + 255) / 256;
  const int64_t share = (static_cast<int64_t>(num_sms()) * 8 + nprob - 1) / nprob;
  if (g > share) g = share;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

cudaError_t launch_init_t_all(const Prob *dev_probs, int nprob, int64_t max_cells,
                              cudaStream_t stream) {
  if (nprob <= 0 || max_cells <= 0) return cudaSuccess;
  const int gx = per_prob_blocks(nprob, max_cells);
  for (int first = 0; first < nprob; first += 65535) {
    const int ny = nprob - first < 65535 ? nprob - first : 65535;
    init_t_all_kernel<<<dim3(gx, ny), 256, 0, stream>>>(dev_probs, first);
    note_launches(1);
  }
  return cudaGetLastError();
}

// Item y of the copy list, chunks of 16 bytes where both ends are 16-byte
// aligned (else 8); blocks of one item stride over it.
__global__ void copy_items_kernel(const CopyItem *__restrict__ items, int first) {
  const CopyItem it = items[first + blockIdx.y];
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  const bool wide = ((reinterpret_cast<uintptr_t>(it.src) | reinterpret_cast<uintptr_t>(it.dst)) & 15u) == 0u;
  if (wide) {
    const int64_t n2 = it.n >> 1;
    const double2 *s2 = reinterpret_cast<const double2 *>(it.src);
    double2 *d2 = reinterpret_cast<double2 *>(it.dst);
    for (int64_t k = i; k < n2; k += stride) d2[k] = s2[k];
    if ((it.n & 1) && i == 0) it.dst[it.n - 1] = it.src[it.n - 1];
  } else {
    for (int64_t k = i; k < it.n; k += stride) it.dst[k] = it.src[k];
  }
}

cudaError_t launch_copy_items(const CopyItem *items, int nitems, int64_t max_n, cudaStream_t stream) {
  if (nitems <= 0 || max_n <= 0) return cudaSuccess;
  const int gx = per_prob_blocks(nitems, (max_n + 1) / 2);
  for (int first = 0; first < nitems; first += 65535) {
    const int ny = nitems - first < 65535 ? nitems - first : 65535;
    copy_items_kernel<<<dim3(gx, ny), 256, 0, stream>>>(items, first);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_checksum_all(const Prob *dev_probs, int nprob, int64_t max_cells,
                               unsigned long long *out, cudaStream_t stream) {
  if (nprob <= 0 || max_cells <= 0) return cudaSuccess;
  const int gx = per_prob_blocks(nprob, max_cells);
  for (int first = 0; first < nprob; first += 65535) {
    const int ny = nprob - first < 65535 ? nprob - first : 65535;
    checksum_all_kernel<<<dim3(gx, ny), 256, 0, stream>>>(dev_probs, first, out);
    note_launches(1);
  }
  return cudaGetLastError();
}

cudaError_t launch_count_finite_all(const Prob *dev_probs, int nprob, int64_t max_cells,
                                    unsigned long long *out, cudaStream_t stream) {
  if (nprob <= 0 || max_cells <= 0) return cudaSuccess;
  const int gx = per_prob_blocks(nprob, max_cells);
  for (int first = 0; first < nprob; first += 65535) {
    const int ny = nprob - first < 65535 ? nprob - first : 65535;
    count_finite_all_kernel<<<dim3(gx, ny), 256, 0, stream>>>(dev_probs, first, out);
    note_launches(1);
  }
  return cudaGetLastError();
}

static void tile_dims(const SolveParams &p, int &tx, int &ty, int &tz) {
  const TileShape ts = tile_shape_of(p.ndim, p.tile_shape);
  tx = ts.tx;
  ty = ts.ty;
  tz = ts.tz;
}

cudaError_t launch_seed(const SolveParams &p, const SeedItem *items, int64_t nitems,
                        double k_delta, double delta_fixed, cudaStream_t stream) {
  int tx, ty, tz;
  tile_dims(p, tx, ty, tz);
  const int grid = grid_for(nitems > 0 ? nitems : 1, 4);
  seed_kernel<<<grid, 256, 0, stream>>>(p, items, nitems, k_delta, delta_fixed, tx, ty, tz);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_reseed(const SolveParams &p, const Prob *host_probs, int nprob,
                          cudaStream_t stream) {
  int tx, ty, tz;
  tile_dims(p, tx, ty, tz);
  const Prob &last = host_probs[nprob - 1];
  const int64_t total = last.tile_base + last.ntx * last.nty * last.ntz;
  reseed_kernel<<<grid_for(total, 4), 256, 0, stream>>>(p, tx, ty, tz, total);
  note_launches(1);
  return cudaGetLastError();
}

// Launch / occupancy per (dimension, shape, arithmetic).  The integer-pipe
// arithmetic exists for the default shapes only.
bool persistent_launch_is_lean(const SolveParams &p) {
  return p.arith != kArithInt && p.counters == 0 && p.update == 0 && !p.track_changes &&
         p.lane_group_cells == 0 && p.trace == nullptr && p.visit_budget == 0ull;
}

template <int D, int TX, int TY, int TZ, bool WithInt, bool Wide = false>
struct ShapeOps {
  static int wide_blocks_per_sm(int arith) {
    int nb = 0;
    if constexpr (Wide) {
      if (arith == kArithFp64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, persistent_kernel<D, TX, TY, TZ, kArithFp64, true, true>, TX * TY * TZ, 0);
    }
    return nb;
  }
  static int blocks_per_sm(int arith) {
    int nb = 0;
    if constexpr (WithInt) {
      if (arith == kArithInt) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, persistent_kernel<D, TX, TY, TZ, kArithInt, false>, TX * TY * TZ, 0);
        return nb;
      }
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &nb, persistent_kernel<D, TX, TY, TZ, kArithFp64, false>, TX * TY * TZ, 0);
    return nb;
  }
  static cudaError_t launch(const SolveParams &p, int grid, cudaStream_t stream) {
    if (p.arith == kArithInt) {
      if constexpr (WithInt) {
        persistent_kernel<D, TX, TY, TZ, kArithInt, false><<<grid, TX * TY * TZ, 0, stream>>>(p);
        return cudaGetLastError();
      } else {
        return cudaErrorInvalidValue;
      }
    }
    if (persistent_launch_is_lean(p)) {
      if constexpr (Wide) {
        if (p.wide) {
          persistent_kernel<D, TX, TY, TZ, kArithFp64, true, true><<<grid, TX * TY * TZ, 0, stream>>>(p);
          return cudaGetLastError();
        }
      }
      persistent_kernel<D, TX, TY, TZ, kArithFp64, true><<<grid, TX * TY * TZ, 0, stream>>>(p);
    } else
      persistent_kernel<D, TX, TY, TZ, kArithFp64, false><<<grid, TX * TY * TZ, 0, stream>>>(p);
    return cudaGetLastError();
  }
};

#define EIK_SHAPE_SWITCH(ndim, shape, CALL)                                   \
  do {                                                                       \
    if ((ndim) == 3) {                                                       \
      switch (shape) {                                                       \
        case 1: { using S = ShapeOps<3, 16, 4, 4, false>; CALL; } break;     \
        case 2: { using S = ShapeOps<3, 32, 4, 2, false>; CALL; } break;     \
        case 3: { using S = ShapeOps<3, 8, 4, 4, false>; CALL; } break;      \
        case 4: { using S = ShapeOps<3, 4, 4, 4, false, true>; CALL; } break; \
        default: { using S = ShapeOps<3, kTX3, kTY3, kTZ3, true>; CALL; }    \
      }                                                                      \
    } else {                                                                 \
      switch (shape) {                                                       \
        case 1: { using S = ShapeOps<2, 32, 8, 1, false>; CALL; } break;     \
        case 2: { using S = ShapeOps<2, 32, 4, 1, false>; CALL; } break;     \
        case 3: { using S = ShapeOps<2, 16, 8, 1, false>; CALL; } break;     \
        case 4: { using S = ShapeOps<2, 16, 4, 1, false>; CALL; } break;     \
        default: { using S = ShapeOps<2, kTX2, kTY2, 1, true>; CALL; }       \
      }                                                                      \
    }                                                                        \
  } while (0)

int persistent_blocks_per_sm(int ndim, int arith, int tile_shape) {
  int nb = 0;
  EIK_SHAPE_SWITCH(ndim, tile_shape, nb = S::blocks_per_sm(arith));
  return nb > 0 ? nb : 1;
}

int persistent_wide_blocks_per_sm(int ndim, int arith, int tile_shape) {
  int nb = 0;
  EIK_SHAPE_SWITCH(ndim, tile_shape, nb = S::wide_blocks_per_sm(arith));
  return nb > 0 ? nb : 0;
}

cudaError_t launch_persistent(const SolveParams &p, int grid, cudaStream_t stream) {
  cudaError_t e = cudaSuccess;
  EIK_SHAPE_SWITCH(p.ndim, p.tile_shape, e = S::launch(p, grid, stream));
  note_launches(1);
  return e;
}

cudaError_t launch_count_finite(const Prob *host_probs, int nprob, unsigned long long *out,
                                cudaStream_t stream) {
  for (int i = 0; i < nprob; ++i) {
    const Prob &P = host_probs[i];
    const int64_t n = P.nx * P.ny * P.nz;
    count_finite_kernel<<<grid_for(n, 8), 256, 0, stream>>>(P.t, n, out);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace eik
