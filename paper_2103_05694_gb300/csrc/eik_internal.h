// Internal declarations shared by the CUDA translation units of the Eikonal
// solver (kernels in eik_solver.cu, host API in eik_api.cu).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

namespace eik {

// The process-wide lock that serialises the C ABI's calls, and the message
// returned by eik_last_error (both owned by eik_api.cu).
std::mutex &api_mutex();
void set_last_error(const char *fmt, ...);

// Bucket ring: NB slots; bucket b lives in slot b & (NB - 1).  Each slot is a
// ring of `cap` 64-bit entries (cap a power of two) with one sequence word per
// position.  For the entry of index i (position i & (cap - 1)) the word reads
// i & ~(cap - 1) while the position is free for it and that + 1 once the entry
// is written; the entry's taker moves it on by cap (free for the next lap).
// Sequence words are zero before every solve.
constexpr uint32_t kNumSlots = 128;
constexpr uint64_t kEmpty = ~0ull;
constexpr uint32_t kMaxBucket = (1u << 30) - 1;
constexpr int kCounterPad = 16;          // u32 counters padded to 64 bytes

// Tile state word: bits 0..29 bucket, bits 32..38 face mask, bits 40..41 status.
constexpr uint64_t kStIdle = 0, kStQueued = 1, kStRunning = 2, kStDirty = 3;
constexpr int kFaceFull = 6;             // face bit 6: evaluate every cell

// Device status codes (match eik_status).
constexpr unsigned kOk = 0, kEinval = 1, kEcapacity = 3, kEtimeout = 4;

enum StatIdx {
  kStatEvals = 0, kStatDecreases, kStatVisits, kStatPushes, kStatStale, kStatRounds,
  kStatCommits, kStatMaxQueue, kStatVisitNs, kStatIdleNs,
  // detailed timing (counters >= 2): cycles of thread 0 per phase, d-bar paths
  kStatCycLoad, kStatCycA, kStatCycB, kStatCycC, kStatCycCommit,
  kStatNewton, kStatWalk, kStatBisect, kStatDbarCalls, kNumStats
};

// Control block, zeroed before every solve.
struct Ctl {
  int work;                 // frontier entries pushed and not yet finished
  int pad0[31];
  unsigned cur;             // hint: lowest bucket that may be non-empty
  int pad1[31];
  unsigned status;          // first error (0 = ok)
  unsigned done;            // termination detected
  unsigned never_set;       // stays 0: the stall test waits on it
  int pad2[29];
  double rsum;              // sum of r = h/v over all cells (auto bucket width)
  unsigned long long rcount;
  double delta;             // bucket width used
  double inv_delta;
  unsigned long long rmin_bits;   // smallest r (bit pattern; all r > 0)
  int pad3[22];
  unsigned long long stats[kNumStats];
  unsigned long long error_info[4];   // where a wait gave up / what was invalid
  unsigned long long trace_n;         // trace records written (may exceed the capacity)
  unsigned push[kNumSlots * kCounterPad];
  unsigned pop[kNumSlots * kCounterPad];
  unsigned run[kNumSlots * kCounterPad];   // tiles claimed from the slot and still running
  int avail[kNumSlots * kCounterPad];      // entries written and not yet reserved by a popper
                                           // (may dip below 0 while a failed reservation
                                           // is being undone)
  unsigned long long visits_total;         // tile visits claimed (checked against visit_budget)
};

// One grid of a (possibly batched) solve, as the kernels see it.
struct Prob {
  double *t;                // arrival times (working field and result)
  const double *c;          // per cell c = fl(fl(h / v)^2)
  const int64_t *src_idx;   // sorted unique source indices (device)
  const double *src_t;      // their times (device), same order
  int64_t nsrc;
  int64_t nx, ny, nz;       // extents (nz = 1 in 2D)
  int64_t ntx, nty, ntz;    // tiles per axis
  int64_t tile_base;        // first global tile id of this problem
};

struct SolveParams {
  const Prob *probs;
  int nprob;
  int ndim;
  unsigned long long *state;      // per global tile
  unsigned char *tile_src;        // per global tile: 1 if it holds a source
  unsigned *pend;                 // per global tile, kPendWords words: cells deferred by
                                  // the last visit (to evaluate at the next one)
  unsigned long long *slots;      // kNumSlots * cap
  unsigned *seq;                  // kNumSlots * cap sequence words (see the bucket ring)
  unsigned cap_mask;              // cap - 1
  Ctl *ctl;
  long long timeout_ns;
  int counters;
  int test_stall;
  unsigned window;                // buckets above the lowest active one that may be popped
  double band;                    // in-tile acceptance band, in units of min r / sqrt(D)
  int arith;                      // kArithFp64 or kArithInt
  int gate_pending_only;          // window follows pending entries only, not running tiles
  int tile_shape;                 // index into tile_shape_of (0: default)
  int update;                     // 0: d-bar; 2D ablation: 1 = d-tilde, 2 = d-hat, 3 = d-hat
                                  // then Newton (c holds r)
  unsigned long long visit_budget;  // 0: none; else the solve stops with EIK_ETIMEOUT after
                                    // this many tile visits (change tracking, which may not
                                    // terminate, runs with one)
  int track_changes;              // explicit forms only: a cell whose recomputed value differs
                                  // from its value (up or down) takes it and re-activates its
                                  // neighbours (the paper's conservative work tracking)
  int lane_group_cells;           // lists of at most this many cells use lane groups (0: never)
  struct TraceRec *trace;         // optional visit trace (device), NULL when off
  unsigned long long trace_cap;
  int wide;                       // lean launches of 4x4x4 3D tiles: the build compiled for
                                  // EIK_WIDE_CTAS_64 CTAs per SM (fewer registers)
};

// One tile visit, for timeline analysis (opts.trace).
struct TraceRec {
  long long t_claim, t_end;       // %globaltimer ns
  unsigned tile, lo, rounds, flags;   // flags: bit 0 deferred cells, bits 8.. CTA index
};

constexpr int kPendWords = 8;            // pending-mask words per tile (up to 256 cells)
constexpr int kArithFp64 = 1, kArithInt = 2;   // d-bar on the FP64 unit / on the integer pipes

// Tile shapes (cells): one thread per cell.  Shape 0 of each dimension is the
// default; the others are alternatives (opts.tile) for the autotuner.
constexpr int kTX2 = 16, kTY2 = 16;                // 2D default
constexpr int kTX3 = 8, kTY3 = 8, kTZ3 = 4;        // 3D default
constexpr int kNumTileShapes = 5;
// Resident CTAs per SM that the register budget of the persistent kernel
// allows, by tile size (launch bounds; the solve is latency-bound per CTA, so
// small tiles run many CTAs per SM).
#ifndef EIK_MIN_CTAS_256
#define EIK_MIN_CTAS_256 2
#endif
#ifndef EIK_MIN_CTAS_128
#define EIK_MIN_CTAS_128 8
#endif
#ifndef EIK_MIN_CTAS_64
#define EIK_MIN_CTAS_64 16
#endif
// The lean 3D 4x4x4 kernel also has a wide build, compiled for more resident
// CTAs per SM with fewer registers: a batch of many fronts keeps them busy.
#ifndef EIK_WIDE_CTAS_64
#define EIK_WIDE_CTAS_64 20
#endif
constexpr int resident_ctas(int tile_cells) {
  return tile_cells >= 256 ? EIK_MIN_CTAS_256 : tile_cells >= 128 ? EIK_MIN_CTAS_128 : EIK_MIN_CTAS_64;
}
struct TileShape {
  int tx, ty, tz;
};
__host__ __device__ inline TileShape tile_shape_of(int ndim, int shape) {
  if (ndim == 3) {
    switch (shape) {
      case 1: return TileShape{16, 4, 4};
      case 2: return TileShape{32, 4, 2};
      case 3: return TileShape{8, 4, 4};
      case 4: return TileShape{4, 4, 4};
      default: return TileShape{kTX3, kTY3, kTZ3};
    }
  }
  switch (shape) {
    case 1: return TileShape{32, 8, 1};
    case 2: return TileShape{32, 4, 1};
    case 3: return TileShape{16, 8, 1};
    case 4: return TileShape{16, 4, 1};
    default: return TileShape{kTX2, kTY2, 1};
  }
}

// Launch wrappers (eik_solver.cu).  All enqueue on `stream`.
// store_r: write r = fl(h/v) instead of c (the explicit update forms use r).
// from_slowness: `speed` holds slowness s, and v = fl(1/s) is used.
cudaError_t launch_init_c(const double *speed, double h, double *c, int64_t n, Ctl *ctl,
                          cudaStream_t stream, int store_r = 0, int from_slowness = 0);
// dst[i] = (((+0 + src[0][i]) + src[1][i]) + ...) + src[k-1][i], every addition
// rounded to nearest in that order (src: device array of k device pointers).
cudaError_t launch_sum_ordered(const double *const *src, int k, double *dst, int64_t n,
                               cudaStream_t stream);
cudaError_t launch_init_t(double *t, int64_t n, cudaStream_t stream);
// t = +inf on every problem of a batch in one launch (dev_probs: device array;
// max_cells: the largest problem's cell count).
cudaError_t launch_init_t_all(const Prob *dev_probs, int nprob, int64_t max_cells,
                              cudaStream_t stream);
// One contiguous copy of n doubles; src and dst are device memory or pinned
// host memory mapped into the device's address space (host <-> device copies
// run as stores and loads of the SMs over the chip-to-chip link, not on the
// copy engines).
struct CopyItem {
  const double *src;
  double *dst;
  int64_t n;
};
// All items in one launch (items: device array of nitems; max_n: the largest n).
cudaError_t launch_copy_items(const CopyItem *items, int nitems, int64_t max_n, cudaStream_t stream);
// One source of one problem, flattened over the batch for the seed kernel.
struct SeedItem {
  int64_t prob;
  int64_t idx;
  double t0;
};

cudaError_t launch_seed(const SolveParams &p, const SeedItem *items, int64_t nitems,
                        double k_delta, double delta_fixed, cudaStream_t stream);
cudaError_t launch_reseed(const SolveParams &p, const Prob *host_probs, int nprob,
                          cudaStream_t stream);
cudaError_t launch_persistent(const SolveParams &p, int grid, cudaStream_t stream);
cudaError_t launch_count_finite(const Prob *host_probs, int nprob, unsigned long long *out,
                                cudaStream_t stream);
// Finite times over every problem of a batch in one launch (adds into *out).
cudaError_t launch_count_finite_all(const Prob *dev_probs, int nprob, int64_t max_cells,
                                    unsigned long long *out, cudaStream_t stream);
// 128-bit digest (out[0] sum, out[1] xor; caller zeroes) of all problems' times.
cudaError_t launch_checksum_all(const Prob *dev_probs, int nprob, int64_t max_cells,
                               unsigned long long *out, cudaStream_t stream);
// Kernels this library has launched (or enqueued into a stream capture) since
// it was loaded; every launch wrapper adds its launches.
void note_launches(unsigned long long n);
unsigned long long kernel_launches();
int persistent_blocks_per_sm(int ndim, int arith, int tile_shape);
// Resident CTAs per SM of the shape's wide lean build; 0 when it has none.
int persistent_wide_blocks_per_sm(int ndim, int arith, int tile_shape);
// Whether launch_persistent runs the lean instantiation for these parameters.
bool persistent_launch_is_lean(const SolveParams &p);

// Other schedules of the same update (eik_schedules.cu): opts.schedule.
constexpr int kScheduleAmm = 0, kScheduleFim = 1, kScheduleTopo = 2, kScheduleFsm = 3;

struct BspCtl {
  unsigned long long nfront[3];   // worklist sizes (FIM) / changes per iteration (topology, FSM)
  unsigned long long pad0[13];
  unsigned bar_count, bar_gen;
  unsigned pad1[30];
  unsigned long long evals, decreases, rounds;
  unsigned status;
};

struct BspParams {
  double *t;
  const double *c;                // c = fl(fl(h/v)^2)
  int ndim;
  int64_t nx, ny, nz;
  unsigned char *fixed;           // 1 at source cells
  unsigned *mark[2];              // round stamps: w_r is mark[r & 1] == r
  unsigned long long *front[2];   // worklists of consecutive rounds
  BspCtl *ctl;
  long long timeout_ns;
};

cudaError_t launch_bsp_seed(const BspParams &p, const int64_t *src_idx, const double *src_t,
                            int64_t nsrc, cudaStream_t stream);
cudaError_t launch_schedule(int schedule, BspParams p, cudaStream_t stream);

// Update-form ablation (eik_ablation.cu): Algorithm 1 / d-bar at n points, and
// the Table 3 residual of one field (out[0] += count, out[1] = max bits).
cudaError_t launch_eval_update(int form, const double *speed, double h, const double *t_h,
                               const double *t_v, int64_t n, double *out, cudaStream_t stream);
cudaError_t launch_residual(int form, int ndim, const double *speed, double h, const double *t,
                            int64_t nx, int64_t ny, int64_t nz, const int64_t *src_idx,
                            const double *src_t, int64_t nsrc, unsigned long long *out,
                            cudaStream_t stream);

// Adjoint (eik_adjoint.cu).
struct AdjProb {
  const double *t;          // forward arrival times (the exact fixed point)
  const double *v;          // speed (slowness s when v_is_slowness: v = fl(1/s))
  int v_is_slowness;
  const double *g;          // dL/dt (NULL: 0)
  double *grad;             // dL/ds output
  double *lam;              // adjoint variable (workspace; NULL in the tile schedule)
  double *W[3];             // per axis: weight of the axis' upwind side(s) (workspace); in
                            // the tile schedule lambda * weight once the cell is processed
  unsigned char *mask;      // upwind sides (bit 2k + side) of each cell (workspace)
  int *cnt;                 // downwind users not yet processed (workspace); with tiles:
                            // the users inside the cell's own tile
  int *cnt_out;             // with tiles: the users in other tiles (workspace)
  unsigned char *status;    // with tiles: 0 unreached, 1 pending, 2 processed (workspace)
  const int64_t *src_idx;   // sorted unique sources
  int64_t nsrc;
  int64_t nx, ny, nz;
  int ndim;
  int64_t base;             // first global cell index of this problem
  double hh;                // fl(h * h)
  int64_t ntx, nty, ntz;    // tiles per axis (tile schedule)
  int64_t tile_base;        // first global tile index of this problem
};

// Control block of the adjoint.  Level-synchronous schedule: frontier counts
// rotate over three slots: level L reads slot L % 3, appends to (L + 1) % 3 and
// clears (L + 2) % 3.  Tile schedule: queue counters and visit statistics.
struct AdjCtl {
  unsigned long long reached;        // cells with a finite time
  unsigned long long pad0[15];
  unsigned long long done;           // cells processed
  unsigned long long pad1[15];
  unsigned long long nfront[3];
  unsigned long long pad2[13];
  unsigned bar_count;                // grid barrier: arrivals and generation
  unsigned bar_gen;
  unsigned pad3[30];
  unsigned long long levels;
  unsigned status;
  unsigned pad4[13];
  unsigned long long head;           // tile schedule: queue tickets taken and pushed
  unsigned long long pad5[15];
  unsigned long long tail;
  unsigned long long pad6[15];
  unsigned long long visits;         // tile visits
  unsigned long long rounds;         // rounds summed over tile visits
  unsigned long long visit_ns;       // visit time summed over CTAs
  unsigned long long idle_ns;        // time CTAs spent waiting for a tile
  unsigned long long ctas;           // persistent CTAs of the tile launch
  unsigned long long cycles[4];      // SM cycles of thread 0 per CTA: waiting for a tile,
                                     // visit loads, rounds, stores and releases
};

// set-up (masks, weights, coefficients, counts), first frontier, and one
// cooperative persistent launch over the frontiers.  `front` holds 2 * total
// entries.
cudaError_t launch_adjoint(const AdjProb *probs_dev, int nprob, int64_t total, AdjCtl *ctl,
                           unsigned long long *front, long long timeout_ns, cudaStream_t stream);
// The tile schedule: set-up with counts split by tile, the initial queue, and a
// persistent launch that relaxes ready tiles in shared memory.  tile_state
// holds total_tiles words, zero on entry; queue holds qcap slots (a power of two
// >= total_tiles, set up by the launch).  ndim: of every problem (one tile shape
// per launch).  The tiles are kAdjTile2 in 2D and kAdjTile3 in 3D.  ctas_per_sm
// caps the persistent CTAs per SM (0: occupancy).
// 2D adjoint tile (compile-time): 16x8 cells, 8 resident CTAs of 128 threads per SM
// (32-source tomography adjoint 11.6 ms, against 12.9 ms with 16x16 tiles at 4
// CTAs per SM, 14.0 with 32x8 and 15.7 with 32x16)
#ifndef EIK_ADJ_TILE2_X
#define EIK_ADJ_TILE2_X 16
#endif
#ifndef EIK_ADJ_TILE2_Y
#define EIK_ADJ_TILE2_Y 8
#endif
constexpr int kAdjTile2[3] = {EIK_ADJ_TILE2_X, EIK_ADJ_TILE2_Y, 1};
constexpr int kAdjTile3[3] = {8, 8, 4};
// timing: collect the visit and wait clocks (eik_stats timing fields).
cudaError_t launch_adjoint_tiles(const AdjProb *probs_dev, int nprob, int64_t total,
                                 int64_t total_tiles, int ndim, AdjCtl *ctl, unsigned *tile_state,
                                 unsigned long long *queue, unsigned long long qcap,
                                 int ctas_per_sm, long long timeout_ns, bool timing,
                                 cudaStream_t stream);

}  // namespace eik
