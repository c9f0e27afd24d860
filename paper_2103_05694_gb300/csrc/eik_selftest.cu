// Self-test of the integer-pipe exact arithmetic (eik_exact.cuh) against the
// hardware FP64 unit, bit for bit, on random and tie-heavy inputs generated on
// the device from a counter-based hash (splitmix64 of seed and index).
//
// Checked: fl(x - y), fl(m * m), fl(x + y), G(tau) in 2D and 3D, and d-bar in
// 2D and 3D, where the reference d-bar is the plain definition: bisection over
// bit patterns for the smallest tau with G_hw(tau) >= c, G_hw built from
// __dsub_rn / __dmul_rn / __dadd_rn.
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "../../include/eik.h"
#include "eik_exact.cuh"
#include "eik_internal.h"

namespace eik {
namespace {

using xf::as_d;
using xf::as_u;
using xf::kInf;

__device__ __forceinline__ unsigned long long mix(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

template <int D>
__device__ unsigned long long G_hw(unsigned long long tau, const unsigned long long (&a)[D]) {
  double g = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double m = __dsub_rn(as_d(tau), as_d(a[k]));
    if (!(m > 0.0)) m = 0.0;
    g = k == 0 ? __dmul_rn(m, m) : __dadd_rn(g, __dmul_rn(m, m));
  }
  return as_u(g);
}

template <int D>
__device__ unsigned long long dbar_ref(const unsigned long long (&a)[D], unsigned long long cb) {
  unsigned long long amin = a[0];
  for (int k = 1; k < D; ++k) amin = amin < a[k] ? amin : a[k];
  if (amin >= kInf) return kInf;
  unsigned long long lo = amin;
  unsigned long long hi = as_u(__dadd_rn(as_d(amin), __dmul_rn(2.0, sqrt(as_d(cb)))));
  if (hi <= lo) hi = lo + 1ull;
  for (int it = 0; it < 64 && G_hw<D>(hi, a) < cb; ++it) {
    lo = hi;
    hi = hi + (hi - amin);
    if (hi > kInf) hi = kInf;
  }
  while (hi - lo > 1ull) {
    const unsigned long long mid = lo + (hi - lo) / 2ull;
    if (G_hw<D>(mid, a) >= cb) hi = mid; else lo = mid;
  }
  return hi;
}

__device__ unsigned long long rand_double(unsigned long long h, int emin, int erange) {
  const unsigned long long e = static_cast<unsigned long long>(emin + static_cast<int>((h >> 52) % erange));
  unsigned long long m = h & xf::kFrac;
  const unsigned sel = static_cast<unsigned>((h >> 40) & 7u);
  if (sel == 0) m &= ~((1ull << ((h >> 32) % 53)) - 1ull);   // few low bits: more exact ties
  if (sel == 1) m = 0ull;
  return (e << 52) | m;
}

// The lane-group update of one cell (all L lanes take the cell of the group's
// first lane) against the reference: decrease iff d-bar < best, value d-bar.
template <int D, int L>
__device__ bool group_ok(const unsigned long long (&a_in)[D], unsigned long long cb_in,
                         unsigned long long h) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lead = lane & ~(L - 1u);
  unsigned long long a[D];
#pragma unroll
  for (int k = 0; k < D; ++k) a[k] = __shfl_sync(0xffffffffu, a_in[k], lead);
  const unsigned long long cb = __shfl_sync(0xffffffffu, cb_in, lead);
  const unsigned long long ref = dbar_ref<D>(a, cb);
  const unsigned long long hh = __shfl_sync(0xffffffffu, h, lead);
  unsigned long long best;
  switch (hh & 3u) {
    case 0: best = kInf; break;
    case 1: best = ref; break;
    case 2: best = ref + 1ull + ((hh >> 8) % 100u); break;
    default: best = ref > 2ull ? ref - 1ull - ((hh >> 8) % 2u) : ref; break;
  }
  unsigned long long out = 0;
  const bool dec = hw::relax_group<D, L>(best, a, cb, true, out);
  const bool want = ref < best;
  return dec == want && (!dec || out == ref);
}

// counters: 0 sub, 1 sq, 2 add, 3 G2, 4 G3, 5 dbar2, 6 dbar3, 7 group 2D x8,
// 8 group 3D x8, 9 group 2D x4, 10 FP64-unit dbar 2D, 11 3D; [15] trials;
// [16 + k] first failing trial of check k
__global__ void selftest_kernel(int64_t n, unsigned long long seed, unsigned long long *bad,
                                unsigned long long *first) {
  // whole warps iterate together (the lane-group checks use warp collectives)
  const int64_t span = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t base = blockIdx.x * static_cast<int64_t>(blockDim.x); base < n; base += span) {
    const int64_t i = base + threadIdx.x;
    const bool live = i < n;
    const unsigned long long h0 = mix(seed ^ mix(static_cast<unsigned long long>(i)));
    const unsigned long long h1 = mix(h0), h2 = mix(h1), h3 = mix(h2), h4 = mix(h3), h5 = mix(h4);
    unsigned long long nb[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    // sub and add: x >= y > 0 with exponent gaps 0..70
    {
      unsigned long long x = rand_double(h1, 900, 250);
      const int d = static_cast<int>((h2 >> 58) < 48 ? (h2 >> 58) % 12 : (h2 >> 50) % 70);
      int ey = static_cast<int>(x >> 52) - d;
      if (ey < 1) ey = 1;
      unsigned long long y = (static_cast<unsigned long long>(ey) << 52) | (h3 & xf::kFrac);
      if ((h3 >> 60) == 0) y = (y & ~xf::kFrac) | (x & xf::kFrac);
      if ((h3 >> 58) == 1) y &= ~((1ull << ((h3 >> 20) % 53)) - 1ull);
      if (y > x) { const unsigned long long t = x; x = y; y = t; }
      if (x == y) x += 1ull;
      if (xf::sub_pos(x, y) != as_u(__dsub_rn(as_d(x), as_d(y)))) nb[0] = 1;
      if (xf::add_pos(x, y) != as_u(__dadd_rn(as_d(x), as_d(y)))) nb[2] = 1;
      if (xf::add_pos(y, x) != as_u(__dadd_rn(as_d(y), as_d(x)))) nb[2] = 1;
    }
    {
      const unsigned long long m = rand_double(h4, 700, 650);
      if (xf::sq(m) != as_u(__dmul_rn(as_d(m), as_d(m)))) nb[1] = 1;
    }
    // G and d-bar on minima near a common arrival time
    {
      const double a0 = as_d(rand_double(h5, 1000, 40));
      const double r = as_d(rand_double(mix(h5 ^ 1), 1000, 24)) * 1e-3;
      const unsigned long long cb = as_u(__dmul_rn(r, r));
      unsigned long long a3[3];
      unsigned long long hh = mix(h5 ^ 2);
      for (int k = 0; k < 3; ++k) {
        hh = mix(hh);
        const double u = static_cast<double>(hh >> 11) * 0x1.0p-53 * 1.6 * r;
        a3[k] = (hh & 7u) == 0 ? kInf : as_u(__dadd_rn(a0, u));
      }
      if (a3[0] == kInf && a3[1] == kInf && a3[2] == kInf) a3[0] = as_u(a0);
      const unsigned long long a2[2] = {a3[0] == kInf && a3[1] == kInf ? as_u(a0) : a3[0], a3[1]};
      hh = mix(hh);
      const unsigned long long tau =
          as_u(__dadd_rn(a0, static_cast<double>(hh >> 11) * 0x1.0p-53 * 2.0 * r));
      if (xf::G<2>(tau, a2) != G_hw<2>(tau, a2)) nb[3] = 1;
      if (xf::G<3>(tau, a3) != G_hw<3>(tau, a3)) nb[4] = 1;
      if (xf::dbar<2>(a2, cb) != dbar_ref<2>(a2, cb)) nb[5] = 1;
      if (xf::dbar<3>(a3, cb) != dbar_ref<3>(a3, cb)) nb[6] = 1;
      if (hw::dbar<2>(a2, cb) != dbar_ref<2>(a2, cb)) nb[10] = 1;
      if (hw::dbar<3>(a3, cb) != dbar_ref<3>(a3, cb)) nb[11] = 1;
      const unsigned long long hg = mix(h5 ^ 3);
      if (!group_ok<2, 8>(a2, cb, hg)) nb[7] = 1;
      if (!group_ok<3, 8>(a3, cb, hg)) nb[8] = 1;
      if (!group_ok<2, 4>(a2, cb, hg ^ 1)) nb[9] = 1;
    }
    for (int k = 0; k < 12; ++k) {
      if (live && nb[k]) {
        atomicAdd(&bad[k], 1ull);
        atomicCAS(&first[k], ~0ull, static_cast<unsigned long long>(i));
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&bad[15], static_cast<unsigned long long>(n));
}

// FP64 add throughput: eight independent DADD chains per thread (enough to
// cover the pipe's latency with the resident warps), `iters` steps each.  The
// sum is written so the chains are not removed.
__global__ void __launch_bounds__(256) fp64_rate_kernel(double *out, int64_t iters, double step) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = static_cast<double>(threadIdx.x * 8 + k);
#pragma unroll 1
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __dadd_rn(a[k], step);
  }
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) sum = __dadd_rn(sum, a[k]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

}  // namespace
}  // namespace eik

// Instrument (the paper has no counterpart): FP64 add throughput of the
// current device, for the FP64 roofline of the solver.
extern "C" eik_status eik_fp64_rate(int64_t iters, double *inst_per_s, void *stream) {
  if (iters <= 0 || !inst_per_s) return EIK_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = 8 * sms, block = 256;
  double *d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * grid * block) != cudaSuccess) {
    cudaGetLastError();
    return EIK_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  eik::fp64_rate_kernel<<<grid, block, 0, s>>>(d, iters / 8 + 1, 1.0);   // warm-up
  cudaEventRecord(e0, s);
  eik::fp64_rate_kernel<<<grid, block, 0, s>>>(d, iters, 1.0);
  cudaEventRecord(e1, s);
  eik::note_launches(2);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (e != cudaSuccess || !(ms > 0.f)) {
    cudaGetLastError();
    return EIK_ECUDA;
  }
  *inst_per_s = static_cast<double>(grid) * block * 8.0 * static_cast<double>(iters) / (ms * 1e-3);
  return EIK_OK;
}

extern "C" eik_status eik_selftest(int64_t n, uint64_t seed, int64_t *mismatches, void *stream) {
  if (n < 0 || !mismatches) return EIK_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long *d = nullptr;
  if (cudaMalloc(&d, 32 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return EIK_ENOMEM;
  }
  cudaMemsetAsync(d, 0, 16 * sizeof(unsigned long long), s);
  cudaMemsetAsync(d + 16, 0xff, 16 * sizeof(unsigned long long), s);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t grid = (n + 255) / 256;
  if (grid > 8 * sms) grid = 8 * sms;
  if (grid < 1) grid = 1;
  eik::selftest_kernel<<<static_cast<int>(grid), 256, 0, s>>>(n, seed, d, d + 16);
  eik::note_launches(1);
  unsigned long long h[32];
  cudaError_t e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return EIK_ECUDA;
  for (int k = 0; k < 32; ++k) mismatches[k] = static_cast<int64_t>(h[k]);
  return EIK_OK;
}
