// Kernels of the update-form ablation (Mitigation Strategies section and
// Table 3): evaluation of one update at many points, and the fixed-point
// residual of a field under d-bar or an explicit root.
#include <cstdint>
#include <cuda_runtime.h>

#include "eik_exact.cuh"
#include "eik_forms.cuh"
#include "eik_internal.h"

namespace eik {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// d-bar of the 2D/3D minima a (bit patterns), +inf when all are +inf.
template <int D>
__device__ __forceinline__ unsigned long long dbar_or_inf(const unsigned long long (&a)[D],
                                                          unsigned long long cb) {
  unsigned long long amin = a[0];
#pragma unroll
  for (int k = 1; k < D; ++k) amin = amin < a[k] ? amin : a[k];
  if (amin >= forms::kInf) return forms::kInf;
  return hw::dbar<D>(a, cb);
}

__global__ void eval_update_kernel(int form, const double *__restrict__ speed, double h,
                                   const double *__restrict__ t_h, const double *__restrict__ t_v,
                                   int64_t n, double *__restrict__ out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double r = __ddiv_rn(h, speed[i]);
    const unsigned long long a[2] = {forms::as_u(t_h[i]), forms::as_u(t_v[i])};
    unsigned long long tau;
    if (form == 0) tau = dbar_or_inf<2>(a, forms::as_u(__dmul_rn(r, r)));
    else tau = forms::explicit_update(form, a[0], a[1], r);
    out[i] = forms::as_d(tau);
  }
}

__device__ __forceinline__ bool sorted_find(const int64_t *idx, int64_t n, int64_t key, int64_t &pos) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) >> 1;
    const int64_t v = idx[mid];
    if (v == key) { pos = mid; return true; }
    if (v < key) lo = mid + 1; else hi = mid - 1;
  }
  return false;
}

// One cell per thread: re-apply the update with the final neighbour values;
// out[0] += cells whose value changes (sources: value != t0), out[1] = max of
// |t - tau| / t over finite positive t and tau (bit pattern; +inf otherwise).
template <int D>
__global__ void residual_kernel(int form, const double *__restrict__ speed, double h,
                                const double *__restrict__ t, int64_t nx, int64_t ny, int64_t nz,
                                const int64_t *__restrict__ src_idx,
                                const double *__restrict__ src_t, int64_t nsrc,
                                unsigned long long *out) {
  const int64_t n = nx * ny * nz;
  unsigned long long bad = 0, worst = 0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const double ti = t[i];
    int64_t pos = 0;
    if (nsrc > 0 && sorted_find(src_idx, nsrc, i, pos)) {
      if (!(ti == src_t[pos])) ++bad;
      continue;
    }
    const int64_t x = i % nx, yz = i / nx, y = yz % ny, z = yz / ny;
    unsigned long long a[D];
    {
      const unsigned long long l = x > 0 ? forms::as_u(t[i - 1]) : forms::kInf;
      const unsigned long long r = x + 1 < nx ? forms::as_u(t[i + 1]) : forms::kInf;
      a[0] = l < r ? l : r;
    }
    {
      const unsigned long long l = y > 0 ? forms::as_u(t[i - nx]) : forms::kInf;
      const unsigned long long r = y + 1 < ny ? forms::as_u(t[i + nx]) : forms::kInf;
      a[1] = l < r ? l : r;
    }
    if constexpr (D == 3) {
      const unsigned long long l = z > 0 ? forms::as_u(t[i - nx * ny]) : forms::kInf;
      const unsigned long long r = z + 1 < nz ? forms::as_u(t[i + nx * ny]) : forms::kInf;
      a[2] = l < r ? l : r;
    }
    const double r = __ddiv_rn(h, speed[i]);
    unsigned long long tb;
    if (form == 0) tb = dbar_or_inf<D>(a, forms::as_u(__dmul_rn(r, r)));
    else tb = forms::explicit_update(form, a[0], a[1], r);
    const double tau = forms::as_d(tb);
    if (!(tau == ti)) {
      ++bad;
      unsigned long long rel = forms::kInf;
      if (forms::as_u(ti) < forms::kInf && forms::as_u(tau) < forms::kInf && ti > 0.0)
        rel = forms::as_u(__ddiv_rn(fabs(__dsub_rn(ti, tau)), ti));
      worst = worst > rel ? worst : rel;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bad += __shfl_xor_sync(kFull, bad, o);
    const unsigned long long w = __shfl_xor_sync(kFull, worst, o);
    worst = worst > w ? worst : w;
  }
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicAdd(out, bad);
    if (worst) atomicMax(out + 1, worst);
  }
}

int blocks_for(int64_t n) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (n + 255) / 256;
  if (g > static_cast<int64_t>(sms) * 8) g = static_cast<int64_t>(sms) * 8;
  return static_cast<int>(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_eval_update(int form, const double *speed, double h, const double *t_h,
                               const double *t_v, int64_t n, double *out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  eval_update_kernel<<<blocks_for(n), 256, 0, stream>>>(form, speed, h, t_h, t_v, n, out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_residual(int form, int ndim, const double *speed, double h, const double *t,
                            int64_t nx, int64_t ny, int64_t nz, const int64_t *src_idx,
                            const double *src_t, int64_t nsrc, unsigned long long *out,
                            cudaStream_t stream) {
  const int64_t n = nx * ny * nz;
  if (n <= 0) return cudaSuccess;
  if (ndim == 3)
    residual_kernel<3><<<blocks_for(n), 256, 0, stream>>>(form, speed, h, t, nx, ny, nz, src_idx,
                                                          src_t, nsrc, out);
  else
    residual_kernel<2><<<blocks_for(n), 256, 0, stream>>>(form, speed, h, t, nx, ny, nz, src_idx,
                                                          src_t, nsrc, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace eik
