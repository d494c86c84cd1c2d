// Binning of escaped rays on the sky and in frequency (Sec. 2.2: the power
// reaching a bin of the sphere at infinity is the sum of the weights of the
// rays that land in it).  Sums are kept in 64-bit fixed point, so the result
// does not depend on the order of the atomics:
//   1. max_kernel      largest escaped weight (atomicMax on the bit pattern,
//                      which orders like the value for non-negative doubles);
//   2. accum_kernel    q = rint(w * 2^e) added to the 3-D histogram (global
//                      atomics) and to sky / spectrum marginals in shared
//                      memory, flushed once per block; 2^e is the largest
//                      power of two with n * wmax * 2^e < 2^62;
//   3. finalize_kernel q / 2^e to float64.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <cmath>
#include <mutex>

#include "rt.h"
#include "rt_device.cuh"
#include "rt_internal.h"

namespace rtk {

namespace {

constexpr int SMEM_SKY_MAX = 4096;   // int64 entries of the shared sky map
constexpr int SMEM_SPEC_MAX = 1024;

__device__ __forceinline__ double fixed_scale(long long wmax_bits, int64_t n) {
  const double wmax = __longlong_as_double(wmax_bits);
  if (!(wmax > 0.0)) return 1.0;
  const double bound = wmax * (double)(n > 0 ? n : 1);
  return ldexp(1.0, 61 - ilogb(bound));
}

__global__ void max_kernel(BinParams p) {
  long long best = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (p.status[i] != RAY_ESCAPED) continue;
    const double w = p.weight[i];
    if (w > 0.0) {
      const long long b = __double_as_longlong(w);
      best = b > best ? b : best;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long v = __shfl_down_sync(0xffffffffu, best, o);
    best = v > best ? v : best;
  }
  if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(&p.acc[0], best);
}

__global__ void accum_kernel(BinParams p) {
  __shared__ long long s_sky[SMEM_SKY_MAX];
  __shared__ long long s_spec[SMEM_SPEC_MAX];
  const int nsky = p.nth * p.nph;
  const bool sky_smem = nsky <= SMEM_SKY_MAX;
  const bool spec_smem = p.nnu <= SMEM_SPEC_MAX;
  for (int j = threadIdx.x; j < SMEM_SKY_MAX; j += blockDim.x) s_sky[j] = 0;
  for (int j = threadIdx.x; j < SMEM_SPEC_MAX; j += blockDim.x) s_spec[j] = 0;
  __syncthreads();
  const double scale = fixed_scale(p.acc[0], p.n);
  const StarDev& s = *p.star;
  long long* g_hist = p.acc + 2;
  long long* g_sky = g_hist + (size_t)nsky * p.nnu;
  long long* g_spec = g_sky + nsky;
  const double dth = PI / p.nth, dph = 2.0 * PI / p.nph;
  const double dnu = (p.nu_hi - p.nu_lo) / p.nnu;
  const double y_unit = 0.5 * s.v0 * s.v0;
  const int64_t n = p.n, ld = p.ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (p.status[i] != RAY_ESCAPED) continue;
    const long long q = llrint(p.weight[i] * scale);
    const double y = p.state[6 * ld + i] / y_unit;
    if (!(y >= p.nu_lo && y < p.nu_hi)) {
      atomicAdd((unsigned long long*)&p.acc[1], (unsigned long long)q);
      continue;
    }
    int inu = (int)floor((y - p.nu_lo) / dnu);
    if (inu >= p.nnu) inu = p.nnu - 1;
    // direction of the orthonormal-frame momentum at the end point
    const double iR = 1.0 / s.R_km;
    const double x0 = p.state[i] * iR, x1 = p.state[ld + i] * iR;
    const double x2 = p.state[2 * ld + i] * iR;
    const double k0 = p.state[3 * ld + i], k1 = p.state[4 * ld + i], k2 = p.state[5 * ld + i];
    const double ir = rsqrt(x0 * x0 + x1 * x1 + x2 * x2);
    const double n0 = x0 * ir, n1 = x1 * ir, n2 = x2 * ir;
    const double A = 1.0 - s.rs_prop * ir;
    const double cr = (sqrt(A) - 1.0) * (n0 * k0 + n1 * k1 + n2 * k2);
    const double o0 = k0 + cr * n0, o1 = k1 + cr * n1, o2 = k2 + cr * n2;
    const double kmag = sqrt(o0 * o0 + o1 * o1 + o2 * o2);
    const double th = acos(fmax(-1.0, fmin(1.0, o2 / kmag)));
    double ph = atan2(o1, o0);
    if (ph < 0.0) ph += 2.0 * PI;
    int ith = (int)floor(th / dth);
    if (ith >= p.nth) ith = p.nth - 1;
    int iph = (int)floor(ph / dph);
    if (iph >= p.nph) iph -= p.nph;
    const int isky = ith * p.nph + iph;
    atomicAdd((unsigned long long*)&g_hist[(size_t)isky * p.nnu + inu], (unsigned long long)q);
    if (sky_smem) atomicAdd((unsigned long long*)&s_sky[isky], (unsigned long long)q);
    else atomicAdd((unsigned long long*)&g_sky[isky], (unsigned long long)q);
    if (spec_smem) atomicAdd((unsigned long long*)&s_spec[inu], (unsigned long long)q);
    else atomicAdd((unsigned long long*)&g_spec[inu], (unsigned long long)q);
  }
  __syncthreads();
  if (sky_smem)
    for (int j = threadIdx.x; j < nsky; j += blockDim.x)
      if (s_sky[j]) atomicAdd((unsigned long long*)&g_sky[j], (unsigned long long)s_sky[j]);
  if (spec_smem)
    for (int j = threadIdx.x; j < p.nnu; j += blockDim.x)
      if (s_spec[j]) atomicAdd((unsigned long long*)&g_spec[j], (unsigned long long)s_spec[j]);
}

__global__ void finalize_kernel(BinParams p) {
  const double inv = 1.0 / fixed_scale(p.acc[0], p.n);
  const int nsky = p.nth * p.nph;
  const int64_t nh = (int64_t)nsky * p.nnu;
  const long long* g_hist = p.acc + 2;
  const long long* g_sky = g_hist + nh;
  const long long* g_spec = g_sky + nsky;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nh;
       j += (int64_t)gridDim.x * blockDim.x) {
    p.hist[j] = (double)g_hist[j] * inv;
    if (p.sky && j < nsky) p.sky[j] = (double)g_sky[j] * inv;
    if (p.spec && j < p.nnu) p.spec[j] = (double)g_spec[j] * inv;
    if (j == 0) *p.oor = (double)p.acc[1] * inv;
  }
}

}  // namespace

cudaError_t launch_bin(const BinParams& p, cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const size_t entries = bin_scratch_entries(p.nth, p.nph, p.nnu);
  e = cudaMemsetAsync(p.acc, 0, entries * sizeof(long long), stream);
  if (e != cudaSuccess) return e;
  const int block = 256;
  int64_t grid = (p.n + block - 1) / block;
  if (grid > (int64_t)nsm * 4) grid = (int64_t)nsm * 4;
  if (grid < 1) grid = 1;
  max_kernel<<<(unsigned)grid, block, 0, stream>>>(p);
  accum_kernel<<<(unsigned)grid, block, 0, stream>>>(p);
  const int64_t nh = (int64_t)p.nth * p.nph * p.nnu;
  int64_t gf = (nh + block - 1) / block;
  if (gf > (int64_t)nsm * 8) gf = (int64_t)nsm * 8;
  if (gf < 1) gf = 1;
  finalize_kernel<<<(unsigned)gf, block, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk
