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

// ---------------------------------------------------------------------------
// Allocation-free variant of the binning entry point.
//
// Some callers may not allocate device memory from inside the library: code
// that runs under a device-memory budget managed by someone else (a
// framework's caching allocator, a fixed memory pool shared through MPS), or a
// real-time pipeline that cannot afford the device synchronisation that
// cudaMalloc / cudaFree may imply.  rt_bin_spectrum_noalloc serves them: its
// fixed-point accumulator is a file-scope __device__ array of a fixed maximum
// size that every GPU loading this library holds until exit, instead of the
// handle-owned scratch that rt_bin_spectrum allocates on first use.  It takes
// the star parameters by value (the three numbers binning needs), so it does
// not need an rt_star handle either.

namespace rtk {
namespace {

constexpr size_t NOALLOC_ENTRIES = (size_t)RT_BIN_NOALLOC_MAX_ENTRIES;  // 4 MiB of int64
static __device__ __align__(256) long long g_noalloc_acc[NOALLOC_ENTRIES];

struct NoAllocBin {
  int64_t n;
  const double* state;
  const double* weight;
  const uint8_t* status;
  int nth, nph, nnu;
  double nu_lo, nu_hi;
  double R_km, rs_prop, v0;
  long long* acc;
  double* hist;
  double* sky;
  double* spec;
  double* oor;
};

__global__ void noalloc_max_kernel(NoAllocBin p) {
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

__global__ void noalloc_accum_kernel(NoAllocBin p) {
  __shared__ long long s_sky[SMEM_SKY_MAX];
  __shared__ long long s_spec[SMEM_SPEC_MAX];
  const int nsky = p.nth * p.nph;
  const bool sky_smem = nsky <= SMEM_SKY_MAX;
  const bool spec_smem = p.nnu <= SMEM_SPEC_MAX;
  for (int j = threadIdx.x; j < SMEM_SKY_MAX; j += blockDim.x) s_sky[j] = 0;
  for (int j = threadIdx.x; j < SMEM_SPEC_MAX; j += blockDim.x) s_spec[j] = 0;
  __syncthreads();
  const double scale = fixed_scale(p.acc[0], p.n);
  long long* g_hist = p.acc + 2;
  long long* g_sky = g_hist + (size_t)nsky * p.nnu;
  long long* g_spec = g_sky + nsky;
  const double dth = PI / p.nth, dph = 2.0 * PI / p.nph;
  const double dnu = (p.nu_hi - p.nu_lo) / p.nnu;
  const double y_unit = 0.5 * p.v0 * p.v0;
  const int64_t n = p.n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (p.status[i] != RAY_ESCAPED) continue;
    const long long q = llrint(p.weight[i] * scale);
    const double y = p.state[6 * n + i] / y_unit;
    if (!(y >= p.nu_lo && y < p.nu_hi)) {
      atomicAdd((unsigned long long*)&p.acc[1], (unsigned long long)q);
      continue;
    }
    int inu = (int)floor((y - p.nu_lo) / dnu);
    if (inu >= p.nnu) inu = p.nnu - 1;
    const double iR = 1.0 / p.R_km;
    const double x0 = p.state[i] * iR, x1 = p.state[n + i] * iR, x2 = p.state[2 * n + i] * iR;
    const double k0 = p.state[3 * n + i], k1 = p.state[4 * n + i], k2 = p.state[5 * n + i];
    const double ir = rsqrt(x0 * x0 + x1 * x1 + x2 * x2);
    const double n0 = x0 * ir, n1 = x1 * ir, n2 = x2 * ir;
    const double A = 1.0 - p.rs_prop * ir;
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

__global__ void noalloc_finalize_kernel(NoAllocBin p) {
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

// Device address of g_noalloc_acc, looked up once per device (with that
// device current) by the first call on it.
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
long long* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

}  // namespace

}  // namespace rtk

extern "C" rt_status rt_bin_spectrum_noalloc(const rt_star_params* params, int64_t n,
                                             const double* d_state, const double* d_weight,
                                             const uint8_t* d_status, int32_t nth, int32_t nph,
                                             int32_t nnu, double nu_lo, double nu_hi,
                                             double* d_hist, double* d_sky, double* d_spec,
                                             double* d_out_of_range, void* stream) {
  using namespace rtk;
  auto fail = [](rt_status s, const char* msg) {
    set_last_error(msg);   // readable through rt_last_error()
    return s;
  };
  if (!params) return fail(RT_EINVAL, "params is NULL");
  if (n < 0) return fail(RT_EINVAL, "n must be >= 0");
  if (nth < 1 || nph < 1 || nnu < 1) return fail(RT_EINVAL, "bin counts must be >= 1");
  if (!(nu_hi > nu_lo) || !std::isfinite(nu_lo) || !std::isfinite(nu_hi))
    return fail(RT_EINVAL, "need finite nu_lo < nu_hi");
  if (!(params->R_km > 0) || !(params->v0_kms > 0) || params->M_sun < 0)
    return fail(RT_EINVAL, "invalid star parameters");
  if ((int64_t)nth * nph * nnu > (int64_t)NOALLOC_ENTRIES)
    return fail(RT_EINVAL,
                "histogram too large for the static accumulator: need 2 + nth*nph*nnu + "
                "nth*nph + nnu <= RT_BIN_NOALLOC_MAX_ENTRIES (524288)");
  const size_t need = bin_scratch_entries(nth, nph, nnu);
  if (need > NOALLOC_ENTRIES)
    return fail(RT_EINVAL,
                "histogram too large for the static accumulator: need 2 + nth*nph*nnu + "
                "nth*nph + nnu <= RT_BIN_NOALLOC_MAX_ENTRIES (524288)");
  if (!d_hist || !d_out_of_range || (n > 0 && (!d_state || !d_weight || !d_status)))
    return fail(RT_EINVAL, "NULL device array");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(RT_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(RT_EINVAL, "device index too large");
  long long* acc;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_acc);
      if (e != cudaSuccess || ptr == nullptr)
        return fail(RT_ECUDA, "cudaGetSymbolAddress of the static accumulator failed");
      g_noalloc_ptr[dev] = (long long*)ptr;
    }
    acc = g_noalloc_ptr[dev];
  }
  NoAllocBin p;
  p.n = n;
  p.state = d_state;
  p.weight = d_weight;
  p.status = d_status;
  p.nth = nth;
  p.nph = nph;
  p.nnu = nnu;
  p.nu_lo = nu_lo;
  p.nu_hi = nu_hi;
  p.R_km = params->R_km;
  const double rs = 2.0 * params->M_sun * 1.4766250 / params->R_km;
  p.rs_prop = (params->prop_metric == RT_METRIC_FLAT) ? 0.0 : rs;
  p.v0 = params->v0_kms / 299792.458;
  p.acc = acc;
  p.hist = d_hist;
  p.sky = d_sky;
  p.spec = d_spec;
  p.oor = d_out_of_range;
  cudaStream_t s = (cudaStream_t)stream;
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(RT_ECUDA, cudaGetErrorString(e));
  e = cudaMemsetAsync(acc, 0, need * sizeof(long long), s);   // clears the previous call's sums
  if (e != cudaSuccess) return fail(RT_ECUDA, cudaGetErrorString(e));
  const int block = 256;
  int64_t grid = (n + block - 1) / block;
  if (grid > (int64_t)nsm * 4) grid = (int64_t)nsm * 4;
  if (grid < 1) grid = 1;
  noalloc_max_kernel<<<(unsigned)grid, block, 0, s>>>(p);
  noalloc_accum_kernel<<<(unsigned)grid, block, 0, s>>>(p);
  const int64_t nh = (int64_t)nth * nph * nnu;
  int64_t gf = (nh + block - 1) / block;
  if (gf > (int64_t)nsm * 8) gf = (int64_t)nsm * 8;
  if (gf < 1) gf = 1;
  noalloc_finalize_kernel<<<(unsigned)gf, block, 0, s>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(RT_ECUDA, cudaGetErrorString(e));
  return RT_OK;
}
