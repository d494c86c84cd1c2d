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
// n in the bound is BinParams::n_scale: the rays of this call, or of all shards
// of a sharded binning (rt_bin_part_*), whose int64 sums add exactly.
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
  const double scale = fixed_scale(p.acc[0], p.n_scale);
  long long* g_hist = p.acc + 2;
  long long* g_sky = g_hist + (size_t)nsky * p.nnu;
  long long* g_spec = g_sky + nsky;
  const double dth = PI / p.nth, dph = 2.0 * PI / p.nph;
  const double dnu = (p.nu_hi - p.nu_lo) / p.nnu;
  const double y_unit = 0.5 * p.v0 * p.v0;
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
    const double iR = 1.0 / p.R_km;
    const double x0 = p.state[i] * iR, x1 = p.state[ld + i] * iR;
    const double x2 = p.state[2 * ld + i] * iR;
    const double k0 = p.state[3 * ld + i], k1 = p.state[4 * ld + i], k2 = p.state[5 * ld + i];
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

__global__ void finalize_kernel(BinParams p) {
  const double inv = 1.0 / fixed_scale(p.acc[0], p.n_scale);
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

namespace {

cudaError_t sm_count(int* nsm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  return cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev);
}

constexpr int BIN_BLOCK = 256;

// Grid of the per-ray kernels: one thread per ray up to 4 blocks per SM.
unsigned ray_grid(int64_t n, int nsm) {
  int64_t grid = (n + BIN_BLOCK - 1) / BIN_BLOCK;
  if (grid > (int64_t)nsm * 4) grid = (int64_t)nsm * 4;
  return (unsigned)(grid < 1 ? 1 : grid);
}

}  // namespace

cudaError_t launch_bin_max(const BinParams& p, cudaStream_t stream) {
  int nsm = 0;
  cudaError_t e = sm_count(&nsm);
  if (e != cudaSuccess) return e;
  const size_t entries = bin_scratch_entries(p.nth, p.nph, p.nnu);
  e = cudaMemsetAsync(p.acc, 0, entries * sizeof(long long), stream);
  if (e != cudaSuccess) return e;
  max_kernel<<<ray_grid(p.n, nsm), BIN_BLOCK, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_bin_accum(const BinParams& p, cudaStream_t stream) {
  int nsm = 0;
  cudaError_t e = sm_count(&nsm);
  if (e != cudaSuccess) return e;
  accum_kernel<<<ray_grid(p.n, nsm), BIN_BLOCK, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_bin_finalize(const BinParams& p, cudaStream_t stream) {
  int nsm = 0;
  cudaError_t e = sm_count(&nsm);
  if (e != cudaSuccess) return e;
  const int64_t nh = (int64_t)p.nth * p.nph * p.nnu;
  int64_t gf = (nh + BIN_BLOCK - 1) / BIN_BLOCK;
  if (gf > (int64_t)nsm * 8) gf = (int64_t)nsm * 8;
  if (gf < 1) gf = 1;
  finalize_kernel<<<(unsigned)gf, BIN_BLOCK, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_bin(const BinParams& p, cudaStream_t stream) {
  cudaError_t e = launch_bin_max(p, stream);
  if (e == cudaSuccess) e = launch_bin_accum(p, stream);
  if (e == cudaSuccess) e = launch_bin_finalize(p, stream);
  return e;
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
// not need an rt_star handle either; the kernels are those of rt_bin_spectrum.

namespace rtk {
namespace {

constexpr size_t NOALLOC_ENTRIES = (size_t)RT_BIN_NOALLOC_MAX_ENTRIES;  // 4 MiB of int64
static __device__ __align__(256) long long g_noalloc_acc[NOALLOC_ENTRIES];

// Device address of g_noalloc_acc, looked up once per device (with that
// device current) by the first call on it.  cudaDeviceReset destroys the
// context that this address belongs to (documented in rt.h).
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
long long* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

rt_status bin_fail(rt_status s, const char* msg) {
  set_last_error(msg);   // readable through rt_last_error()
  return s;
}

rt_status bin_cuda_fail(cudaError_t e) {
  cudaGetLastError();    // clear a sticky launch error so that later calls do not see it
  return bin_fail(RT_ECUDA, cudaGetErrorString(e));
}

// Checks shared by the entry points of this file.
rt_status check_bins(int32_t nth, int32_t nph, int32_t nnu) {
  if (nth < 1 || nph < 1 || nnu < 1) return bin_fail(RT_EINVAL, "bin counts must be >= 1");
  if ((int64_t)nth * nph * nnu > (int64_t)1 << 28) return bin_fail(RT_EINVAL, "too many bins");
  return RT_OK;
}

rt_status check_rays(int64_t n, const double* d_state, const double* d_weight,
                     const uint8_t* d_status) {
  if (n <= 0) return RT_OK;
  rt_status st;
  if (d_state && (st = check_device_array(d_state, "d_state")) != RT_OK) return st;
  if ((st = check_device_array(d_weight, "d_weight")) != RT_OK) return st;
  if ((st = check_device_array(d_status, "d_status")) != RT_OK) return st;
  return RT_OK;
}

rt_status check_outputs(const double* d_hist, const double* d_sky, const double* d_spec,
                        const double* d_oor) {
  rt_status st;
  if ((st = check_device_array(d_hist, "d_hist")) != RT_OK) return st;
  if ((st = check_device_array(d_oor, "d_out_of_range")) != RT_OK) return st;
  if (d_sky && (st = check_device_array(d_sky, "d_sky")) != RT_OK) return st;
  if (d_spec && (st = check_device_array(d_spec, "d_spec")) != RT_OK) return st;
  return RT_OK;
}

}  // namespace
}  // namespace rtk

extern "C" rt_status rt_bin_spectrum_noalloc(const rt_star_params* params, int64_t n,
                                             const double* d_state, const double* d_weight,
                                             const uint8_t* d_status, int32_t nth, int32_t nph,
                                             int32_t nnu, double nu_lo, double nu_hi,
                                             double* d_hist, double* d_sky, double* d_spec,
                                             double* d_out_of_range, void* stream) {
  rtk::NvtxRange nvtx_range("rt_bin_spectrum_noalloc");
  using namespace rtk;
  rt_status st;
  if ((st = check_star_params(params)) != RT_OK) return st;
  if (n < 0) return bin_fail(RT_EINVAL, "n must be >= 0");
  if ((st = check_bins(nth, nph, nnu)) != RT_OK) return st;
  if (!(nu_hi > nu_lo) || !std::isfinite(nu_lo) || !std::isfinite(nu_hi))
    return bin_fail(RT_EINVAL, "need finite nu_lo < nu_hi");
  const size_t need = bin_scratch_entries(nth, nph, nnu);
  if (need > NOALLOC_ENTRIES)
    return bin_fail(RT_EINVAL,
                    "histogram too large for the static accumulator: need 2 + nth*nph*nnu + "
                    "nth*nph + nnu <= RT_BIN_NOALLOC_MAX_ENTRIES (524288)");
  if (n > 0 && !d_state) return bin_fail(RT_EINVAL, "d_state is NULL");
  if ((st = check_rays(n, d_state, d_weight, d_status)) != RT_OK) return st;
  if ((st = check_outputs(d_hist, d_sky, d_spec, d_out_of_range)) != RT_OK) return st;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bin_cuda_fail(e);
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return bin_fail(RT_EINVAL, "device index too large");
  long long* acc;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_acc);
      if (e != cudaSuccess || ptr == nullptr) {
        cudaGetLastError();
        return bin_fail(RT_ECUDA, "cudaGetSymbolAddress of the static accumulator failed");
      }
      g_noalloc_ptr[dev] = (long long*)ptr;
    }
    acc = g_noalloc_ptr[dev];
  }
  BinParams p;
  p.R_km = params->R_km;
  const double rs = 2.0 * params->M_sun * 1.4766250 / params->R_km;
  p.rs_prop = (params->prop_metric == RT_METRIC_FLAT) ? 0.0 : rs;
  p.v0 = params->v0_kms / 299792.458;
  p.n = n;
  p.ld = n;
  p.n_scale = n;
  p.state = d_state;
  p.weight = d_weight;
  p.status = d_status;
  p.nth = nth;
  p.nph = nph;
  p.nnu = nnu;
  p.nu_lo = nu_lo;
  p.nu_hi = nu_hi;
  p.acc = acc;        // launch_bin clears the part of it this call uses
  p.hist = d_hist;
  p.sky = d_sky;
  p.spec = d_spec;
  p.oor = d_out_of_range;
  e = launch_bin(p, (cudaStream_t)stream);
  if (e != cudaSuccess) return bin_cuda_fail(e);
  return RT_OK;
}

// ---------------------------------------------------------------------------
// Sharded binning: the three phases of rt_bin_spectrum around caller-owned
// int64 sums, reduced exactly between the phases by the caller (one process
// per GPU, each with a contiguous range of one workload's rays).

namespace {

rtk::BinParams part_params(int64_t n, int64_t n_total, const double* d_state,
                           const double* d_weight, const uint8_t* d_status, int32_t nth,
                           int32_t nph, int32_t nnu, double nu_lo, double nu_hi, int64_t* d_acc) {
  rtk::BinParams p;
  p.R_km = 1.0;
  p.rs_prop = 0.0;
  p.v0 = 1.0;
  p.n = n;
  p.ld = n;
  p.n_scale = n_total;
  p.state = d_state;
  p.weight = d_weight;
  p.status = d_status;
  p.nth = nth;
  p.nph = nph;
  p.nnu = nnu;
  p.nu_lo = nu_lo;
  p.nu_hi = nu_hi;
  p.acc = (long long*)d_acc;
  p.hist = p.sky = p.spec = p.oor = nullptr;
  return p;
}

}  // namespace

extern "C" rt_status rt_bin_part_max(int64_t n, const double* d_weight, const uint8_t* d_status,
                                     int32_t nth, int32_t nph, int32_t nnu, int64_t* d_acc,
                                     void* stream) {
  rtk::NvtxRange nvtx_range("rt_bin_part_max");
  using namespace rtk;
  rt_status st;
  if (n < 0) return bin_fail(RT_EINVAL, "n must be >= 0");
  if ((st = check_bins(nth, nph, nnu)) != RT_OK) return st;
  if ((st = check_rays(n, nullptr, d_weight, d_status)) != RT_OK) return st;
  if ((st = check_device_array(d_acc, "d_acc")) != RT_OK) return st;
  const BinParams p =
      part_params(n, n, nullptr, d_weight, d_status, nth, nph, nnu, 0.0, 1.0, d_acc);
  const cudaError_t e = launch_bin_max(p, (cudaStream_t)stream);
  if (e != cudaSuccess) return bin_cuda_fail(e);
  return RT_OK;
}

extern "C" rt_status rt_bin_part_accumulate(const rt_star* star, int64_t n, int64_t ld,
                                            int64_t n_total, const double* d_state,
                                            const double* d_weight,
                                            const uint8_t* d_status, int32_t nth, int32_t nph,
                                            int32_t nnu, double nu_lo, double nu_hi,
                                            int64_t* d_acc, void* stream) {
  rtk::NvtxRange nvtx_range("rt_bin_part_accumulate");
  using namespace rtk;
  rt_status st;
  if (!star) return bin_fail(RT_EINVAL, "star is NULL");
  if (n < 0 || n_total < n) return bin_fail(RT_EINVAL, "need 0 <= n <= n_total");
  if (ld < n) return bin_fail(RT_EINVAL, "need ld >= n");
  if ((st = check_bins(nth, nph, nnu)) != RT_OK) return st;
  if (!(nu_hi > nu_lo) || !std::isfinite(nu_lo) || !std::isfinite(nu_hi))
    return bin_fail(RT_EINVAL, "need finite nu_lo < nu_hi");
  if (n > 0 && !d_state) return bin_fail(RT_EINVAL, "d_state is NULL");
  if ((st = check_rays(n, d_state, d_weight, d_status)) != RT_OK) return st;
  if ((st = check_device_array(d_acc, "d_acc")) != RT_OK) return st;
  BinParams p =
      part_params(n, n_total, d_state, d_weight, d_status, nth, nph, nnu, nu_lo, nu_hi, d_acc);
  const StarDev& h = star_host_desc(star);
  p.ld = ld;
  p.R_km = h.R_km;
  p.rs_prop = h.rs_prop;
  p.v0 = h.v0;
  const cudaError_t e = launch_bin_accum(p, (cudaStream_t)stream);
  if (e != cudaSuccess) return bin_cuda_fail(e);
  return RT_OK;
}

extern "C" rt_status rt_bin_part_finalize(int32_t nth, int32_t nph, int32_t nnu, int64_t n_total,
                                          const int64_t* d_acc, double* d_hist, double* d_sky,
                                          double* d_spec, double* d_out_of_range, void* stream) {
  rtk::NvtxRange nvtx_range("rt_bin_part_finalize");
  using namespace rtk;
  rt_status st;
  if (n_total < 0) return bin_fail(RT_EINVAL, "n_total must be >= 0");
  if ((st = check_bins(nth, nph, nnu)) != RT_OK) return st;
  if ((st = check_device_array(d_acc, "d_acc")) != RT_OK) return st;
  if ((st = check_outputs(d_hist, d_sky, d_spec, d_out_of_range)) != RT_OK) return st;
  BinParams p = part_params(0, n_total, nullptr, nullptr, nullptr, nth, nph, nnu, 0.0, 1.0,
                            const_cast<int64_t*>(d_acc));
  p.hist = d_hist;
  p.sky = d_sky;
  p.spec = d_spec;
  p.oor = d_out_of_range;
  const cudaError_t e = launch_bin_finalize(p, (cudaStream_t)stream);
  if (e != cudaSuccess) return bin_cuda_fail(e);
  return RT_OK;
}
