// Sampling kernel: one thread per sample, FP64 (see rt_sample_core.cuh).
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_internal.h"
#include "rt_sample_core.cuh"

namespace rtk {

namespace {

using namespace sampling;

__global__ void sample_kernel(SampleParams p) {
  const StarDev& s = p.s;
  const int64_t n = p.n, ld = p.ld;   // count and SoA row stride
  SampConst<double> c;
  c.rs = s.rs;
  c.cp = s.cp;
  c.sin_tm = s.sin_tm;
  c.cos_tm = s.cos_tm;
  c.B0_eV2 = s.B0_eV2;
  c.R_eV = s.R_eV;
  c.n_inf = s.n_inf;
  c.ma_eV = s.ma_eV;
  c.v0 = s.v0;
  c.psi_fixed = s.psi_fixed;
  c.plasma_a = s.plasma_a;
  c.rlc = s.rlc;
  c.g_eV = s.g_eV;
  c.w_unit = s.w_unit;
  c.disp = s.dispersion;
  c.plasma = s.plasma;
  c.fa_model = s.fa_model;
  c.phase_mode = s.phase_mode;
  c.weight_mode = s.weight_mode;
  c.per_cm3 = PER_CM3_EV3;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double u[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) u[j] = p.u[j * ld + i];
    SampOut<double> o;
    sample_core(c, u, (double)p.n_norm, o);
    p.state[6 * ld + i] = o.delta;
    p.state[7 * ld + i] = o.psi;
    if (!o.ok) {
#pragma unroll
      for (int j = 0; j < 6; ++j) p.state[j * ld + i] = 0.0;
      p.weight[i] = 0.0;
      p.status[i] = RAY_NO_ROOT;
      continue;
    }
    p.weight[i] = o.w;
    p.state[i] = o.x[0] * s.R_km;
    p.state[ld + i] = o.x[1] * s.R_km;
    p.state[2 * ld + i] = o.x[2] * s.R_km;
    p.state[3 * ld + i] = o.k[0] * s.ma_eV;
    p.state[4 * ld + i] = o.k[1] * s.ma_eV;
    p.state[5 * ld + i] = o.k[2] * s.ma_eV;
    p.status[i] = RAY_READY;
  }
}

}  // namespace

cudaError_t launch_sample(const SampleParams& p, cudaStream_t stream) {
  if (p.n <= 0) return cudaSuccess;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int block = 128;
  int64_t grid = (p.n + block - 1) / block;
  const int64_t cap = (int64_t)nsm * 8;
  if (grid > cap) grid = cap;
  sample_kernel<<<(unsigned)grid, block, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk
