// Hamilton's equations at given phase-space points: the right-hand side that
// the FP64 integrators step with (rhs64 of rt_integrator.cuh, i.e. ham_rhs of
// rt_device.cuh), exposed so that it can be checked point by point.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt.h"
#include "rt_device.cuh"
#include "rt_integrator.cuh"
#include "rt_internal.h"

namespace rtk {
namespace {

__global__ void hamilton_rhs_kernel(StarDev s, int64_t n, const double* state, double* H,
                                    double* dydl) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double iR = 1.0 / s.R_km, im = 1.0 / s.ma_eV;
    double y[6];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      y[r] = state[r * n + i] * iR;
      y[3 + r] = state[(3 + r) * n + i] * im;
    }
    const double om = 1.0 + state[6 * n + i];
    double sp, cpsi;
    sincos(state[7 * n + i], &sp, &cpsi);
    RayConst<double> c;
    c.rs = s.rs_prop;
    c.cp = s.cp;
    c.pa = s.plasma_a;
    c.W2 = om * om;
    c.iW2 = 1.0 / (om * om);
    c.m0 = s.sin_tm * cpsi;
    c.m1 = s.sin_tm * sp;
    c.m2 = s.cos_tm;
    c.disp = s.dispersion;
    c.plasma = s.plasma;
    c.sig = gj_side<double>(c.m0, c.m1, c.m2, y[0], y[1], y[2]);
    double f[6];
    rhs64(c, y, f);
#pragma unroll
    for (int r = 0; r < 6; ++r) dydl[r * n + i] = f[r];
    if (H) H[i] = ham_value(c, y, y + 3);
  }
}

}  // namespace
}  // namespace rtk

extern "C" rt_status rt_hamilton_rhs(const rt_star* star, int64_t n, const double* d_state,
                                     double* d_H, double* d_dydl, void* stream) {
  rtk::NvtxRange nvtx_range("rt_hamilton_rhs");
  using namespace rtk;
  if (!star) {
    set_last_error("star is NULL");
    return RT_EINVAL;
  }
  if (n < 0) {
    set_last_error("n must be >= 0");
    return RT_EINVAL;
  }
  if (n == 0) return RT_OK;
  rt_status st;
  if ((st = check_device_array(d_state, "d_state")) != RT_OK) return st;
  if ((st = check_device_array(d_dydl, "d_dydl")) != RT_OK) return st;
  if (d_H && (st = check_device_array(d_H, "d_H")) != RT_OK) return st;
  const StarDev& h = star_host_desc(star);
  if (h.rotation != ROTATION_SNAPSHOT) {
    set_last_error("rt_hamilton_rhs evaluates the frozen-magnetosphere Hamiltonian only");
    return RT_EUNSUPPORTED;
  }
  int64_t grid = (n + 127) / 128;
  if (grid > 65535) grid = 65535;
  hamilton_rhs_kernel<<<(unsigned)grid, 128, 0, (cudaStream_t)stream>>>(h, n, d_state, d_H,
                                                                         d_dydl);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return RT_ECUDA;
  }
  return RT_OK;
}
