// C ABI of the ray tracer (include/rt.h): argument validation, derived star
// constants, handle-owned scratch, and kernel launches on the caller's stream.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "rt.h"
#include "rt_device.cuh"
#include "rt_backward.cuh"
#include "rt_internal.h"

namespace {

// Constants (the values the paper asks to keep identical everywhere, Sec. 2.4).
constexpr double PI = 3.14159265358979323846;
constexpr double HBARC_EV_KM = 1.973269804e-10;  // hbar c [eV km], CODATA 2018
constexpr double HBAR_EV_S = 6.582119569e-16;     // hbar [eV s], CODATA 2018
constexpr double ALPHA = 7.2973525693e-3;         // fine-structure constant, CODATA 2018
constexpr double ME_EV = 510998.95;               // electron mass [eV], CODATA 2018
constexpr double EV_J = 1.602176634e-19;          // exact
constexpr double C_KM_S = 299792.458;             // exact
constexpr double GM_SUN_KM = 1.4766250;           // G Msun / c^2 [km], IAU 2015 nominal

thread_local std::string g_err;

rt_status fail(rt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

rt_status cuda_fail(cudaError_t e, const char* where) {
  return fail(RT_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool is_finite_val(double v) { return std::isfinite(v); }

// Device arrays must be device (or managed) memory of the current device.
rt_status check_dev_ptr(const void* p, const char* name) {
  if (p == nullptr) return fail(RT_EINVAL, "%s is NULL", name);
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RT_EINVAL, "%s is not a CUDA pointer", name);
  }
  if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
    return fail(RT_EINVAL, "%s must be device memory", name);
  int dev = 0;
  cudaGetDevice(&dev);
  if (a.type == cudaMemoryTypeDevice && a.device != dev)
    return fail(RT_EINVAL, "%s lives on device %d, current device is %d", name, a.device, dev);
  return RT_OK;
}

}  // namespace

void rtk::set_last_error(const char* msg) { g_err = msg; }

rt_status rtk::check_device_array(const void* p, const char* name) {
  return check_dev_ptr(p, name);
}

rt_status rtk::check_star_params(const rt_star_params* p) {
  if (p == nullptr) return fail(RT_EINVAL, "params is NULL");
  const double vals[] = {p->M_sun, p->R_km, p->B0_G, p->P_s, p->theta_m_rad, p->psi_rad,
                         p->m_a_eV, p->g_agg_GeVinv, p->rho_dm_GeV_cm3, p->v0_kms,
                         p->plasma_a};
  for (double v : vals)
    if (!is_finite_val(v)) return fail(RT_EINVAL, "non-finite star parameter");
  if (p->M_sun < 0) return fail(RT_EINVAL, "M_sun must be >= 0");
  if (!(p->R_km > 0)) return fail(RT_EINVAL, "R_km must be > 0");
  const double rs = 2.0 * p->M_sun * GM_SUN_KM / p->R_km;
  if (!(rs < 1.0)) return fail(RT_EINVAL, "R_km must exceed the Schwarzschild radius");
  if (!(p->m_a_eV > 0)) return fail(RT_EINVAL, "m_a_eV must be > 0");
  if (!(p->P_s > 0)) return fail(RT_EINVAL, "P_s must be > 0");
  if (p->B0_G < 0 || p->g_agg_GeVinv < 0 || p->rho_dm_GeV_cm3 < 0)
    return fail(RT_EINVAL, "B0_G, g_agg_GeVinv and rho_dm_GeV_cm3 must be >= 0");
  if (!(p->v0_kms > 0 && p->v0_kms < C_KM_S)) return fail(RT_EINVAL, "v0_kms out of range");
  if (p->dispersion != RT_DISP_ANISO && p->dispersion != RT_DISP_ISO)
    return fail(RT_EUNSUPPORTED, "unknown dispersion %d", p->dispersion);
  if (p->resonance != RT_RES_KINEMATIC)
    return fail(RT_EUNSUPPORTED, "unsupported resonance mode %d", p->resonance);
  if (p->fa_model != RT_FA_MAXWELL && p->fa_model != RT_FA_DELTA)
    return fail(RT_EUNSUPPORTED, "unknown fa_model %d", p->fa_model);
  if (p->weight_mode != RT_WEIGHT_PAG && p->weight_mode != RT_WEIGHT_UNIT_P &&
      p->weight_mode != RT_WEIGHT_RENORM)
    return fail(RT_EUNSUPPORTED, "unsupported weight_mode %d", p->weight_mode);
  if (p->prop_metric != RT_METRIC_FULL && p->prop_metric != RT_METRIC_FLAT)
    return fail(RT_EUNSUPPORTED, "unknown prop_metric %d", p->prop_metric);
  if (p->rotation != RT_ROTATION_SNAPSHOT && p->rotation != RT_ROTATION_RIGID)
    return fail(RT_EUNSUPPORTED, "unknown rotation %d", p->rotation);
  if (p->phase_mode != RT_PHASE_FIXED && p->phase_mode != RT_PHASE_UNIFORM)
    return fail(RT_EUNSUPPORTED, "unknown phase_mode %d", p->phase_mode);
  if (p->plasma < RT_PLASMA_GJ || p->plasma > RT_PLASMA_TWISTED)
    return fail(RT_EUNSUPPORTED, "unknown plasma %d", p->plasma);
  if (p->plasma == RT_PLASMA_TWISTED && !(p->plasma_a > 0))
    return fail(RT_EINVAL, "RT_PLASMA_TWISTED needs plasma_a = lambda psi > 0");
  return RT_OK;
}

struct rt_star {
  rt_star_params p;
  rtk::StarDev h;               // host copy of the descriptor
  rtk::StarDev* d = nullptr;    // device copy
  unsigned long long* d_queue = nullptr;  // trace work-queue counter (scratch)
  long long* d_bins = nullptr;  // binning accumulator (scratch)
  size_t bins_cap = 0;
  int device = 0;
  double wp2_surface_max = 0.0;
  bool empty = false;
  double* d_park = nullptr;     // tail-mode park buffer (allocated on first use)
  int64_t park_cap = 0;
  int32_t* d_promo = nullptr;   // mixed backward: [count | pixels handed to FP64]
  int64_t promo_cap = 0;
};

const rtk::StarDev& rtk::star_host_desc(const rt_star* s) { return s->h; }

extern "C" {

const char* rt_last_error(void) { return g_err.c_str(); }

int32_t rt_version(void) { return 20000; }

rt_status rt_init_star(const rt_star_params* p, rt_star** out) {
  if (out == nullptr) return fail(RT_EINVAL, "out is NULL");
  *out = nullptr;
  const rt_status chk = rtk::check_star_params(p);
  if (chk != RT_OK) return chk;
  const double rs = 2.0 * p->M_sun * GM_SUN_KM / p->R_km;

  rt_star* s = new (std::nothrow) rt_star;
  if (!s) return fail(RT_ENOMEM, "host allocation failed");
  s->p = *p;
  rtk::StarDev& h = s->h;
  memset(&h, 0, sizeof(h));
  h.rs = rs;
  h.rs_prop = (p->prop_metric == RT_METRIC_FLAT) ? 0.0 : rs;
  // Goldreich-Julian: n_e = 2 |Omega.B| / e, omega_p^2 = e^2 n_e / m_e (Eq.
  // GJDensity, Heaviside-Lorentz natural units), dipole B = B0/2 (R/r)^3 (...)
  const double e_hl = std::sqrt(4.0 * PI * ALPHA);
  const double omega_eV = HBAR_EV_S * 2.0 * PI / p->P_s;
  const double hbarc_cm = HBARC_EV_KM * 1e5;
  const double B0_eV2 =
      p->B0_G * std::sqrt((1e-7 / EV_J) * hbarc_cm * hbarc_cm * hbarc_cm / (4.0 * PI));
  h.cp = e_hl * omega_eV * B0_eV2 / ME_EV / (p->m_a_eV * p->m_a_eV);
  if (p->plasma == RT_PLASMA_TWISTED) {
    // twisted magnetosphere (Eq. neMag): n_e = lambda psi sin^2(theta) B0 (R/r)^3
    // / (e r), omega_p^2 / m_a^2 = cp sin^2(theta) (R/r)^4 with
    // cp = e lambda psi B0 / (R m_e m_a^2) (Heaviside-Lorentz natural units)
    h.cp = e_hl * p->plasma_a * B0_eV2 / (p->R_km / HBARC_EV_KM) / ME_EV /
           (p->m_a_eV * p->m_a_eV);
  }
  h.rlc = C_KM_S * p->P_s / (2.0 * PI * p->R_km);
  h.plasma_a = p->plasma_a;
  h.cos_tm = std::cos(p->theta_m_rad);
  h.sin_tm = std::sin(p->theta_m_rad);
  h.psi_fixed = p->psi_rad;
  h.v0 = p->v0_kms / C_KM_S;
  h.R_km = p->R_km;
  h.ma_eV = p->m_a_eV;
  h.R_eV = p->R_km / HBARC_EV_KM;
  h.B0_eV2 = B0_eV2;
  h.g_eV = p->g_agg_GeVinv * 1e-9;
  h.n_inf = p->rho_dm_GeV_cm3 * 1e9 * hbarc_cm * hbarc_cm * hbarc_cm / p->m_a_eV;
  h.w_unit = EV_J / HBAR_EV_S;
  h.dispersion = p->dispersion;
  h.plasma = p->plasma;
  h.fa_model = p->fa_model;
  h.phase_mode = p->phase_mode;
  h.weight_mode = p->weight_mode;
  h.rotation = p->rotation;
  // Largest omega_p^2 / m_a^2 on the surface: max over n of
  // |3 n_z (m.n) - cos th_m| = (3 + |cos th_m|) / 2 (eigenvalues of the
  // symmetrised z m^T).  A kinematic resonance needs omega_p > m_a somewhere.
  switch (p->plasma) {
    case RT_PLASMA_GJ: s->wp2_surface_max = h.cp * 0.5 * (3.0 + std::fabs(h.cos_tm)); break;
    case RT_PLASMA_HOMOG: s->wp2_surface_max = p->plasma_a; break;
    case RT_PLASMA_LINEAR_Z: s->wp2_surface_max = std::fabs(p->plasma_a) * 1e30; break;
    case RT_PLASMA_RADIAL: s->wp2_surface_max = p->plasma_a; break;
    case RT_PLASMA_TWISTED: s->wp2_surface_max = h.cp; break;     // sin^2 = 1
    default: s->wp2_surface_max = 0.0; break;
  }
  s->empty = !(s->wp2_surface_max > 1.0);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) {
    delete s;
    return cuda_fail(e, "cudaGetDevice");
  }
  void* blk = nullptr;
  e = cudaMalloc(&blk, 256 + sizeof(rtk::StarDev));
  if (e != cudaSuccess) {
    delete s;
    return (e == cudaErrorMemoryAllocation) ? fail(RT_ENOMEM, "cudaMalloc failed")
                                            : cuda_fail(e, "cudaMalloc");
  }
  s->d_queue = (unsigned long long*)blk;
  s->d = (rtk::StarDev*)((char*)blk + 256);
  e = cudaMemcpy(s->d, &h, sizeof(h), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(blk);
    delete s;
    return cuda_fail(e, "cudaMemcpy");
  }
  *out = s;
  return RT_OK;
}

void rt_destroy_star(rt_star* s) {
  if (!s) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != s->device) cudaSetDevice(s->device);
  if (s->d_bins) cudaFree(s->d_bins);
  if (s->d_queue) cudaFree(s->d_queue);
  if (s->d_park) cudaFree(s->d_park);
  if (s->d_promo) cudaFree(s->d_promo);
  if (cur != s->device) cudaSetDevice(cur);
  delete s;
}

rt_status rt_star_info(const rt_star* s, double* out) {
  if (!s || !out) return fail(RT_EINVAL, "NULL argument");
  out[0] = s->h.rs;
  out[1] = s->h.cp;
  out[2] = s->h.B0_eV2;
  out[3] = s->h.R_eV;
  out[4] = s->h.n_inf;
  out[5] = s->h.v0;
  out[6] = s->wp2_surface_max;
  out[7] = s->empty ? 1.0 : 0.0;
  return RT_OK;
}

rt_status rt_sample_conversion_surface(const rt_star* s, int64_t n, const double* d_u,
                                       double* d_state, double* d_weight, uint8_t* d_status,
                                       void* stream) {
  return rt_sample_conversion_surface_part(s, n, n > 0 ? n : 1, d_u, d_state, d_weight, d_status,
                                           stream);
}

rt_status rt_sample_conversion_surface_part(const rt_star* s, int64_t n, int64_t n_norm,
                                            const double* d_u, double* d_state,
                                            double* d_weight, uint8_t* d_status, void* stream) {
  rtk::NvtxRange nvtx_range("rt_sample_conversion_surface_part");
  if (!s) return fail(RT_EINVAL, "star is NULL");
  if (n < 0) return fail(RT_EINVAL, "n must be >= 0");
  if (n_norm < n || n_norm < 1) return fail(RT_EINVAL, "need n_norm >= max(n, 1)");
  if (n == 0) return s->empty ? RT_EEMPTY_SURFACE : RT_OK;
  rt_status st;
  if ((st = check_dev_ptr(d_u, "d_uniforms")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_state, "d_state")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_weight, "d_weight")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  rtk::SampleParams p;
  p.s = s->h;
  p.n = n;
  p.ld = n;
  p.n_norm = n_norm;
  p.u = d_u;
  p.state = d_state;
  p.weight = d_weight;
  p.status = d_status;
  cudaError_t e = rtk::launch_sample(p, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sample kernel");
  return s->empty ? RT_EEMPTY_SURFACE : RT_OK;
}

// The tail-mode park buffer: two counters, then park_capacity entries.
static rt_status ensure_park(double** buf, int64_t* cap) {
  if (*buf) return RT_OK;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t c = rtk::park_capacity(nsm > 0 ? nsm : 1);
  void* p = nullptr;
  // [256 B counters | c park records | express area]
  if (cudaMalloc(&p, 256 + (size_t)c * rtk::PARKREC * sizeof(double) + rtk::express_bytes()) !=
      cudaSuccess) {
    cudaGetLastError();
    return fail(RT_ENOMEM, "cannot allocate the tail-mode park buffer");
  }
  *buf = (double*)p;
  *cap = c;
  return RT_OK;
}

static void set_park(rtk::TraceParams& p, double* buf, int64_t cap, const rt_trace_opts* o) {
  if (o->tail != 1 && buf) {
    p.park_count = (unsigned long long*)buf;
    p.park_next = p.park_count + 1;
    p.park = buf + 32;           // after the 256-byte counter block
    p.park_cap = cap;
    p.park_live = (o->tail == 0) ? rtk::PARK_LIVE_MAX : o->tail;
  } else {
    p.park = nullptr;
    p.park_count = p.park_next = nullptr;
    p.park_cap = 0;
  }
}

// The express area after the park records (cost-ordered FP64 tracing with a
// park buffer): the bucket-0 rays are traced six lanes per ray from the start.
static void set_express(rtk::TraceParams& p) {
  if (!p.order || !p.park) {
    p.xrec = nullptr;
    return;
  }
  char* x = (char*)(p.park + p.park_cap * rtk::PARKREC);
  p.xcount = (unsigned long long*)x;
  p.xslot = (int*)(x + 64);
  p.xcand = (unsigned long long*)(x + 64 + rtk::XSLOTS * sizeof(int));
  p.xrec = (double*)(x + 64 + rtk::XSLOTS * sizeof(int) +
                     (size_t)rtk::XCAP * 2 * sizeof(unsigned long long));
  p.xcap = rtk::XCAP;
  p.xpark = (p.n >= rtk::XPARK_MIN_RAYS) ? 1 : 0;
}

static rt_status check_opts(const rt_trace_opts* o) {
  if (!o) return fail(RT_EINVAL, "opts is NULL");
  if (!(o->rtol > 0 && o->rtol < 1) || !(o->atol > 0 && o->atol < 1))
    return fail(RT_EINVAL, "rtol and atol must be in (0, 1)");
  if (!(o->r_capture_over_R > 0) || !(o->r_out_over_R > o->r_capture_over_R) ||
      !is_finite_val(o->r_out_over_R))
    return fail(RT_EINVAL, "need 0 < r_capture_over_R < r_out_over_R < inf");
  if (!(o->lambda_max >= 0) || !is_finite_val(o->lambda_max))
    return fail(RT_EINVAL, "lambda_max must be finite and >= 0");
  if (o->max_steps <= 0) return fail(RT_EINVAL, "max_steps must be > 0");
  if (o->max_steps > (1 << 28)) return fail(RT_EINVAL, "max_steps too large");
  if (o->precision != RT_PREC_FP64 && o->precision != RT_PREC_MIXED &&
      o->precision != RT_PREC_DF)
    return fail(RT_EINVAL, "unknown precision %d", o->precision);
  if (o->block < 0 || o->blocks_per_sm < 0) return fail(RT_EINVAL, "negative launch parameter");
  if (o->tail < 0 || o->tail > 31) return fail(RT_EINVAL, "tail must be in [0, 31]");
  if (o->claim_order != RT_CLAIM_COST && o->claim_order != RT_CLAIM_INDEX)
    return fail(RT_EINVAL, "unknown claim_order %d", o->claim_order);
  if (o->refill_min < 0 || o->refill_min > 32)
    return fail(RT_EINVAL, "refill_min must be in [0, 32]");
  if (o->rays_per_claim < 0 || o->rays_per_claim > 64)
    return fail(RT_EINVAL, "rays_per_claim must be in [0, 64]");
  return RT_OK;
}

// The work-claiming knobs of opts (0: the given defaults, e.g. autotuned).
// Default refill thresholds per precision, measured on the eight-step
// benchmark launch (16 x 65536 rays x 8, cost order): a warp that refills only
// once several lanes are free loads their rays in one divergent pass instead
// of one each -- double-float 2.67 -> 2.29 s (16), mixed 253 -> 195 ms (16),
// FP64 3.61 -> 3.39 s (8; 16 is slower again).
static int default_refill(int precision) {
  return precision == RT_PREC_FP64 ? 8 : 16;
}

static void set_claiming(rtk::TraceParams& p, const rt_trace_opts* o, int refill_auto,
                         int claim_auto) {
  p.refill_min = o->refill_min > 0 ? o->refill_min
                                   : (refill_auto > 0 ? refill_auto : default_refill(o->precision));
  p.claim_size = o->rays_per_claim > 0 ? o->rays_per_claim : (claim_auto > 0 ? claim_auto : 1);
}

rt_status rt_trace_forward(const rt_star* s, int64_t n, double* d_state, uint8_t* d_status,
                           int32_t* d_nacc, int32_t* d_nrej, int64_t* d_counters,
                           const rt_trace_opts* o, void* stream) {
  rtk::NvtxRange nvtx_range("rt_trace_forward");
  if (!s) return fail(RT_EINVAL, "star is NULL");
  if (n < 0) return fail(RT_EINVAL, "n must be >= 0");
  rt_status st;
  if ((st = check_opts(o)) != RT_OK) return st;
  if (n == 0) return RT_OK;
  if ((st = check_dev_ptr(d_state, "d_state")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  if (d_nacc && (st = check_dev_ptr(d_nacc, "d_nacc")) != RT_OK) return st;
  if (d_nrej && (st = check_dev_ptr(d_nrej, "d_nrej")) != RT_OK) return st;
  if (d_counters && (st = check_dev_ptr(d_counters, "d_counters")) != RT_OK) return st;
  if (o->precision != RT_PREC_FP64 && o->lambda_max > 0)
    return fail(RT_EUNSUPPORTED, "lambda_max is only supported with RT_PREC_FP64");
  const bool rigid = (s->p.rotation == RT_ROTATION_RIGID);
  if (rigid && o->precision != RT_PREC_FP64)
    return fail(RT_EUNSUPPORTED, "a rotating magnetosphere is traced in RT_PREC_FP64 only");
  rtk::TraceParams p;
  p.stars = s->d;
  p.nstars = 1;
  p.offsets = nullptr;
  p.n = n;
  p.state = d_state;
  p.status = d_status;
  p.nacc = d_nacc;
  p.nrej = d_nrej;
  p.counters = d_counters;
  p.queue = s->d_queue;
  p.ts = (unsigned long long*)o->timestamps;
  if (o->tail != 1 && o->lambda_max == 0.0 && !rigid && o->precision != RT_PREC_DF) {
    rt_star* sm = const_cast<rt_star*>(s);
    if ((st = ensure_park(&sm->d_park, &sm->park_cap)) != RT_OK) return st;
    set_park(p, sm->d_park, sm->park_cap, o);
  } else {
    set_park(p, nullptr, 0, o);
  }
  p.rtol = o->rtol;
  p.atol = o->atol;
  p.r_out = o->r_out_over_R;
  p.lambda_max = o->lambda_max;
  p.r_capture = o->r_capture_over_R;
  p.max_steps = o->max_steps;
  p.claim_status = rtk::RAY_READY;
  p.order = (o->claim_order == RT_CLAIM_COST) ? 1 : 0;
  if (o->precision == RT_PREC_FP64) set_express(p);
  set_claiming(p, o, 0, 0);
  cudaError_t e;
  if (rigid) {
    e = rtk::launch_trace_rot(p, o->block, o->blocks_per_sm, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "rotating-magnetosphere trace kernel");
    return RT_OK;
  }
  if (o->precision == RT_PREC_DF) {
    e = rtk::launch_trace_df(p, o->block, o->blocks_per_sm, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "double-float trace kernel");
    return RT_OK;
  }
  if (o->precision == RT_PREC_MIXED) {
    e = rtk::launch_trace_mixed(p, o->block, o->blocks_per_sm, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mixed trace kernel");
    p.claim_status = rtk::RAY_PROMOTED;   // FP64 pass over the promoted rays
    p.order = 0;
    p.xrec = nullptr;
    e = rtk::launch_trace_fp64(p, 0, 0, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "trace kernel (promoted rays)");
    return RT_OK;
  }
  e = rtk::launch_trace_fp64(p, o->block, o->blocks_per_sm, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "trace kernel");
  return RT_OK;
}

// Checks of one image's geometry (rt_trace_backward's arguments).
static rt_status check_image(int32_t nx, int32_t ny, double incl_rad, double dist_over_R,
                             double bmax_over_R, double Lc_cut_km) {
  if (nx < 1 || ny < 1) return fail(RT_EINVAL, "nx and ny must be >= 1");
  if ((int64_t)nx * ny > ((int64_t)1 << 31)) return fail(RT_EINVAL, "nx * ny > 2^31");
  if (!is_finite_val(incl_rad) || !is_finite_val(dist_over_R) || !is_finite_val(bmax_over_R) ||
      !is_finite_val(Lc_cut_km))
    return fail(RT_EINVAL, "non-finite argument");
  if (!(bmax_over_R > 0)) return fail(RT_EINVAL, "bmax_over_R must be > 0");
  if (!(dist_over_R > bmax_over_R * std::sqrt(2.0) + 1.0))
    return fail(RT_EINVAL, "dist_over_R must exceed bmax_over_R * sqrt(2) + 1");
  if (Lc_cut_km < 0) return fail(RT_EINVAL, "Lc_cut_km must be >= 0");
  return RT_OK;
}

// Line centre, pixel scale and cut of one image (Sec. 2.1, Eq. BackPower).
static void image_setup(const rtk::StarDev& h, int32_t nx, int32_t ny, double bmax_over_R,
                        double Lc_cut_km, double* W, double* img_scale, double* Lc_cut) {
  // line centre and the analytic frequency integral of f_a (Eq. GaussianDist)
  *W = std::sqrt(1.0 + h.v0 * h.v0);
  const double k0 = h.v0 * h.ma_eV, w0 = *W * h.ma_eV;
  const double Fa = (h.fa_model == rtk::FA_DELTA) ? w0 * h.n_inf / (4.0 * PI * k0)
                                                  : w0 * h.n_inf / (2.0 * std::pow(PI, 1.5) * k0);
  const double dbx = 2.0 * bmax_over_R / nx * h.R_eV, dby = 2.0 * bmax_over_R / ny * h.R_eV;
  *img_scale = dbx * dby * Fa * h.w_unit;
  *Lc_cut = Lc_cut_km / h.R_km;
}

rt_status rt_trace_backward(const rt_star* s, int32_t nx, int32_t ny, double incl_rad,
                            double dist_over_R, double bmax_over_R, double Lc_cut_km,
                            double* d_image, uint8_t* d_status, int32_t* d_ncross,
                            int64_t* d_counters, const rt_trace_opts* o, void* stream) {
  rtk::NvtxRange nvtx_range("rt_trace_backward");
  if (!s) return fail(RT_EINVAL, "star is NULL");
  rt_status st;
  if ((st = check_opts(o)) != RT_OK) return st;
  if (o->precision == RT_PREC_DF)
    return fail(RT_EUNSUPPORTED, "images are traced in RT_PREC_FP64 or RT_PREC_MIXED");
  if ((st = check_image(nx, ny, incl_rad, dist_over_R, bmax_over_R, Lc_cut_km)) != RT_OK)
    return st;
  if ((st = check_dev_ptr(d_image, "d_image")) != RT_OK) return st;
  if (s->p.weight_mode != RT_WEIGHT_PAG)
    return fail(RT_EUNSUPPORTED, "rt_trace_backward needs RT_WEIGHT_PAG");
  if (s->p.rotation != RT_ROTATION_SNAPSHOT)
    return fail(RT_EUNSUPPORTED, "rt_trace_backward needs RT_ROTATION_SNAPSHOT");
  if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  if (d_ncross && (st = check_dev_ptr(d_ncross, "d_ncross")) != RT_OK) return st;
  if (d_counters && (st = check_dev_ptr(d_counters, "d_counters")) != RT_OK) return st;
  const rtk::StarDev& h = s->h;
  double W, img_scale, Lc_cut;
  image_setup(h, nx, ny, bmax_over_R, Lc_cut_km, &W, &img_scale, &Lc_cut);
  rtk::BackLaunch b;
  b.star = &h;
  b.nx = nx;
  b.ny = ny;
  b.incl = incl_rad;
  b.D = dist_over_R;
  b.bmax = bmax_over_R;
  b.W = W;
  b.Lc_cut = Lc_cut;
  b.img_scale = img_scale;
  b.rtol = o->rtol;
  b.atol = o->atol;
  b.r_capture = o->r_capture_over_R;
  b.max_steps = o->max_steps;
  b.image = d_image;
  b.status = d_status;
  b.ncross = d_ncross;
  b.counters = d_counters;
  b.queue = s->d_queue;
  b.ts = (unsigned long long*)o->timestamps;
  b.prec = o->precision;
  b.promo = nullptr;
  b.promo_n = nullptr;
  if (o->precision == RT_PREC_MIXED) {
    // list of the pixels handed to the FP64 kernel (each at most once)
    const int64_t npix = (int64_t)nx * ny;
    rt_star* sm = const_cast<rt_star*>(s);
    if (sm->promo_cap < npix) {
      if (sm->d_promo) cudaFree(sm->d_promo);
      sm->d_promo = nullptr;
      sm->promo_cap = 0;
      void* p = nullptr;
      if (cudaMalloc(&p, 256 + (size_t)npix * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        return fail(RT_ENOMEM, "cannot allocate the promoted-pixel list");
      }
      sm->d_promo = (int32_t*)p;
      sm->promo_cap = npix;
    }
    b.promo_n = (unsigned long long*)sm->d_promo;
    b.promo = sm->d_promo + 64;        // after the 256-byte counter block
  }
  cudaError_t e = rtk::launch_backward(b, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "backward kernel");
  return RT_OK;
}

static double vmf_norm(double kappa) {
  return kappa / (2.0 * PI * -std::expm1(-2.0 * kappa));
}

rt_status rt_flux_value(const rt_star* s, int64_t n, const double* d_state,
                        const double* d_weight, const uint8_t* d_status, double incl_rad,
                        double kappa, double* d_F_ray, double* d_F, void* stream) {
  rtk::NvtxRange nvtx_range("rt_flux_value");
  if (!s) return fail(RT_EINVAL, "star is NULL");
  if (n < 1) return fail(RT_EINVAL, "n must be >= 1");
  if (!is_finite_val(incl_rad) || !(kappa > 0) || !is_finite_val(kappa))
    return fail(RT_EINVAL, "need finite incl_rad and 0 < kappa < inf");
  rt_status st;
  if ((st = check_dev_ptr(d_state, "d_state")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_weight, "d_weight")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_F_ray, "d_F_ray")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_F, "d_F")) != RT_OK) return st;
  cudaError_t e = rtk::launch_flux_value(s->d, n, d_state, d_weight, d_status, incl_rad, kappa,
                                         vmf_norm(kappa), d_F_ray, d_F, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "flux value kernel");
  return RT_OK;
}

rt_status rt_flux_gradient(const rt_star* s, int64_t n, const double* d_uniforms,
                           const int32_t* d_nacc, double incl_rad, double kappa,
                           const rt_trace_opts* o, double* d_grad, double* d_F,
                           uint8_t* d_status, int64_t* d_counters, int64_t tape_max_bytes,
                           int64_t* store_bytes, void* stream) {
  rtk::NvtxRange nvtx_range("rt_flux_gradient");
  if (!s) return fail(RT_EINVAL, "star is NULL");
  if (n < 1) return fail(RT_EINVAL, "n must be >= 1");
  rt_status st;
  if ((st = check_opts(o)) != RT_OK) return st;
  if (o->lambda_max != 0.0) return fail(RT_EUNSUPPORTED, "lambda_max must be 0");
  if (!is_finite_val(incl_rad) || !(kappa > 0) || !is_finite_val(kappa))
    return fail(RT_EINVAL, "need finite incl_rad and 0 < kappa < inf");
  if ((st = check_dev_ptr(d_uniforms, "d_uniforms")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_nacc, "d_nacc")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_grad, "d_grad")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_F, "d_F")) != RT_OK) return st;
  if (d_status && (st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  if (d_counters && (st = check_dev_ptr(d_counters, "d_counters")) != RT_OK) return st;
  const rt_star_params& p = s->p;
  const rtk::StarDev& h = s->h;
  if (p.plasma != RT_PLASMA_GJ) return fail(RT_EUNSUPPORTED, "the gradient needs RT_PLASMA_GJ");
  if (p.weight_mode != RT_WEIGHT_PAG)
    return fail(RT_EUNSUPPORTED, "the gradient needs RT_WEIGHT_PAG");
  if (p.rotation != RT_ROTATION_SNAPSHOT)
    return fail(RT_EUNSUPPORTED, "the gradient needs RT_ROTATION_SNAPSHOT");
  if (!(p.M_sun > 0) || !(p.B0_G > 0))
    return fail(RT_EINVAL, "the gradient needs M_sun > 0 and B0_G > 0");
  typedef rtk::Dual<rtk::NSAMP_TANGENTS> D5;
  rtk::AdjLaunch a;
  // sampling constants with their derivatives (m_a, B0, theta_m, M, R): each a
  // monomial in the parameters (rt_init_star)
  D5 c;
  c = D5(h.rs);
  c.d[rtk::PAR_M] = h.rs / p.M_sun;
  c.d[rtk::PAR_R] = -h.rs / p.R_km;
  a.sc.rs = c;
  c = D5(h.cp);
  c.d[rtk::PAR_MA] = -2.0 * h.cp / p.m_a_eV;
  c.d[rtk::PAR_B0] = h.cp / p.B0_G;
  a.sc.cp = c;
  c = D5(h.sin_tm);
  c.d[rtk::PAR_THM] = h.cos_tm;
  a.sc.sin_tm = c;
  c = D5(h.cos_tm);
  c.d[rtk::PAR_THM] = -h.sin_tm;
  a.sc.cos_tm = c;
  c = D5(h.B0_eV2);
  c.d[rtk::PAR_B0] = h.B0_eV2 / p.B0_G;
  a.sc.B0_eV2 = c;
  c = D5(h.R_eV);
  c.d[rtk::PAR_R] = h.R_eV / p.R_km;
  a.sc.R_eV = c;
  c = D5(h.n_inf);
  c.d[rtk::PAR_MA] = -h.n_inf / p.m_a_eV;
  a.sc.n_inf = c;
  c = D5(h.ma_eV);
  c.d[rtk::PAR_MA] = 1.0;
  a.sc.ma_eV = c;
  a.sc.v0 = h.v0;
  a.sc.psi_fixed = h.psi_fixed;
  a.sc.plasma_a = h.plasma_a;
  a.sc.rlc = h.rlc;
  a.sc.per_cm3 = rtk::PER_CM3_EV3;
  a.sc.g_eV = h.g_eV;
  a.sc.w_unit = h.w_unit;
  a.sc.disp = h.dispersion;
  a.sc.plasma = h.plasma;
  a.sc.fa_model = h.fa_model;
  a.sc.phase_mode = h.phase_mode;
  a.star = &h;
  const bool flat = (p.prop_metric == RT_METRIC_FLAT);
  a.drsp_dM = flat ? 0.0 : h.rs / p.M_sun;
  a.drsp_dR = flat ? 0.0 : -h.rs / p.R_km;
  a.dcp_dma = -2.0 * h.cp / p.m_a_eV;
  a.dcp_dB0 = h.cp / p.B0_G;
  a.incl = incl_rad;
  a.kappa = kappa;
  a.knorm = vmf_norm(kappa);
  a.rtol = o->rtol;
  a.atol = o->atol;
  a.r_out = o->r_out_over_R;
  a.r_capture = o->r_capture_over_R;
  a.max_steps = o->max_steps;
  a.n = n;
  a.u = d_uniforms;
  a.grad = d_grad;
  a.F = d_F;
  a.counters = d_counters;
  a.queue = s->d_queue;
  cudaStream_t cs = (cudaStream_t)stream;
  a.prec = o->precision;
  a.ck_off = nullptr;
  a.ck = a.seg = nullptr;
  a.tape_off = nullptr;
  a.tape = a.head = nullptr;
  a.order = nullptr;
  a.bucket = nullptr;
  a.grid = a.block = 0;
  cudaError_t e = cudaSuccess;
  // scratch: tape or checkpoint offsets, per-ray results; then the full step
  // tape (with the per-ray heads and the longest-first order) when it fits
  // under tape_max_bytes, else the checkpoints and the segment records
  int64_t* off = nullptr;
  double *ck = nullptr, *seg = nullptr, *Fr = nullptr, *Gr = nullptr, *tape = nullptr,
         *head = nullptr;
  int64_t* order = nullptr;
  unsigned long long* bucket = nullptr;
  uint8_t* stt = nullptr;
  int32_t* flg = nullptr;
  auto cleanup = [&]() {
    cudaFree(off);
    cudaFree(ck);
    cudaFree(seg);
    cudaFree(Fr);
    cudaFree(Gr);
    cudaFree(tape);
    cudaFree(head);
    cudaFree(order);
    cudaFree(bucket);
    if (!d_status) cudaFree(stt);
    cudaFree(flg);
  };
  auto alloc_fail = [&](cudaError_t err, const char* what) {
    cleanup();
    return (err == cudaErrorMemoryAllocation) ? fail(RT_ENOMEM, what)
                                              : cuda_fail(err, "cudaMalloc");
  };
  if ((e = cudaMalloc(&off, (n + 1) * sizeof(int64_t))) != cudaSuccess ||
      (e = cudaMalloc(&Fr, n * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&Gr, (size_t)rtk::NPARAMS * n * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&flg, n * sizeof(int32_t))) != cudaSuccess ||
      (!d_status && (e = cudaMalloc(&stt, n)) != cudaSuccess))
    return alloc_fail(e, "adjoint scratch allocation failed");
  if (d_status) stt = d_status;
  a.F_ray = Fr;
  a.G_ray = Gr;
  a.status = stt;
  a.flags = flg;
  a.nacc = d_nacc;
  // the tape's size from the forward step counts
  int64_t total = 0;
  if ((e = rtk::launch_tape_offsets(d_nacc, n, off, cs)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&total, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, cs)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(cs)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "tape offsets");
  }
  const int64_t tape_bytes = total * rtk::SEGREC * (int64_t)sizeof(double) +
                             n * (rtk::HEADREC * (int64_t)sizeof(double) + 8);
  int64_t limit = tape_max_bytes;
  if (limit < 0) {
    size_t fr = 0, tot = 0;
    if ((e = cudaMemGetInfo(&fr, &tot)) != cudaSuccess) {
      cleanup();
      return cuda_fail(e, "cudaMemGetInfo");
    }
    limit = (int64_t)(fr / 2);
  }
  bool use_tape = tape_bytes <= limit;
  if (use_tape &&
      ((e = cudaMalloc(&tape, (size_t)total * rtk::SEGREC * sizeof(double))) != cudaSuccess ||
       (e = cudaMalloc(&head, (size_t)n * rtk::HEADREC * sizeof(double))) != cudaSuccess ||
       (e = cudaMalloc(&order, (size_t)n * sizeof(int64_t))) != cudaSuccess ||
       (e = cudaMalloc(&bucket, 32 * sizeof(unsigned long long))) != cudaSuccess)) {
    if (e != cudaErrorMemoryAllocation) return alloc_fail(e, "step tape allocation failed");
    // the tape did not fit after all (fragmentation): the checkpoints instead
    cudaGetLastError();
    cudaFree(tape);
    cudaFree(head);
    cudaFree(order);
    cudaFree(bucket);
    tape = head = nullptr;
    order = nullptr;
    bucket = nullptr;
    use_tape = false;
  }
  if (use_tape) {
    if (store_bytes) *store_bytes = tape_bytes;
    a.tape_off = off;
    a.tape = tape;
    a.head = head;
    a.order = order;
    a.bucket = bucket;
    e = rtk::launch_adjoint_tape(a, cs);
  } else {
    e = rtk::adjoint_grid(a.prec, &a.grid, &a.block);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_fail(e, "adjoint occupancy");
    }
    const size_t seg_n = (size_t)a.grid * a.block * rtk::CK * rtk::SEGREC;
    if ((e = cudaMalloc(&seg, seg_n * sizeof(double))) != cudaSuccess)
      return alloc_fail(e, "adjoint segment scratch allocation failed");
    if ((e = rtk::launch_ck_offsets(d_nacc, n, off, cs)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&total, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, cs)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(cs)) != cudaSuccess) {
      cleanup();
      return cuda_fail(e, "checkpoint offsets");
    }
    if ((e = cudaMalloc(&ck, (size_t)total * rtk::CKREC * sizeof(double))) != cudaSuccess)
      return alloc_fail(e, "checkpoint allocation failed");
    if (store_bytes) *store_bytes = total * rtk::CKREC * (int64_t)sizeof(double);
    a.ck_off = off;
    a.ck = ck;
    a.seg = seg;
    e = rtk::launch_adjoint(a, cs);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel");
  return RT_OK;
}

rt_status rt_bin_spectrum(const rt_star* s_, int64_t n, const double* d_state,
                          const double* d_weight, const uint8_t* d_status, int32_t nth,
                          int32_t nph, int32_t nnu, double nu_lo, double nu_hi, double* d_hist,
                          double* d_sky, double* d_spec, double* d_oor, void* stream) {
  rtk::NvtxRange nvtx_range("rt_bin_spectrum");
  rt_star* s = const_cast<rt_star*>(s_);
  if (!s) return fail(RT_EINVAL, "star is NULL");
  if (n < 0) return fail(RT_EINVAL, "n must be >= 0");
  if (nth < 1 || nph < 1 || nnu < 1) return fail(RT_EINVAL, "bin counts must be >= 1");
  if ((int64_t)nth * nph * nnu > (int64_t)1 << 28) return fail(RT_EINVAL, "too many bins");
  if (!is_finite_val(nu_lo) || !is_finite_val(nu_hi) || !(nu_hi > nu_lo))
    return fail(RT_EINVAL, "need finite nu_lo < nu_hi");
  rt_status st;
  if (n > 0) {
    if ((st = check_dev_ptr(d_state, "d_state")) != RT_OK) return st;
    if ((st = check_dev_ptr(d_weight, "d_weight")) != RT_OK) return st;
    if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  }
  if ((st = check_dev_ptr(d_hist, "d_hist")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_oor, "d_out_of_range")) != RT_OK) return st;
  if (d_sky && (st = check_dev_ptr(d_sky, "d_sky")) != RT_OK) return st;
  if (d_spec && (st = check_dev_ptr(d_spec, "d_spec")) != RT_OK) return st;
  const size_t need = rtk::bin_scratch_entries(nth, nph, nnu);
  if (need > s->bins_cap) {
    if (s->d_bins) {
      cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
      cudaFree(s->d_bins);
      s->d_bins = nullptr;
      s->bins_cap = 0;
    }
    void* b = nullptr;
    cudaError_t e = cudaMalloc(&b, need * sizeof(long long));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RT_ENOMEM, "cannot allocate %zu bytes of binning scratch",
                  need * sizeof(long long));
    }
    s->d_bins = (long long*)b;
    s->bins_cap = need;
  }
  rtk::BinParams p;
  p.R_km = s->h.R_km;
  p.rs_prop = s->h.rs_prop;
  p.v0 = s->h.v0;
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
  p.acc = s->d_bins;
  p.hist = d_hist;
  p.sky = d_sky;
  p.spec = d_spec;
  p.oor = d_oor;
  cudaError_t e = rtk::launch_bin(p, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "bin kernels");
  return RT_OK;
}

// --- batches of stars (one persistent launch over all of them) ---------------

}  // extern "C"

struct rt_batch {
  std::vector<const rt_star*> stars;
  std::vector<int64_t> off;           // nstars + 1 host offsets
  int64_t N = 0;
  rtk::StarDev* d_stars = nullptr;    // device table
  int64_t* d_off = nullptr;           // device offsets
  unsigned long long* d_queue = nullptr;
  long long* d_bins = nullptr;        // nstars x per-star binning accumulators
  size_t bins_per_star = 0;
  int device = 0;
  bool all_empty = true;
  std::vector<int64_t> norm;          // per-star weight normalisation (empty: the counts)
  bool rigid = false;                 // every star RT_ROTATION_RIGID (rt_trace_rot.cu)
  // autotuned launch per precision and kind (rays only / with images); 0 = default
  struct Tuned {
    int block = 0, bps = 0, refill = 0, claim = 0;
  } tuned[3][2];       // [precision: FP64, mixed, double-float][rays only, with images]
  double* d_park = nullptr;           // tail-mode park buffer (allocated on first use)
  int64_t park_cap = 0;
  // backward images traced in the same launch (rt_batch_set_images)
  int nimg = 0;
  int64_t npix = 0;
  void* d_img_block = nullptr;        // [promo count | image table | offsets | promo list]
  rtk::BackParams* d_img = nullptr;
  int64_t* d_img_off = nullptr;
  unsigned long long* d_promo_n = nullptr;
  int32_t* d_promo = nullptr;
  // host copies of the images' geometry and stars (the autotuner's coarse copies)
  std::vector<rt_image_desc> h_desc;
  std::vector<const rt_star*> h_img_star;
};

extern "C" {

rt_status rt_init_batch(const rt_star* const* stars, int32_t nstars, const int64_t* counts,
                        rt_batch** out) {
  if (!out) return fail(RT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!stars || !counts || nstars < 1) return fail(RT_EINVAL, "need nstars >= 1 stars and counts");
  rt_batch* b = new (std::nothrow) rt_batch;
  if (!b) return fail(RT_ENOMEM, "host allocation failed");
  b->off.assign((size_t)nstars + 1, 0);
  std::vector<rtk::StarDev> table((size_t)nstars);
  for (int s = 0; s < nstars; ++s) {
    if (!stars[s] || counts[s] < 0) {
      delete b;
      return fail(RT_EINVAL, "star %d is NULL or has a negative count", s);
    }
    if (stars[s]->p.rotation != stars[0]->p.rotation) {
      delete b;
      return fail(RT_EUNSUPPORTED, "star %d: a batch cannot mix rotation modes", s);
    }
    b->stars.push_back(stars[s]);
    table[s] = stars[s]->h;
    b->off[s + 1] = b->off[s] + counts[s];
    b->all_empty = b->all_empty && stars[s]->empty;
  }
  b->rigid = (stars[0]->p.rotation == RT_ROTATION_RIGID);
  b->N = b->off[nstars];
  cudaGetDevice(&b->device);
  const size_t tbl = sizeof(rtk::StarDev) * nstars, offb = sizeof(int64_t) * (nstars + 1);
  void* blk = nullptr;
  cudaError_t e = cudaMalloc(&blk, 256 + tbl + 256 + offb);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(RT_ENOMEM, "cudaMalloc failed for the batch tables");
  }
  b->d_queue = (unsigned long long*)blk;
  b->d_stars = (rtk::StarDev*)((char*)blk + 256);
  b->d_off = (int64_t*)((char*)blk + 256 + ((tbl + 255) / 256) * 256);
  e = cudaMemcpy(b->d_stars, table.data(), tbl, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_off, b->off.data(), offb, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(blk);
    delete b;
    return cuda_fail(e, "cudaMemcpy");
  }
  *out = b;
  return RT_OK;
}

void rt_destroy_batch(rt_batch* b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != b->device) cudaSetDevice(b->device);
  if (b->d_bins) cudaFree(b->d_bins);
  if (b->d_queue) cudaFree(b->d_queue);
  if (b->d_park) cudaFree(b->d_park);
  if (b->d_img_block) cudaFree(b->d_img_block);
  if (cur != b->device) cudaSetDevice(cur);
  delete b;
}

rt_status rt_batch_set_images(rt_batch* b, int32_t nimg, const rt_star* const* stars,
                              const rt_image_desc* descs, double* d_image, uint8_t* d_img_status,
                              int32_t* d_ncross) {
  if (!b) return fail(RT_EINVAL, "batch is NULL");
  if (nimg < 0) return fail(RT_EINVAL, "nimg must be >= 0");
  if (nimg > 0 && (!stars || !descs)) return fail(RT_EINVAL, "stars and descs are required");
  rt_status st;
  std::vector<rtk::BackParams> tbl((size_t)nimg);
  std::vector<int64_t> off((size_t)nimg + 1, 0);
  for (int32_t j = 0; j < nimg; ++j) {
    const rt_image_desc& d = descs[j];
    if (!stars[j]) return fail(RT_EINVAL, "image %d: star is NULL", j);
    if (stars[j]->p.weight_mode != RT_WEIGHT_PAG)
      return fail(RT_EUNSUPPORTED, "image %d: backward images need RT_WEIGHT_PAG", j);
    if (stars[j]->p.rotation != RT_ROTATION_SNAPSHOT)
      return fail(RT_EUNSUPPORTED, "image %d: backward images need RT_ROTATION_SNAPSHOT", j);
    if ((st = check_image(d.nx, d.ny, d.incl_rad, d.dist_over_R, d.bmax_over_R, d.Lc_cut_km)) !=
        RT_OK)
      return st;
    off[j + 1] = off[j] + (int64_t)d.nx * d.ny;
  }
  const int64_t npix = off[nimg];
  if (npix > ((int64_t)1 << 31)) return fail(RT_EINVAL, "more than 2^31 pixels in all images");
  if (npix > 0) {
    if ((st = check_dev_ptr(d_image, "d_image")) != RT_OK) return st;
    if ((st = check_dev_ptr(d_img_status, "d_img_status")) != RT_OK) return st;
    if (d_ncross && (st = check_dev_ptr(d_ncross, "d_ncross")) != RT_OK) return st;
  }
  std::vector<rt_image_desc> h_desc(descs, descs + nimg);
  std::vector<const rt_star*> h_star(stars, stars + nimg);
  for (int32_t j = 0; j < nimg; ++j) {
    const rt_image_desc& d = descs[j];
    const rtk::StarDev& h = stars[j]->h;
    rtk::BackParams& bp = tbl[j];
    memset(&bp, 0, sizeof(bp));
    bp.s = h;
    bp.nx = d.nx;
    bp.ny = d.ny;
    bp.incl = d.incl_rad;
    bp.D = d.dist_over_R;
    bp.bmax = d.bmax_over_R;
    image_setup(h, d.nx, d.ny, d.bmax_over_R, d.Lc_cut_km, &bp.W, &bp.img_scale, &bp.Lc_cut);
    bp.image = d_image + off[j];
    bp.status = d_img_status + off[j];
    bp.ncross = d_ncross ? d_ncross + off[j] : nullptr;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != b->device) cudaSetDevice(b->device);
  if (b->d_img_block) cudaFree(b->d_img_block);
  b->d_img_block = nullptr;
  b->d_img = nullptr;
  b->d_img_off = nullptr;
  b->d_promo_n = nullptr;
  b->d_promo = nullptr;
  b->nimg = 0;
  b->npix = 0;
  b->h_desc.clear();
  b->h_img_star.clear();
  rt_status out = RT_OK;
  if (nimg > 0) {
    const size_t tb = ((sizeof(rtk::BackParams) * nimg + 255) / 256) * 256;
    const size_t ob = (((size_t)nimg + 1) * sizeof(int64_t) + 255) / 256 * 256;
    void* blk = nullptr;
    cudaError_t e = cudaMalloc(&blk, 256 + tb + ob + (size_t)npix * sizeof(int32_t));
    if (e == cudaSuccess) {
      char* c = (char*)blk;
      e = cudaMemcpy(c + 256, tbl.data(), sizeof(rtk::BackParams) * nimg, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(c + 256 + tb, off.data(), off.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice);
      if (e == cudaSuccess) {
        b->d_img_block = blk;
        b->d_promo_n = (unsigned long long*)c;
        b->d_img = (rtk::BackParams*)(c + 256);
        b->d_img_off = (int64_t*)(c + 256 + tb);
        b->d_promo = (int32_t*)(c + 256 + tb + ob);
        b->nimg = nimg;
        b->npix = npix;
        b->h_desc.swap(h_desc);
        b->h_img_star.swap(h_star);
      } else {
        cudaFree(blk);
      }
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      out = (e == cudaErrorMemoryAllocation) ? fail(RT_ENOMEM, "image table allocation failed")
                                             : cuda_fail(e, "image table upload");
    }
  }
  if (cur != b->device) cudaSetDevice(cur);
  return out;
}

rt_status rt_sample_batch(rt_batch* b, const double* d_u, double* d_state, double* d_weight,
                          uint8_t* d_status, void* stream) {
  rtk::NvtxRange nvtx_range("rt_sample_batch");
  if (!b) return fail(RT_EINVAL, "batch is NULL");
  if (b->N == 0) return RT_OK;
  rt_status st;
  if ((st = check_dev_ptr(d_u, "d_uniforms")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_state, "d_state")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_weight, "d_weight")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  for (size_t s = 0; s < b->stars.size(); ++s) {
    const int64_t o = b->off[s], cnt = b->off[s + 1] - o;
    if (cnt == 0) continue;
    rtk::SampleParams p;
    p.s = b->stars[s]->h;
    p.n = cnt;
    p.ld = b->N;
    p.n_norm = b->norm.empty() ? cnt : b->norm[s];
    p.u = d_u + o;
    p.state = d_state + o;
    p.weight = d_weight + o;
    p.status = d_status + o;
    cudaError_t e = rtk::launch_sample(p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "sample kernel");
  }
  return b->all_empty ? RT_EEMPTY_SURFACE : RT_OK;
}

rt_status rt_batch_set_norm(rt_batch* b, const int64_t* n_norm) {
  if (!b) return fail(RT_EINVAL, "batch is NULL");
  if (!n_norm) {
    b->norm.clear();
    return RT_OK;
  }
  const size_t nst = b->stars.size();
  for (size_t s = 0; s < nst; ++s)
    if (n_norm[s] < b->off[s + 1] - b->off[s] || n_norm[s] < 1)
      return fail(RT_EINVAL, "n_norm[%zu] = %lld is below the star's ray count or 1", s,
                  (long long)n_norm[s]);
  b->norm.assign(n_norm, n_norm + nst);
  return RT_OK;
}

rt_status rt_trace_batch(rt_batch* b, double* d_state, uint8_t* d_status, int32_t* d_nacc,
                         int32_t* d_nrej, int64_t* d_counters, const rt_trace_opts* o,
                         void* stream) {
  rtk::NvtxRange nvtx_range("rt_trace_batch");
  if (!b) return fail(RT_EINVAL, "batch is NULL");
  rt_status st;
  if ((st = check_opts(o)) != RT_OK) return st;
  if (b->N == 0 && b->npix == 0) return RT_OK;
  if ((st = check_dev_ptr(d_state, "d_state")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  if (d_nacc && (st = check_dev_ptr(d_nacc, "d_nacc")) != RT_OK) return st;
  if (d_nrej && (st = check_dev_ptr(d_nrej, "d_nrej")) != RT_OK) return st;
  if (d_counters && (st = check_dev_ptr(d_counters, "d_counters")) != RT_OK) return st;
  if (o->precision != RT_PREC_FP64 && o->lambda_max > 0)
    return fail(RT_EUNSUPPORTED, "lambda_max is only supported with RT_PREC_FP64");
  if (o->precision == RT_PREC_DF && b->npix > 0)
    return fail(RT_EUNSUPPORTED, "a batch with images is traced in RT_PREC_FP64 or RT_PREC_MIXED");
  if (b->rigid && o->precision != RT_PREC_FP64)
    return fail(RT_EUNSUPPORTED, "a rotating magnetosphere is traced in RT_PREC_FP64 only");
  rtk::TraceParams p;
  p.stars = b->d_stars;
  p.nstars = (int)b->stars.size();
  p.offsets = b->d_off;
  p.n = b->N;
  p.state = d_state;
  p.status = d_status;
  p.nacc = d_nacc;
  p.nrej = d_nrej;
  p.counters = d_counters;
  p.queue = b->d_queue;
  p.ts = (unsigned long long*)o->timestamps;
  if (o->tail != 1 && o->lambda_max == 0.0 && !b->rigid && o->precision != RT_PREC_DF) {
    if ((st = ensure_park(&b->d_park, &b->park_cap)) != RT_OK) return st;
    set_park(p, b->d_park, b->park_cap, o);
  } else {
    set_park(p, nullptr, 0, o);
  }
  p.rtol = o->rtol;
  p.atol = o->atol;
  p.r_out = o->r_out_over_R;
  p.lambda_max = o->lambda_max;
  p.r_capture = o->r_capture_over_R;
  p.max_steps = o->max_steps;
  p.claim_status = rtk::RAY_READY;
  // cost-ordered claims for the rays-only launches (not with images); the
  // express lane for FP64 ones
  p.order = (o->claim_order == RT_CLAIM_COST && b->npix == 0) ? 1 : 0;
  if (o->precision == RT_PREC_FP64) set_express(p);
  const int pi = (o->precision == RT_PREC_MIXED) ? 1 : (o->precision == RT_PREC_DF) ? 2 : 0;
  const rt_batch::Tuned& tu = b->tuned[pi][b->npix > 0 ? 1 : 0];
  const int blk = o->block > 0 ? o->block : tu.block;
  const int bps = o->block > 0 ? o->blocks_per_sm : tu.bps;
  set_claiming(p, o, tu.refill, tu.claim);
  cudaError_t e;
  if (b->rigid) {   // no images: rt_batch_set_images rejects rotating stars
    e = rtk::launch_trace_rot(p, o->block, o->blocks_per_sm, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "rotating-magnetosphere trace kernel");
    return RT_OK;
  }
  if (b->npix > 0) {
    // rays and pixels in one persistent launch (no tail mode)
    if (o->lambda_max != 0.0)
      return fail(RT_EUNSUPPORTED, "lambda_max must be 0 for a batch with images");
    rtk::ImgTable t;
    t.img = b->d_img;
    t.off = b->d_img_off;
    t.nimg = b->nimg;
    t.npix = b->npix;
    t.promo = b->d_promo;
    t.promo_n = b->d_promo_n;
    t.list = nullptr;
    t.list_n = nullptr;
    t.ts = o->timestamps ? (unsigned long long*)o->timestamps + 1 + b->stars.size() : nullptr;
    if (o->precision == RT_PREC_MIXED) {
      e = cudaMemsetAsync(b->d_promo_n, 0, sizeof(unsigned long long), (cudaStream_t)stream);
      if (e == cudaSuccess) e = rtk::launch_batch_mixed(p, t, blk, bps, (cudaStream_t)stream);
      if (e != cudaSuccess) return cuda_fail(e, "mixed batch kernel");
      // FP64: the promoted rays from where they stopped, the listed pixels anew
      p.claim_status = rtk::RAY_PROMOTED;
      p.refill_min = p.claim_size = 1;
      t.list = b->d_promo;
      t.list_n = b->d_promo_n;
      e = rtk::launch_batch_fp64(p, t, 0, 0, (cudaStream_t)stream);
      if (e != cudaSuccess) return cuda_fail(e, "batch kernel (promoted rays and pixels)");
      return RT_OK;
    }
    e = rtk::launch_batch_fp64(p, t, blk, bps, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel");
    return RT_OK;
  }
  if (o->precision == RT_PREC_DF) {
    e = rtk::launch_trace_df(p, blk, bps, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "double-float trace kernel");
    return RT_OK;
  }
  if (o->precision == RT_PREC_MIXED) {
    e = rtk::launch_trace_mixed(p, blk, bps, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mixed trace kernel");
    p.claim_status = rtk::RAY_PROMOTED;
    p.refill_min = p.claim_size = 1;
    p.order = 0;
    p.xrec = nullptr;
    e = rtk::launch_trace_fp64(p, 0, 0, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "trace kernel (promoted rays)");
    return RT_OK;
  }
  e = rtk::launch_trace_fp64(p, blk, bps, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "trace kernel");
  return RT_OK;
}

}  // extern "C"

// The batch's binning scratch, grown when a larger histogram is requested
// (synchronises the stream before freeing the old one).
static rt_status ensure_batch_bins(rt_batch* b, int32_t nth, int32_t nph, int32_t nnu,
                                   void* stream) {
  const size_t per = rtk::bin_scratch_entries(nth, nph, nnu);
  if (per <= b->bins_per_star) return RT_OK;
  if (b->d_bins) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    cudaFree(b->d_bins);
    b->d_bins = nullptr;
    b->bins_per_star = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, per * b->stars.size() * sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail(RT_ENOMEM, "cannot allocate the batch binning scratch");
  }
  b->d_bins = (long long*)p;
  b->bins_per_star = per;
  return RT_OK;
}

extern "C" {

rt_status rt_bin_batch(rt_batch* b, const double* d_state, const double* d_weight,
                       const uint8_t* d_status, int32_t nth, int32_t nph, int32_t nnu,
                       double nu_lo, double nu_hi, double* d_hist, double* d_oor, void* stream) {
  rtk::NvtxRange nvtx_range("rt_bin_batch");
  if (!b) return fail(RT_EINVAL, "batch is NULL");
  if (nth < 1 || nph < 1 || nnu < 1) return fail(RT_EINVAL, "bin counts must be >= 1");
  if ((int64_t)nth * nph * nnu > (int64_t)1 << 28) return fail(RT_EINVAL, "too many bins");
  if (!is_finite_val(nu_lo) || !is_finite_val(nu_hi) || !(nu_hi > nu_lo))
    return fail(RT_EINVAL, "need finite nu_lo < nu_hi");
  rt_status st;
  if (b->N > 0) {
    if ((st = check_dev_ptr(d_state, "d_state")) != RT_OK) return st;
    if ((st = check_dev_ptr(d_weight, "d_weight")) != RT_OK) return st;
    if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  }
  if ((st = check_dev_ptr(d_hist, "d_hist")) != RT_OK) return st;
  if ((st = check_dev_ptr(d_oor, "d_out_of_range")) != RT_OK) return st;
  const size_t nst = b->stars.size();
  if ((st = ensure_batch_bins(b, nth, nph, nnu, stream)) != RT_OK) return st;
  const size_t nbins = (size_t)nth * nph * nnu;
  for (size_t s = 0; s < nst; ++s) {
    const int64_t o = b->off[s], cnt = b->off[s + 1] - o;
    rtk::BinParams p;
    p.R_km = b->stars[s]->h.R_km;
    p.rs_prop = b->stars[s]->h.rs_prop;
    p.v0 = b->stars[s]->h.v0;
    p.n = cnt;
    p.ld = b->N;
    p.n_scale = cnt;
    p.state = d_state + o;
    p.weight = d_weight + o;
    p.status = d_status + o;
    p.nth = nth;
    p.nph = nph;
    p.nnu = nnu;
    p.nu_lo = nu_lo;
    p.nu_hi = nu_hi;
    p.acc = b->d_bins + s * b->bins_per_star;
    p.hist = d_hist + s * nbins;
    p.sky = nullptr;
    p.spec = nullptr;
    p.oor = d_oor + s;
    cudaError_t e = rtk::launch_bin(p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "bin kernels");
  }
  return RT_OK;
}

rt_status rt_timestamps_reset(uint64_t* d_ts, int32_t n_instances, void* stream) {
  if (n_instances < 1) return fail(RT_EINVAL, "n_instances must be >= 1");
  rt_status st;
  if ((st = check_dev_ptr(d_ts, "d_timestamps")) != RT_OK) return st;
  cudaError_t e = rtk::launch_ts_reset((unsigned long long*)d_ts, n_instances,
                                       (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "timestamp reset");
  return RT_OK;
}

struct rt_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
};

rt_status rt_batch_graph_create(rt_batch* b, const double* d_u, double* d_state,
                                double* d_weight, uint8_t* d_status, int64_t* d_counters,
                                const rt_trace_opts* o, int32_t nth, int32_t nph, int32_t nnu,
                                double nu_lo, double nu_hi, double* d_hist, double* d_oor,
                                rt_graph** out) {
  if (!out) return fail(RT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!b) return fail(RT_EINVAL, "batch is NULL");
  if (b->N == 0) return fail(RT_EINVAL, "empty batch");
  rt_status st;
  if ((st = check_opts(o)) != RT_OK) return st;
  if (nth < 1 || nph < 1 || nnu < 1) return fail(RT_EINVAL, "bin counts must be >= 1");
  if ((st = ensure_batch_bins(b, nth, nph, nnu, nullptr)) != RT_OK) return st;
  if (o->tail != 1 && (st = ensure_park(&b->d_park, &b->park_cap)) != RT_OK) return st;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  // sample -> trace -> bin, as the individual calls would enqueue them
  st = RT_OK;
  if (d_counters) {
    e = cudaMemsetAsync(d_counters, 0, RT_COUNTERS * sizeof(int64_t), cs);
    if (e != cudaSuccess) st = cuda_fail(e, "counter reset");
  }
  if (st == RT_OK && o->timestamps)
    st = rt_timestamps_reset(o->timestamps, (int32_t)b->stars.size() + b->nimg, cs);
  if (st == RT_OK) {
    st = rt_sample_batch(b, d_u, d_state, d_weight, d_status, cs);
    if (st == RT_EEMPTY_SURFACE) st = RT_OK;
  }
  if (st == RT_OK) st = rt_trace_batch(b, d_state, d_status, nullptr, nullptr, d_counters, o, cs);
  if (st == RT_OK)
    st = rt_bin_batch(b, d_state, d_weight, d_status, nth, nph, nnu, nu_lo, nu_hi, d_hist,
                      d_oor, cs);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (st != RT_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  rt_graph* r = new (std::nothrow) rt_graph;
  if (!r) {
    cudaGraphExecDestroy(x);
    cudaGraphDestroy(g);
    return fail(RT_ENOMEM, "host allocation failed");
  }
  r->graph = g;
  r->exec = x;
  cudaGetDevice(&r->device);
  *out = r;
  return RT_OK;
}

rt_status rt_graph_launch(rt_graph* g, void* stream) {
  rtk::NvtxRange nvtx_range("rt_graph_launch");
  if (!g) return fail(RT_EINVAL, "graph is NULL");
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return RT_OK;
}

void rt_graph_destroy(rt_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

rt_status rt_batch_autotune(rt_batch* b, const double* d_state, const uint8_t* d_status,
                            const rt_trace_opts* o, int32_t rays_per_star, int32_t* block_out,
                            int32_t* bps_out, int32_t* refill_out, int32_t* claim_out,
                            double* ms_out, int32_t* ncand_out, double* cand_ms,
                            int32_t cand_cap, void* stream) {
  rtk::NvtxRange nvtx_range("rt_batch_autotune");
  if (!b) return fail(RT_EINVAL, "batch is NULL");
  rt_status st;
  if ((st = check_opts(o)) != RT_OK) return st;
  if (rays_per_star < 1) return fail(RT_EINVAL, "rays_per_star must be >= 1");
  if (b->N == 0 && b->npix == 0) return fail(RT_EINVAL, "empty batch");
  if (b->rigid) return fail(RT_EUNSUPPORTED, "the autotuner needs RT_ROTATION_SNAPSHOT stars");
  if (b->N > 0) {
    if ((st = check_dev_ptr(d_state, "d_state")) != RT_OK) return st;
    if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  }
  if (b->npix > 0 && o->lambda_max != 0.0)
    return fail(RT_EUNSUPPORTED, "lambda_max must be 0 for a batch with images");
  const bool mixed = (o->precision == RT_PREC_MIXED);
  const bool df = (o->precision == RT_PREC_DF);
  const bool img = (b->npix > 0);
  if (df && img)
    return fail(RT_EUNSUPPORTED, "a batch with images is traced in RT_PREC_FP64 or RT_PREC_MIXED");
  const size_t nst = b->stars.size();
  // the first rays_per_star rays of every star, in a batch of their own
  std::vector<int64_t> off(nst + 1, 0);
  for (size_t s = 0; s < nst; ++s) {
    const int64_t cnt = b->off[s + 1] - b->off[s];
    off[s + 1] = off[s] + (cnt < rays_per_star ? cnt : rays_per_star);
  }
  const int64_t M = off[nst];
  // coarse copies of the images: the same planes in at most side x side pixels
  const int side = (int)std::ceil(std::sqrt((double)rays_per_star));
  const int nimg = img ? b->nimg : 0;
  std::vector<rtk::BackParams> tbl((size_t)nimg);
  std::vector<int64_t> ioff((size_t)nimg + 1, 0);
  for (int j = 0; j < nimg; ++j) {
    const rt_image_desc& d = b->h_desc[j];
    const int nx = d.nx < side ? d.nx : side, ny = d.ny < side ? d.ny : side;
    ioff[j + 1] = ioff[j] + (int64_t)nx * ny;
  }
  const int64_t P = ioff[nimg];
  if (M + P == 0) return fail(RT_EINVAL, "nothing to tune on");
  cudaStream_t cs = (cudaStream_t)stream;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t b_st = al((size_t)RT_STATE_ROWS * M * sizeof(double));
  const size_t b_s = al((size_t)M);
  const size_t b_off = al((nst + 1) * sizeof(int64_t));
  const size_t b_tbl = al(sizeof(rtk::BackParams) * (size_t)nimg);
  const size_t b_ioff = al(((size_t)nimg + 1) * sizeof(int64_t));
  const size_t b_img = al((size_t)P * sizeof(double));
  const size_t b_ist = al((size_t)P);
  const size_t b_promo = al((size_t)(P > 0 ? P : 1) * sizeof(int32_t));
  const size_t bytes = 256 + 2 * b_st + 2 * b_s + b_off + b_tbl + b_ioff + b_img + b_ist + 256 +
                       b_promo;
  void* blk = nullptr;
  cudaError_t e = cudaMalloc(&blk, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RT_ENOMEM, "autotune scratch allocation failed");
  }
  char* q = (char*)blk;
  unsigned long long* queue = (unsigned long long*)q;
  q += 256;
  double* st0 = (double*)q;
  q += b_st;
  double* st1 = (double*)q;
  q += b_st;
  uint8_t* s0 = (uint8_t*)q;
  q += b_s;
  uint8_t* s1 = (uint8_t*)q;
  q += b_s;
  int64_t* doff = (int64_t*)q;
  q += b_off;
  rtk::BackParams* d_tbl = (rtk::BackParams*)q;
  q += b_tbl;
  int64_t* d_ioff = (int64_t*)q;
  q += b_ioff;
  double* d_iimg = (double*)q;
  q += b_img;
  uint8_t* d_ist = (uint8_t*)q;
  q += b_ist;
  unsigned long long* promo_n = (unsigned long long*)q;
  q += 256;
  int32_t* promo = (int32_t*)q;
  for (size_t s = 0; s < nst && e == cudaSuccess; ++s) {
    const int64_t m = off[s + 1] - off[s];
    if (m == 0) continue;
    for (int r = 0; r < RT_STATE_ROWS && e == cudaSuccess; ++r)
      e = cudaMemcpyAsync(st0 + r * M + off[s], d_state + r * b->N + b->off[s],
                          m * sizeof(double), cudaMemcpyDeviceToDevice, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s0 + off[s], d_status + b->off[s], m, cudaMemcpyDeviceToDevice, cs);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(doff, off.data(), (nst + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                        cs);
  for (int j = 0; j < nimg; ++j) {
    const rt_image_desc& d = b->h_desc[j];
    const rtk::StarDev& h = b->h_img_star[j]->h;
    rtk::BackParams& bp = tbl[j];
    memset(&bp, 0, sizeof(bp));
    bp.s = h;
    bp.nx = d.nx < side ? d.nx : side;
    bp.ny = d.ny < side ? d.ny : side;
    bp.incl = d.incl_rad;
    bp.D = d.dist_over_R;
    bp.bmax = d.bmax_over_R;
    image_setup(h, bp.nx, bp.ny, d.bmax_over_R, d.Lc_cut_km, &bp.W, &bp.img_scale, &bp.Lc_cut);
    bp.image = d_iimg + ioff[j];
    bp.status = d_ist + ioff[j];
    bp.ncross = nullptr;
  }
  if (e == cudaSuccess && nimg > 0)
    e = cudaMemcpyAsync(d_tbl, tbl.data(), sizeof(rtk::BackParams) * nimg,
                        cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && nimg > 0)
    e = cudaMemcpyAsync(d_ioff, ioff.data(), ioff.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) {
    cudaFree(blk);
    return cuda_fail(e, "autotune gather");
  }
  rtk::TraceParams p;
  p.stars = b->d_stars;
  p.nstars = (int)nst;
  p.offsets = doff;
  p.n = M;
  p.state = st1;
  p.status = s1;
  p.nacc = nullptr;
  p.nrej = nullptr;
  p.counters = nullptr;
  p.queue = queue;
  p.ts = nullptr;
  set_park(p, nullptr, 0, o);
  p.rtol = o->rtol;
  p.atol = o->atol;
  p.r_out = o->r_out_over_R;
  p.lambda_max = o->lambda_max;
  p.r_capture = o->r_capture_over_R;
  p.max_steps = o->max_steps;
  rtk::ImgTable t;
  t.img = d_tbl;
  t.off = d_ioff;
  t.nimg = nimg;
  t.npix = P;
  t.promo = promo;
  t.promo_n = promo_n;
  t.list = nullptr;
  t.list_n = nullptr;
  t.ts = nullptr;
  // first-stage candidates: block sizes the kernel's launch bounds allow, every
  // resident count
  std::vector<std::pair<int, int>> cand;
  const int blocks[3] = {mixed ? 64 : 32, mixed ? 128 : 64, mixed ? 256 : 128};
  for (int bi = 0; bi < 3; ++bi) {
    int occ = 0;
    e = img ? (mixed ? rtk::occupancy_batch_mixed(blocks[bi], &occ)
                     : rtk::occupancy_batch_fp64(blocks[bi], &occ))
            : (mixed ? rtk::occupancy_mixed(blocks[bi], &occ)
               : df  ? rtk::occupancy_trace_df(blocks[bi], &occ)
                     : rtk::occupancy_fp64(blocks[bi], &occ));
    if (e != cudaSuccess) break;
    for (int k = 1; k <= occ; ++k) cand.push_back({blocks[bi], k});
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  auto run = [&](int block, int bps, int refill, int claim, float* ms) -> cudaError_t {
    cudaError_t r = cudaSuccess;
    if (M > 0) {
      r = cudaMemcpyAsync(st1, st0, (size_t)RT_STATE_ROWS * M * sizeof(double),
                          cudaMemcpyDeviceToDevice, cs);
      if (r == cudaSuccess) r = cudaMemcpyAsync(s1, s0, M, cudaMemcpyDeviceToDevice, cs);
    }
    if (r == cudaSuccess && img) r = cudaMemsetAsync(promo_n, 0, sizeof(unsigned long long), cs);
    if (r == cudaSuccess) r = cudaEventRecord(ev0, cs);
    p.claim_status = rtk::RAY_READY;
    p.refill_min = refill;
    p.claim_size = claim;
    t.list = nullptr;
    t.list_n = nullptr;
    if (r == cudaSuccess) {
      if (img)
        r = mixed ? rtk::launch_batch_mixed(p, t, block, bps, cs)
                  : rtk::launch_batch_fp64(p, t, block, bps, cs);
      else
        r = mixed ? rtk::launch_trace_mixed(p, block, bps, cs)
            : df  ? rtk::launch_trace_df(p, block, bps, cs)
                  : rtk::launch_trace_fp64(p, block, bps, cs);
    }
    if (r == cudaSuccess && mixed) {
      // the FP64 pass over the promoted rays (and the handed-over pixels)
      p.claim_status = rtk::RAY_PROMOTED;
      p.refill_min = p.claim_size = 1;
      if (img) {
        t.list = promo;
        t.list_n = promo_n;
        r = rtk::launch_batch_fp64(p, t, 0, 0, cs);
      } else {
        r = rtk::launch_trace_fp64(p, 0, 0, cs);
      }
    }
    if (r == cudaSuccess) r = cudaEventRecord(ev1, cs);
    if (r == cudaSuccess) r = cudaEventSynchronize(ev1);
    if (r == cudaSuccess) r = cudaEventElapsedTime(ms, ev0, ev1);
    return r;
  };
  rt_batch::Tuned best;
  float best_ms = 3.0e38f, ms = 0.0f;
  int nc = 0;
  auto trial = [&](int block, int bps, int refill, int claim) -> cudaError_t {
    cudaError_t r = run(block, bps, refill, claim, &ms);
    if (r != cudaSuccess) return r;
    if (cand_ms && nc < cand_cap) cand_ms[nc] = ms;
    ++nc;
    if (ms < best_ms) {
      best_ms = ms;
      best.block = block;
      best.bps = bps;
      best.refill = refill;
      best.claim = claim;
    }
    return cudaSuccess;
  };
  if (e == cudaSuccess && !cand.empty()) e = run(cand[0].first, cand[0].second, 1, 1, &ms);
  for (size_t c = 0; c < cand.size() && e == cudaSuccess; ++c)
    e = trial(cand[c].first, cand[c].second, 1, 1);
  const int refills[4] = {2, 4, 8, 16}, claims[3] = {2, 4, 8};
  const rt_batch::Tuned shape = best;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i)
    e = trial(shape.block, shape.bps, refills[i], 1);
  const int refill = best.refill;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i)
    e = trial(shape.block, shape.bps, refill, claims[i]);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  cudaFree(blk);
  if (e != cudaSuccess) return cuda_fail(e, "autotune trial");
  b->tuned[mixed ? 1 : df ? 2 : 0][img ? 1 : 0] = best;
  if (block_out) *block_out = best.block;
  if (bps_out) *bps_out = best.bps;
  if (refill_out) *refill_out = best.refill;
  if (claim_out) *claim_out = best.claim;
  if (ms_out) *ms_out = best_ms;
  if (ncand_out) *ncand_out = nc;
  return RT_OK;
}

rt_status rt_count_status(int64_t n, const uint8_t* d_status, int64_t* counts, void* stream) {
  if (!counts) return fail(RT_EINVAL, "counts is NULL");
  for (int i = 0; i < RT_RAY_NSTATUS; ++i) counts[i] = 0;
  if (n < 0) return fail(RT_EINVAL, "n must be >= 0");
  if (n == 0) return RT_OK;
  rt_status st;
  if ((st = check_dev_ptr(d_status, "d_status")) != RT_OK) return st;
  std::vector<uint8_t> h((size_t)n);
  cudaError_t e = cudaMemcpyAsync(h.data(), d_status, (size_t)n, cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  for (int64_t i = 0; i < n; ++i) {
    if (h[i] >= RT_RAY_NSTATUS) return fail(RT_EINVAL, "invalid status %d at %lld", h[i], (long long)i);
    counts[h[i]]++;
  }
  if (counts[RT_RAY_MAXSTEPS] || counts[RT_RAY_NAN] || counts[RT_RAY_STIFF]) return RT_EPARTIAL;
  return RT_OK;
}

}  // extern "C"
