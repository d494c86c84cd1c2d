// Host-side declarations shared between the C ABI (rt_abi.cu) and the kernel
// translation units.  Not part of the public interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt.h"
#include "rt_device.cuh"
#include "rt_dual.cuh"
#include "rt_sample_core.cuh"

#include <nvtx3/nvToolsExt.h>

namespace rtk {

// NVTX range over a public entry point (the host-side enqueue of its
// kernels), named after the call, for timeline profilers; without an attached
// tool a push or pop is a check of one pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct TraceParams {
  const StarDev* stars;     // device array of nstars star descriptors
  int nstars;
  const int64_t* offsets;   // device, nstars + 1 ray offsets (unused when nstars == 1)
  int64_t n;
  double* state;
  uint8_t* status;
  int32_t* nacc;
  int32_t* nrej;
  int64_t* counters;
  unsigned long long* queue;  // scratch: next unclaimed ray
  double rtol, atol, r_out, lambda_max, r_capture;
  int max_steps;
  int claim_status;           // rays with this status are traced (READY, or PROMOTED)
  unsigned long long* ts;     // optional: [0] launch start (min), [1 + star] last finish (max)
  // tail mode (FP64): rays of warps left with <= PARK_LIVE_MAX rays once the
  // queue has drained are parked here and continued six lanes per ray
  double* park;               // park_cap entries of PARKREC doubles (NULL: no parking)
  unsigned long long* park_count;
  unsigned long long* park_next;
  int64_t park_cap;
  int park_live;              // park when a drained warp holds at most this many rays
  // claim order of the FP64 forward kernels: 0 = by index; 1 = by predicted
  // cost -- COST_BUCKETS passes over the queue, the first taking the rays that
  // start closest to the Goldreich-Julian null cone (the ones that can be
  // guided along it for tens of thousands of steps), so that the longest rays
  // run from the start of the launch instead of after the bulk
  int order = 0;
  // express lane (cost-ordered FP64 tracing in tail mode): the rays of cost
  // bucket 0, ranked by their distance from the null cone, become park records
  // that six-lane groups of the first block on each of the first SMs continue
  // from the start of the launch, while the other blocks trace the rest one
  // lane per ray (parking only when xpark is set); the tail launch takes any
  // record left over
  double* xrec = nullptr;               // xcap records of PARKREC doubles
  unsigned long long* xcount = nullptr;  // [0] candidates found, [1] next record
  int* xslot = nullptr;                 // per-SM arrival counter (XSLOTS ints)
  unsigned long long* xcand = nullptr;   // xcap (key, ray) pairs
  int64_t xcap = 0;
  // with the express lane the bulk parks its last rays for the tail launch only
  // in launches long enough that the express lane ends before the bulk (the
  // tail launch waits for both); shorter ones keep them one lane per ray
  int xpark = 0;
  // work claiming (claim_items): a warp refills once refill_min lanes wait;
  // a lane claims claim_size consecutive queue entries at a time
  int refill_min = 1;
  int claim_size = 1;
};
constexpr int64_t XPARK_MIN_RAYS = (int64_t)4 << 20;
constexpr int COST_BUCKETS = 3;
constexpr int PARKREC = 14;   // y[6], h, h_resume, sig, flags, na, nr, ray, lambda
constexpr int PARK_LIVE_MAX = 5;
constexpr int XSLOTS = 256;            // per-SM counters (more than any GPU's SMs)
constexpr int64_t XCAP = 8192;         // express records per launch
constexpr int XRAYS_PER_SM = 12;       // one six-lane group in warps 0-1, five in 2-3
// bytes of the express area: counters, per-SM slots, candidates, records
inline size_t express_bytes() {
  return 64 + XSLOTS * sizeof(int) + (size_t)XCAP * 2 * sizeof(unsigned long long) +
         (size_t)XCAP * PARKREC * sizeof(double);
}
// Park capacity that covers any persistent grid on the device (up to 31 rays
// per warp).
inline int64_t park_capacity(int nsm) { return (int64_t)nsm * (2048 / 32) * 31; }

// Per-call counters (int64): accepted steps, rejected steps, rays finished,
// rays escaped, rays promoted from FP32 to FP64, FP64 steps of promoted rays,
// resonance crossings counted by the backward tracer.
enum {
  CTR_ACC = 0, CTR_REJ, CTR_RAYS, CTR_ESC, CTR_PROMOTED, CTR_PROMOTED_STEPS, CTR_CROSS,
  CTR_COUNT = 8
};
// rt_trace_backward uses slot 5 for its FP64 extremum searches (grazing pairs)
constexpr int CTR_SEARCH = CTR_PROMOTED_STEPS;

struct SampleParams {
  StarDev s;
  int64_t n;                // samples
  int64_t ld;               // SoA row stride of u and state (>= n)
  int64_t n_norm;           // the weights are normalised by n_norm (n, or the
                            // samples of all shards of one workload)
  const double* u;
  double* state;
  double* weight;
  uint8_t* status;
};

struct BinParams {
  double R_km, rs_prop, v0; // the star's radius [km], r_s / R of propagation, v0 [c]
  int64_t n;
  int64_t ld;               // SoA row stride of state (>= n)
  int64_t n_scale;          // ray count that bounds the fixed-point sums (n, or the
                            // rays of all shards of a sharded binning)
  const double* state;
  const double* weight;
  const uint8_t* status;
  int nth, nph, nnu;
  double nu_lo, nu_hi;
  long long* acc;           // scratch: [0] max weight bits, [1] out of range, hist, sky, spec
  double* hist;
  double* sky;
  double* spec;
  double* oor;
};

cudaError_t launch_sample(const SampleParams& p, cudaStream_t stream);
// Forward tracing through a rigidly rotating magnetosphere (rt_trace_rot.cu).
cudaError_t launch_trace_rot(const TraceParams& p, int block, int blocks_per_sm,
                             cudaStream_t stream);
cudaError_t launch_trace_fp64(const TraceParams& p, int block, int blocks_per_sm,
                              cudaStream_t stream);
cudaError_t launch_trace_mixed(const TraceParams& p, int block, int blocks_per_sm,
                               cudaStream_t stream);
cudaError_t launch_tail_fp64(const TraceParams& p, cudaStream_t stream);
// Binning: launch_bin = clear p.acc, then the three phases; the phases alone
// serve the sharded binning (rt_bin_part_*), whose callers reduce p.acc
// between them.
cudaError_t launch_bin(const BinParams& p, cudaStream_t stream);
cudaError_t launch_bin_max(const BinParams& p, cudaStream_t stream);
cudaError_t launch_bin_accum(const BinParams& p, cudaStream_t stream);
cudaError_t launch_bin_finalize(const BinParams& p, cudaStream_t stream);
// Resident blocks per SM of the trace kernels at a block size.
cudaError_t occupancy_fp64(int block, int* occ);
cudaError_t occupancy_mixed(int block, int* occ);
cudaError_t occupancy_batch_fp64(int block, int* occ);
cudaError_t occupancy_batch_mixed(int block, int* occ);
// Forward tracing in double-float (rt_trace_df.cu)
cudaError_t launch_trace_df(const TraceParams& p, int block, int blocks_per_sm,
                            cudaStream_t stream);
cudaError_t occupancy_trace_df(int block, int* occ);

// Backward image-plane tracing (one ray per pixel, ny x nx row-major).
struct BackLaunch {
  const StarDev* star;      // host descriptor (copied into the kernel parameters)
  int nx, ny;
  double incl;              // inclination of the line of sight from the rotation axis [rad]
  double D;                 // plane distance / R
  double bmax;              // half-width of the plane / R
  double W;                 // omega_inf / m_a traced
  double Lc_cut;            // conversion-length cut / R (0: none)
  double img_scale;         // multiplies each pixel's crossing sum
  double rtol, atol, r_capture;
  int max_steps;
  double* image;
  uint8_t* status;
  int32_t* ncross;
  int64_t* counters;
  unsigned long long* queue;
  unsigned long long* ts;     // optional: [0] start (min), [1] last pixel finished (max)
  int prec;                   // PREC_FP64, or PREC_MIXED (FP32 stages; FP64 pass for the
                              // pixels listed in promo, count in *promo_n)
  int32_t* promo;
  unsigned long long* promo_n;
};
cudaError_t launch_backward(const BackLaunch& b, cudaStream_t stream);
cudaError_t launch_ts_reset(unsigned long long* ts, int n, cudaStream_t stream);

// Adjoint of the line-flux functional (rt_adjoint.cu).  Parameters, in
// order: m_a [eV], B0 [G], theta_m [rad], M [Msun], R [km], inclination [rad];
// the first NSAMP_TANGENTS move the sampling.
enum { PREC_FP64 = 0, PREC_MIXED = 1, PREC_DF = 2 };   // the values of RT_PREC_*
enum { PAR_MA = 0, PAR_B0, PAR_THM, PAR_M, PAR_R, PAR_INCL, NPARAMS };
constexpr int NSAMP_TANGENTS = 5;
constexpr int CK = 32;        // accepted steps per checkpoint
constexpr int CKREC = 13;     // doubles per checkpoint: y, h, h_resume, sig, flags, counts
// doubles per accepted step of a segment replay: y[6], h, sig, flags, spare,
// and the step's seven stage derivatives K[7][6]
constexpr int SEGREC = 10 + 7 * 6;
// The full step tape (every accepted step of every ray held in device memory
// at once, SEGREC doubles each): a ray with nacc forward steps gets
// tape_slots(nacc) records, the last free one taking its final state.
__host__ __device__ inline int64_t tape_slots(int32_t nacc) {
  const int64_t a = nacc > 0 ? nacc : 0;
  return a + a / 64 + 9;
}
// Per-ray head of the tape: the adjoint seed at the escape point (6), its
// r_s part, K, dm/dtheta_m (3), the number of records (-1: no gradient), the
// sampling tangents (5 x (x 3, k 3, w)), omega_inf^2, its inverse, m (3), the
// initial state (6) and the weight.
constexpr int HEADREC = 60;
enum {
  HD_YBAR = 0, HD_RSBAR = 6, HD_K = 7, HD_DM = 8, HD_NREC = 11, HD_TAN = 12, HD_W2 = 47,
  HD_IW2 = 48, HD_M = 49, HD_Y0 = 52, HD_W = 58
};

struct AdjLaunch {
  const StarDev* star;                          // host descriptor
  sampling::SampConst<Dual<NSAMP_TANGENTS>> sc;  // sampling constants with p-tangents
  double drsp_dM, drsp_dR, dcp_dma, dcp_dB0;
  double incl, kappa, knorm;
  double rtol, atol, r_out, r_capture;
  int max_steps;
  int64_t n;
  const double* u;
  const int64_t* ck_off;
  double* ck;
  double* seg;
  // full-tape mode: tape_off[i] = first record of ray i; head: HEADREC
  // doubles per ray; order: the rays, longest first (n), built from nacc with
  // the 32 counters of bucket
  const int64_t* tape_off;
  double* tape;
  double* head;
  const int32_t* nacc;
  int64_t* order;
  unsigned long long* bucket;
  double* F_ray;
  double* G_ray;
  uint8_t* status;
  int32_t* flags;
  int64_t* counters;
  unsigned long long* queue;
  double* grad;    // NPARAMS
  double* F;       // 1
  int prec;        // reverse sweep in PREC_FP64, PREC_MIXED (FP32) or PREC_DF (double-float)
  int grid, block;
};
cudaError_t launch_flux_value(const StarDev* d_star, int64_t n, const double* state,
                              const double* weight, const uint8_t* status, double incl,
                              double kappa, double knorm, double* F_ray, double* F_total,
                              cudaStream_t stream);
cudaError_t launch_ck_offsets(const int32_t* nacc, int64_t n, int64_t* off, cudaStream_t stream);
cudaError_t launch_tape_offsets(const int32_t* nacc, int64_t n, int64_t* off, cudaStream_t stream);
// the full-tape gradient: longest-first order, tape kernel, sweep kernel, sums
cudaError_t launch_adjoint_tape(const AdjLaunch& a, cudaStream_t stream);
cudaError_t adjoint_grid(int prec, int* grid, int* block);
cudaError_t launch_adjoint(const AdjLaunch& a, cudaStream_t stream);

// Sets the thread-local message returned by rt_last_error().
void set_last_error(const char* msg);

// Argument checks shared by the entry points (rt_abi.cu); on failure they set
// the message of rt_last_error() and return RT_EINVAL / RT_EUNSUPPORTED.
// check_device_array: p is device (or managed) memory of the current device.
rt_status check_device_array(const void* p, const char* name);
// check_star_params: the validation of rt_init_star (finite values, R above
// the Schwarzschild radius, 0 < v0 < c, known model switches, ...).
rt_status check_star_params(const rt_star_params* p);
// The host copy of a handle's derived constants.
const StarDev& star_host_desc(const rt_star* s);

// Number of int64 scratch entries rt_bin_spectrum needs.
inline size_t bin_scratch_entries(int nth, int nph, int nnu) {
  return 2 + (size_t)nth * nph * nnu + (size_t)nth * nph + (size_t)nnu;
}

}  // namespace rtk
