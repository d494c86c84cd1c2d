/*
 * rt.h - C ABI of the GB300 (sm_103a) batched Hamiltonian ray tracer for
 * photons produced by resonant axion-photon conversion in a neutron-star
 * magnetosphere (J. I. McDonald and S. J. Witte, "Generalized Ray Tracing for
 * Axions in Astrophysical Plasmas", arXiv:2309.08655).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All arrays are caller-owned DEVICE pointers (any CUDA allocation on the
 *   current device), accessed on the caller's stream `stream` (a
 *   cudaStream_t passed as void*; NULL = legacy default stream).  Calls are
 *   asynchronous unless stated otherwise; they return after enqueueing work.
 * - Ray state is structure-of-arrays, RT_STATE_ROWS x n float64, row r of ray
 *   i at state[r * n + i]:
 *     rows 0-2  x^i, Cartesianised Schwarzschild position [km]
 *     rows 3-5  k_i, covariant Cartesian momentum [eV]
 *     row  6    delta = omega_inf / m_a - 1, with k_t = -omega_inf conserved
 *     row  7    psi, rotation phase of the frozen magnetosphere [rad]
 * - Per-ray status is one uint8 per ray (RT_RAY_*).
 * - Errors: functions return rt_status and never abort.  Argument errors
 *   return RT_EINVAL, an unsupported option RT_EUNSUPPORTED, CUDA errors
 *   (launch failures, or an earlier asynchronous fault surfacing)
 *   RT_ECUDA; rt_last_error() then returns a thread-local message.  Per-ray
 *   problems are reported in the status array, not by the return value.
 * - Thread safety: rt_star handles are immutable after rt_init_star and may
 *   be used from several host threads, except that rt_bin_spectrum calls
 *   sharing one handle must be serialised on one stream (they share the
 *   handle's scratch accumulator).
 */
#ifndef RT_AXION_H
#define RT_AXION_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RT_STATE_ROWS 8
#define RT_UNIFORM_ROWS 6
#define RT_COUNTERS 8

typedef enum {
  RT_OK = 0,
  RT_EINVAL = 1,
  RT_ENOMEM = 2,
  RT_ECUDA = 3,
  RT_EEMPTY_SURFACE = 4,  /* the resonance cannot exist anywhere outside the star */
  RT_EPARTIAL = 5,        /* returned by rt_count_status when some rays hit a bound */
  RT_EUNSUPPORTED = 6
} rt_status;

/* Per-ray status codes. */
enum {
  RT_RAY_READY = 0,      /* sampled, not yet traced */
  RT_RAY_ESCAPED = 1,    /* reached r = r_out (located exactly on the dense output) */
  RT_RAY_CAPTURED = 2,   /* reached r <= r_capture (the stellar surface) */
  RT_RAY_NO_ROOT = 3,    /* no resonance on this sample's radial line (weight 0) */
  RT_RAY_MAXSTEPS = 4,   /* max_steps accepted steps (or 4 x max_steps attempts) */
  RT_RAY_NAN = 5,        /* non-finite state or error estimate */
  RT_RAY_STIFF = 6,      /* step size fell below 1e-12 (units of R) */
  RT_RAY_LAMBDA_END = 7, /* reached lambda_max (only when lambda_max > 0) */
  RT_RAY_NSTATUS = 8
};

/* Model switches. */
enum { RT_DISP_ANISO = 0, RT_DISP_ISO = 1 };
enum { RT_RES_KINEMATIC = 0 };
enum { RT_FA_MAXWELL = 0, RT_FA_DELTA = 1 };
enum { RT_WEIGHT_PAG = 0, RT_WEIGHT_UNIT_P = 1, RT_WEIGHT_RENORM = 2 };
enum { RT_METRIC_FULL = 0, RT_METRIC_FLAT = 1 };
enum { RT_PHASE_FIXED = 0, RT_PHASE_UNIFORM = 1 };
enum { RT_ROTATION_SNAPSHOT = 0, RT_ROTATION_RIGID = 1 };
enum {
  RT_PLASMA_GJ = 0, RT_PLASMA_VACUUM = 1, RT_PLASMA_HOMOG = 2, RT_PLASMA_LINEAR_Z = 3,
  RT_PLASMA_RADIAL = 4, RT_PLASMA_TWISTED = 5
};
enum { RT_PREC_FP64 = 0, RT_PREC_MIXED = 1, RT_PREC_DF = 2 };
enum { RT_CLAIM_INDEX = 0, RT_CLAIM_COST = 1 };

/*
 * Star, plasma and axion parameters (Sec. 5 fiducials; Eq. GJDensity).
 *   M_sun          stellar mass [solar masses]; r_s = 2 G M / c^2
 *   R_km           stellar radius [km]; also the unit of length inside kernels
 *   B0_G           dipole field at the magnetic pole of the surface [G]
 *   P_s            rotation period [s] (sets Omega in n_GJ = 2 Omega.B / e)
 *   theta_m_rad    misalignment of the magnetic axis from the rotation axis z
 *   psi_rad        rotation phase used when phase_mode == RT_PHASE_FIXED
 *   m_a_eV         axion mass [eV]; also the unit of momentum inside kernels
 *   g_agg_GeVinv   axion-photon coupling [GeV^-1]
 *   rho_dm_GeV_cm3 asymptotic dark-matter density; n_inf = rho / m_a
 *   v0_kms         Maxwellian dispersion, f ~ exp(-|k|^2 / (m_a v0)^2)
 *   dispersion     RT_DISP_ANISO (Eq. StrongBHam) or RT_DISP_ISO (Eq. DispIsotropic)
 *   resonance      RT_RES_KINEMATIC (k^a_mu = k^gamma_mu)
 *   fa_model       RT_FA_MAXWELL (Eq. GaussianDist) or RT_FA_DELTA (|k_inf| = m_a v0)
 *   weight_mode    RT_WEIGHT_PAG (conversion probability, Eq. CPAnisoCurved), or
 *                  RT_WEIGHT_UNIT_P (the probability set to one, Sec. 5.1: each
 *                  weight divided by P_agamma = Psi / |k . dE|, dE the proper-frame
 *                  gradient of E_gamma - E_a, i.e. the axion energy flux through
 *                  the conversion surface), or RT_WEIGHT_RENORM (that, times
 *                  R_i = (1 cm^-3 / n_a(r_i)) (m_a / |k_a|) / sqrt(1 - r_s / r_i) of
 *                  Eq. reweight, n_a = n_inf k_c / k0 the focused density of
 *                  Sec. 4.3); forward sampling only -- the backward tracer and
 *                  the gradient reject both)
 *   prop_metric    RT_METRIC_FULL, or RT_METRIC_FLAT (M = 0 in propagation only)
 *   phase_mode     RT_PHASE_FIXED or RT_PHASE_UNIFORM (psi = 2 pi u5 per sample)
 *   plasma         RT_PLASMA_GJ (Eq. GJDensity), RT_PLASMA_TWISTED (the twisted
 *                  magnetar magnetosphere of Sec. 6, Eq. neMag: n_e = lambda psi
 *                  sin^2(theta) B0 (R/r)^3 / (e r), theta the magnetic colatitude,
 *                  dipole field kept for B; no conversion on open field lines,
 *                  r / sin^2(theta) >= c / Omega: such samples get RT_RAY_NO_ROOT
 *                  and weight 0); the others are analytic test media
 *   plasma_a       TWISTED: lambda psi (charge multiplicity x twist angle [rad],
 *                  > 0); omega_p^2 / m_a^2 (HOMOG), its gradient d/d(z/R)
 *                  (LINEAR_Z), or its value at r = R of the spherical profile
 *                  a (R/r)^3 (RADIAL)
 *   rotation       RT_ROTATION_SNAPSHOT: the magnetosphere frozen at the emission
 *                  phase for the whole flight, k_t conserved.  RT_ROTATION_RIGID:
 *                  it keeps turning about z at Omega = 2 pi / P_s while the photon
 *                  flies (the cos(Omega t) of Eq. GJDensity), so k_t evolves (Eq.
 *                  Hamilton for all four canonical pairs) and the line is Doppler
 *                  shifted; sampling is unchanged (the snapshot at emission).
 *                  rt_trace_forward traces it in RT_PREC_FP64 only (one lane per
 *                  ray throughout), and on return state row 6 holds the final
 *                  omega_inf / m_a - 1 and row 7 the rotation phase psi0 + Omega t
 *                  at the end point.  The backward tracer, backward images
 *                  and the gradient reject it (RT_EUNSUPPORTED); a batch takes
 *                  it when all its stars do.  Before this field existed
 *                  it was reserved and ignored; 0 keeps that behaviour.
 */
typedef struct {
  double M_sun, R_km, B0_G, P_s, theta_m_rad, psi_rad, m_a_eV, g_agg_GeVinv, rho_dm_GeV_cm3,
      v0_kms;
  int32_t dispersion, resonance, fa_model, weight_mode, prop_metric, phase_mode, plasma,
      rotation;
  double plasma_a;
} rt_star_params;

/*
 * Integration options (adaptive Dormand-Prince 5(4), Sec. 2.4's "high
 * precision ODE solvers").
 *   rtol, atol        tolerances on the state scaled to x/R and k/m_a
 *   r_out_over_R      escape radius (event located on the dense output)
 *   lambda_max        stop at this worldline parameter (units: R / m_a^2 scaled
 *                     Hamiltonian); 0 = no limit
 *   r_capture_over_R  capture radius (1 = stellar surface)
 *   precision         RT_PREC_FP64, RT_PREC_MIXED or RT_PREC_DF (RT_PREC_DF:
 *                     rt_trace_forward, rt_trace_batch without images, and the
 *                     backward sweep of rt_flux_gradient)
 *   max_steps         bound on accepted steps per ray
 *   block             threads per block of the persistent kernel (0 = auto, or
 *                     the batch's autotuned value, rt_batch_autotune)
 *   blocks_per_sm     resident blocks per SM for the persistent grid (0 = auto)
 *   tail              0: FP64 tracing parks the rays of warps left with at most 5
 *                     rays once the queue has drained and continues them six lanes
 *                     per ray (one lane per state component); results agree with
 *                     the one-lane-per-ray path to rounding.  2-31: the same with
 *                     that many rays as the threshold.  1: one lane per ray
 *                     throughout.  The handle owns the park buffer (allocated on
 *                     first use, 33 MB on GB300).
 *   claim_order       RT_CLAIM_INDEX (0): rays are claimed in index order.
 *                     RT_CLAIM_COST (1): the forward kernels (FP64 and the FP32
 *                     stages of RT_PREC_MIXED) claim rays by
 *                     predicted cost -- first those that start within 1e-3 rad,
 *                     then 1e-2 rad, of the Goldreich-Julian null cone (the rays
 *                     that can be guided along it for tens of thousands of
 *                     steps), then the rest -- so that the longest rays run from
 *                     the start of the launch.  In tail mode (tail != 1) the
 *                     rays within 1e-3 rad (up to 8192 per call, nearest first)
 *                     of an FP64 call are traced six lanes per ray from the start on a few SMs
 *                     of their own (the express lane), and the others one lane
 *                     per ray (parking their last rays only in calls of 4M rays
 *                     or more); results agree with index order to rounding and
 *                     are bitwise reproducible below 4M rays (unless more than
 *                     8192 rays qualify).  Not with images in a batch.
 *   refill_min        work claiming of the persistent kernels: a warp claims new
 *                     rays (pixels) from the global queue once at least this many of
 *                     its lanes are free (1-32; 0 = auto: the batch's autotuned
 *                     value, else 8 for RT_PREC_FP64 and 16 for RT_PREC_DF and
 *                     RT_PREC_MIXED, measured on the benchmark's eight-step
 *                     launch; 1 refills as soon as any lane is free)
 *   rays_per_claim    queue entries a lane claims at a time (1-64; 0 = auto, as
 *                     refill_min); a lane traces its claimed rays one after the
 *                     other before it claims again.  Neither changes any ray's
 *                     result with one lane per ray (tail = 1); in tail mode the
 *                     set of rays that end in the six-lane kernel may change
 *   timestamps        NULL, or a device array of 1 + (number of instances) uint64
 *                     that the kernels stamp with the GPU's nanosecond global
 *                     timer: [0] the earliest start of a tracing launch (min),
 *                     [1 + s] the moment the last ray (pixel) of instance s
 *                     finished (max; s = the star's index in a batch, 0 for a
 *                     single star or an image).  Reset with rt_timestamps_reset;
 *                     per-instance latency = [1 + s] - [0].
 */
typedef struct {
  double rtol, atol, r_out_over_R, lambda_max, r_capture_over_R;
  int32_t precision, max_steps, block, blocks_per_sm, tail, claim_order;
  uint64_t* timestamps;
  int32_t refill_min, rays_per_claim;
} rt_trace_opts;

/* rt_timestamps_reset - [0] = UINT64_MAX, [1..n_instances] = 0, on stream. */
rt_status rt_timestamps_reset(uint64_t* d_timestamps, int32_t n_instances, void* stream);

typedef struct rt_star rt_star; /* opaque, library-owned */

/*
 * rt_init_star - validate parameters and build a star handle (host only;
 * allocates the handle and a small device block).  Derived constants follow
 * Sec. 5 (Eq. GJDensity) and Sec. 4.1 (Eq. SchwarzshildMetric1).
 * Returns RT_EINVAL on non-finite or out-of-range parameters (R <= r_s,
 * m_a <= 0, ...), RT_EUNSUPPORTED on unknown model switches.  *out is NULL on
 * error.  The handle is bound to the device current at this call.
 */
rt_status rt_init_star(const rt_star_params* params, rt_star** out);
void rt_destroy_star(rt_star* star);

/*
 * rt_star_info - derived constants of a handle (host, synchronous), in
 * out[0..7]: r_s/R, omega_p^2 coefficient / m_a^2 (omega_p^2 / m_a^2 =
 * c r^-3 |3 cos th (m.n) - cos th_m|, r in units of R), B0 [eV^2], R [eV^-1],
 * n_inf [eV^3], v0 [c], maximum omega_p^2 / m_a^2 on the surface, and 1 if the
 * resonance surface is empty for every direction (else 0).
 */
rt_status rt_star_info(const rt_star* star, double* out8);

/*
 * rt_sample_conversion_surface - forward Monte-Carlo samples of the
 * resonant conversion surface and their power weights (Sec. 3, Eq.
 * ForwardTracingEquation1; Sec. 4.2, Eq. PowerCurved with Eq. CPAnisoCurved
 * and Eq. AngleDefAniso; Sec. 4.3, Eq. GaussianDist).
 *   n           number of samples (>= 0); the weights are normalised by n
 *   d_uniforms  RT_UNIFORM_ROWS x n float64 in (0, 1), SoA: rows 0-1 the
 *               direction of the conversion point (cos th = 1 - 2u0,
 *               phi = 2 pi u1), rows 2-3 the momentum direction in the
 *               static orthonormal frame, row 4 the Maxwellian speed
 *               (inverse CDF), row 5 the rotation phase (phase_mode UNIFORM)
 *   d_state     out: RT_STATE_ROWS x n initial photon states
 *   d_weight    out: n power weights [W]; the sum over samples estimates
 *               the total power; 0 for samples without a resonance
 *   d_status    out: RT_RAY_READY or RT_RAY_NO_ROOT
 * The resonance r_k is found in FP64 on the radial line through the sampled
 * direction, with the momentum direction and omega_inf held fixed.
 */
rt_status rt_sample_conversion_surface(const rt_star* star, int64_t n, const double* d_uniforms,
                                       double* d_state, double* d_weight, uint8_t* d_status,
                                       void* stream);

/*
 * rt_sample_conversion_surface_part - rt_sample_conversion_surface for one
 * part of a larger Monte-Carlo sample: the n samples drawn from d_uniforms
 * are normalised by n_norm (the samples of the whole workload, >= n) instead
 * of n.  The weights of contiguous parts sampled by different processes (one
 * GPU each) are then bitwise those of one call over all n_norm samples.  The
 * paper's tracers run on computing clusters (Sec. 2.4); this is how one
 * workload's rays are split across GPUs (with rt_bin_part_*).
 * RT_EINVAL if n_norm < max(n, 1); otherwise as rt_sample_conversion_surface
 * (rt_sample_conversion_surface is this call with n_norm = n).
 */
rt_status rt_sample_conversion_surface_part(const rt_star* star, int64_t n, int64_t n_norm,
                                            const double* d_uniforms, double* d_state,
                                            double* d_weight, uint8_t* d_status, void* stream);

/*
 * rt_trace_forward - integrate Hamilton's equations (Eq. Hamilton) of the
 * strong-field Hamiltonian (Eq. StrongBHam) for every ray whose status is
 * RT_RAY_READY, in place, until escape, capture or a bound (Sec. 2.2).
 * One GPU thread per ray in a persistent kernel whose warps refill finished
 * lanes from a global queue.
 *   d_state    in/out: RT_STATE_ROWS x n; on escape the state at r = r_out
 *   d_status   in/out: READY rays get their final status; others untouched
 *   d_nacc, d_nrej  out (may be NULL): accepted / rejected steps per ray
 *   d_counters in/out (may be NULL): RT_COUNTERS int64 accumulated with
 *              atomics: accepted steps, rejected steps, rays finished, rays
 *              escaped, rays promoted from FP32 to FP64, step attempts of the
 *              promoted rays in FP64, 2 reserved
 *   opts       integration options (host pointer, read during the call)
 * RT_PREC_FP64: every stage in FP64; deterministic (bitwise identical outputs
 * for identical inputs) with the default claim order.  RT_PREC_MIXED: the
 * stages and their combinations run in FP32 and the state accumulates in
 * double-float (two floats, ~48 significant bits; no FP64 arithmetic per
 * step); where the FP32 rounding floor of
 * the embedded error estimate reaches a quarter of the tolerance on a rejected
 * step, the ray continues in FP64 from that point (a second kernel on the same
 * stream).  Use rtol >= 1e-8 with RT_PREC_MIXED; lambda_max must be 0.
 * RT_PREC_DF: the FP64 integrator's steps, events and decisions with every
 * operation in double-float arithmetic on the FP32 pipe (a value is the sum
 * of two floats, ~48 significant bits; an FP64 operation on this GPU issues
 * at 1/64 of the FP32 rate): FP64-class results at a fraction of the cost;
 * one lane per ray (tail ignored), claim_order honoured; lambda_max must be
 * 0; not for rotating stars.
 * Calls sharing one handle must be serialised on one stream (the handle owns
 * the work-queue counter).
 */
rt_status rt_trace_forward(const rt_star* star, int64_t n, double* d_state, uint8_t* d_status,
                           int32_t* d_nacc, int32_t* d_nrej, int64_t* d_counters,
                           const rt_trace_opts* opts, void* stream);

/*
 * rt_bin_spectrum - sky map and spectrum of ESCAPED rays (Sec. 2.2: the
 * power of the rays landing in a bin of the sphere at infinity).  Sky
 * direction = direction of the orthonormal-frame momentum at the end point:
 * theta uniform on [0, pi] (nth bins; theta = pi goes to the last bin), phi
 * on [0, 2 pi) (nph bins).  Frequency variable y = delta / (v0^2 / 2) on
 * [nu_lo, nu_hi) (nnu bins); rays outside add to *d_out_of_range.
 *   d_hist  out: nth x nph x nnu float64 [W per bin], row-major
 *   d_sky   out (may be NULL): nth x nph, the sum over frequency
 *   d_spec  out (may be NULL): nnu, the sum over the sky
 *   d_out_of_range out: 1 float64
 * Sums are accumulated in 64-bit fixed point (scale 2^e chosen from the
 * largest escaped weight so that no sum can overflow) and are therefore
 * independent of the order of the atomics.  Uses a scratch accumulator owned
 * by the handle (allocated on first use, grown when a larger histogram is
 * requested; RT_ENOMEM if that fails).
 */
rt_status rt_bin_spectrum(const rt_star* star, int64_t n, const double* d_state,
                          const double* d_weight, const uint8_t* d_status, int32_t nth,
                          int32_t nph, int32_t nnu, double nu_lo, double nu_hi, double* d_hist,
                          double* d_sky, double* d_spec, double* d_out_of_range, void* stream);

/*
 * Sharded binning: rt_bin_spectrum split into its three phases around
 * caller-owned int64 fixed-point sums, so that the sums of several shards
 * (processes, one GPU each, holding contiguous ranges of one workload's rays;
 * Sec. 2.4's cluster parallelisation) combine exactly by integer addition.
 *   d_acc  device int64 array of RT_BIN_ACC_ENTRIES(nth, nph, nnu) entries:
 *          [0] bit pattern of the largest escaped weight, [1] out-of-range
 *          sum, then the nth x nph x nnu histogram, the nth x nph sky map and
 *          the nnu spectrum, all in units of 2^-e.
 *   rt_bin_part_max         clears d_acc and sets d_acc[0] to the IEEE-754
 *                           bit pattern of the largest weight among the n
 *                           rays' ESCAPED ones (0 if none).  Then reduce
 *                           d_acc[0] with MAX over the shards (for
 *                           non-negative doubles int64 order is value order).
 *   rt_bin_part_accumulate  adds the n rays to d_acc[1 ..] with the scale 2^e
 *                           that the reduced d_acc[0] and n_total (the rays
 *                           of all shards, >= n) fix; d_state is
 *                           RT_STATE_ROWS x ld (row stride ld >= n, e.g. one
 *                           star's slice of a batch).  Then reduce
 *                           d_acc[1 ..] with SUM over the shards.
 *   rt_bin_part_finalize    the float64 outputs of rt_bin_spectrum from the
 *                           reduced sums (the same n_total).
 * The outputs are bitwise those of rt_bin_spectrum over the n_total rays of
 * all shards (one shard with all rays: bitwise rt_bin_spectrum).  The three
 * calls are asynchronous on stream, allocate nothing, and need device memory
 * of the current device for every array (RT_EINVAL otherwise).
 */
#define RT_BIN_ACC_ENTRIES(nth, nph, nnu) \
  (2 + (int64_t)(nth) * (nph) * (nnu) + (int64_t)(nth) * (nph) + (int64_t)(nnu))
rt_status rt_bin_part_max(int64_t n, const double* d_weight, const uint8_t* d_status,
                          int32_t nth, int32_t nph, int32_t nnu, int64_t* d_acc, void* stream);
rt_status rt_bin_part_accumulate(const rt_star* star, int64_t n, int64_t ld, int64_t n_total,
                                 const double* d_state, const double* d_weight,
                                 const uint8_t* d_status, int32_t nth, int32_t nph, int32_t nnu,
                                 double nu_lo, double nu_hi, int64_t* d_acc, void* stream);
rt_status rt_bin_part_finalize(int32_t nth, int32_t nph, int32_t nnu, int64_t n_total,
                               const int64_t* d_acc, double* d_hist, double* d_sky,
                               double* d_spec, double* d_out_of_range, void* stream);

/*
 * rt_trace_backward - image of the axion-induced radio power on a plane far
 * from the star, by backward ray tracing (Sec. 2.1, Eq. BackPower; every
 * resonance crossing counted, Sec. 5.1.3).  By Liouville's theorem the
 * phase-space integral of the forward method equals, per solid angle of the
 * observer, the integral over the plane of the frequency-integrated emission
 * along each ray reaching it.  Pixel (i, j) of an ny x nx grid (row-major, j
 * slow) is the square of side 2 b_max / nx by 2 b_max / ny centred on
 * b = (-b_max + (i + 1/2) db_x, -b_max + (j + 1/2) db_y) on the plane
 * through D o, o = (sin incl, 0, cos incl) the direction to the observer
 * (rotation axis z, magnetic axis at the star's fixed phase psi_rad), plane
 * axes e1 = (cos incl, 0, -sin incl) and e2 = (0, 1, 0).  Its ray leaves the
 * plane along -o with the on-shell momentum at the line centre omega_inf =
 * m_a sqrt(1 + v0^2), is integrated (FP64 DP5(4), opts->rtol/atol,
 * max_steps) until it returns to its starting radius or is captured, and at
 * every crossing of g = E_gamma - E_a = omega - sqrt(m_a^2 + |k|^2) = 0
 * along it adds sqrt(A) Psi |dt/dl| / |dg/dl|.  Crossings are searched on
 * each accepted step's continuous extension, cut into 16 pieces: a sign
 * change of g across a piece, and, where the ray grazes the resonance, the
 * two roots around an extremum of g inside a piece whose ends share a sign
 * (the extremum bracketed by the slope of g along the step and located by
 * bisection); every root is located by FP64 bisection.
 * The pixel value is that sum x pixel area x int domega omega^2 f_a
 * (omega_0 n_inf / (2 pi^{3/2} k0) for the Maxwellian, omega_0 n_inf /
 * (4 pi k0) for the monochromatic distribution): dP/dOmega in W / sr.
 * Crossings whose conversion length E / |dg/ds| (s: proper length) exceeds
 * Lc_cut_km are dropped when Lc_cut_km > 0 (the IR cut, Sec. 4.4).
 *   nx, ny        pixels per side (>= 1, nx * ny <= 2^31)
 *   incl_rad      observer inclination from the rotation axis [rad]
 *   dist_over_R   plane distance / R (> bmax_over_R * sqrt(2) + 1)
 *   bmax_over_R   half-width of the plane / R (> 0)
 *   d_image       out: ny x nx float64 [W / sr]
 *   d_status      out: ny x nx final ray status (RT_RAY_ESCAPED normally)
 *   d_ncross      out (may be NULL): ny x nx crossings counted (after the cut)
 *   d_counters    in/out (may be NULL): RT_COUNTERS int64 accumulated:
 *                 accepted steps, rejected steps, pixels finished, pixels
 *                 escaped, pixels handed from the FP32 to the FP64 kernel
 *                 (RT_PREC_MIXED), FP64 extremum searches of the crossing
 *                 search (pieces where a grazing pair could hide), crossings
 *                 counted
 *   opts          rtol, atol, r_capture_over_R, max_steps, precision used;
 *                 r_out_over_R, lambda_max ignored
 * The sign of g is decided in FP32 where it is certain (on shell, g has the
 * sign of P G - 1 up to the integrator's drift, and that is formed in FP32
 * with a wide margin), else in FP64; bisection and contributions are FP64.
 * RT_PREC_FP64: FP64 stages.  RT_PREC_MIXED: FP32 stages with the
 * double-float state of the forward mixed kernel; the crossing search runs on
 * the FP64 reconstruction of each step's continuous extension; a pixel whose FP32
 * error estimate sits on the rounding floor is traced again from the plane in
 * FP64 (second kernel on the same stream; the first call with a larger image
 * allocates a list of 4 B per pixel on the handle).
 * Deterministic.  Calls sharing one handle must be serialised on one stream.
 */
rt_status rt_trace_backward(const rt_star* star, int32_t nx, int32_t ny, double incl_rad,
                            double dist_over_R, double bmax_over_R, double Lc_cut_km,
                            double* d_image, uint8_t* d_status, int32_t* d_ncross,
                            int64_t* d_counters, const rt_trace_opts* opts, void* stream);

/*
 * Line-flux functional and its adjoint gradient.  The paper differentiates
 * nothing; this is a service for fitting its model (a reading):
 *   F = sum_i w_i K(khat_i . o),  K(mu) = C exp(kappa (mu - 1)),
 *   C = kappa / (2 pi (1 - exp(-2 kappa)))  (von Mises-Fisher kernel, unit mass),
 * over the ESCAPED rays i with weights w_i (Sec. 4.2, Eq. PowerCurved) and
 * khat_i the static orthonormal-frame momentum direction at r = r_out
 * (the direction rt_bin_spectrum bins, Sec. 2.2); o = (sin i, 0, cos i).
 * F is in W/sr: the line flux toward o smoothed over ~1/sqrt(kappa) rad.
 *
 * rt_flux_value - F over already traced rays (state, weight and status as
 *   rt_trace_forward leaves them).  d_F_ray: out, n per-ray terms; d_F: out,
 *   their sum (fixed summation order: deterministic).
 *
 * rt_flux_gradient - dF/dp for p = (m_a [eV], B0 [G], theta_m [rad], M [Msun],
 *   R [km], inclination [rad]) by reverse-mode differentiation of sampling and
 *   the FP64 integrator, at the star's parameters, for the n samples drawn
 *   from d_uniforms (RT_UNIFORM_ROWS x n, as rt_sample_conversion_surface)
 *   and traced with opts (lambda_max 0).  Each ray is re-integrated in FP64
 *   (the same steps as the forward rt_trace_forward run with the same opts,
 *   whose accepted steps per ray d_nacc sizes the store) and swept
 *   backwards: the discrete adjoint of each Dormand-Prince step
 *   (Jacobian-vector products of the analytic right-hand side by forward-mode
 *   dual numbers), the saltation jump where the Goldreich-Julian branch
 *   switches on the null cone, and the escape point's implicit dependence on
 *   the parameters.  The derivatives of the initial state and the weight come
 *   from the sampling code in dual numbers (the resonance root by the
 *   implicit function theorem).  Status, escape and the number of steps are
 *   held fixed (the gradient of the discrete scheme at frozen decisions).
 *   Store: the full step tape (every accepted step with its seven stages,
 *   416 B, plus 488 B per ray) when it fits under tape_max_bytes: one replay
 *   records the rays, longest first, and a second kernel sweeps them
 *   backwards; else a checkpoint every 32 accepted steps (sum over rays of
 *   (nacc/32 + 2) x 104 B) and segment scratch (13 KB per resident thread:
 *   about 500 MB on GB300), each segment re-integrated from its checkpoint
 *   before its sweep (one replay more).
 *   opts.precision sets the arithmetic of the backward sweep (stages, Jacobian
 *   products, adjoint accumulation), the replay being FP64 always:
 *   RT_PREC_FP64 FP64; RT_PREC_MIXED the adjoint of the state and its
 *   Jacobian products in FP64, the tangents of the three constants of the
 *   ray equations (r_s, the omega_p^2 coefficient, the magnetic axis) and
 *   their products with the adjoint in FP32 (about 1e-5 from the FP64 sweep,
 *   in half the FP64 sweep's time); RT_PREC_DF double-float (FP64-class
 *   rounding on the FP32 pipe; slower than the FP64 sweep on GB300).
 *     d_grad     out: 6 float64, dF/dp
 *     d_F        out: 1 float64, F recomputed by the adjoint's replay
 *     d_status   out (may be NULL): n final statuses of the replay
 *     d_counters in/out (may be NULL): [0] replayed step attempts (first
 *                replay), [2] rays, [4] rays left out (replay longer than
 *                d_nacc allows)
 *     tape_max_bytes  most device bytes the full tape may take (-1: half of
 *                the free device memory; 0: checkpoints always); a tape whose
 *                allocation fails falls back to the checkpoints
 *     store_bytes out (host, may be NULL): bytes of the tape or checkpoint store
 *   Needs RT_PLASMA_GJ, M_sun > 0 and B0_G > 0.  Synchronous: allocates the
 *   store and 69 B per ray, and frees them before returning; RT_ENOMEM if
 *   that fails.  Deterministic (fixed-order sums of per-ray terms).
 */
rt_status rt_flux_value(const rt_star* star, int64_t n, const double* d_state,
                        const double* d_weight, const uint8_t* d_status, double incl_rad,
                        double kappa, double* d_F_ray, double* d_F, void* stream);
rt_status rt_flux_gradient(const rt_star* star, int64_t n, const double* d_uniforms,
                           const int32_t* d_nacc, double incl_rad, double kappa,
                           const rt_trace_opts* opts, double* d_grad, double* d_F,
                           uint8_t* d_status, int64_t* d_counters, int64_t tape_max_bytes,
                           int64_t* store_bytes, void* stream);

/*
 * Batches: many stars (different B0, P, misalignment, m_a, ...) traced in ONE
 * persistent launch whose global queue spans all of them, so the long rays of
 * one star overlap with the bulk of the others.  counts[s] rays of star s
 * occupy rays [off_s, off_s + counts[s]) of arrays of total length
 * N = sum(counts), in star order (SoA row stride N).
 *
 * rt_init_batch - host; allocates a device star table, the offsets and a
 *   queue counter.  The star handles must outlive the batch.  All stars share
 *   one rotation mode (RT_EUNSUPPORTED otherwise); a batch of
 *   RT_ROTATION_RIGID stars is traced by the rotating-magnetosphere kernel
 *   (FP64 only, no images, no autotuner).
 * rt_sample_batch - rt_sample_conversion_surface for every star on its range
 *   (each star's weights normalised by its own count); u is 6 x N, state
 *   8 x N.  RT_EEMPTY_SURFACE only when every star's surface is empty.
 * rt_trace_batch - rt_trace_forward over all N rays in one launch (FP64) or
 *   one FP32 launch plus one FP64 pass for promoted rays (RT_PREC_MIXED).
 *   With images set (rt_batch_set_images), the same persistent launch also
 *   traces every pixel of every image (rt_trace_backward's estimator): rays
 *   and pixels share one work queue, rays first, and a lane that finishes
 *   either claims the next item of either kind.  RT_PREC_MIXED then runs one
 *   FP32 launch and one FP64 launch for the promoted rays (from where they
 *   stopped) and the handed-over pixels (anew).  No tail mode in that case;
 *   lambda_max must be 0.  Timestamps: 1 + nstars + nimg entries, [1 + nstars
 *   + j] the last pixel of image j.  Counters add rays and pixels.
 * rt_bin_batch - per-star histograms: d_hist is nstars x nth x nph x nnu,
 *   d_out_of_range nstars; per-star fixed-point scales (binning scratch owned
 *   by the batch, allocated on first use).
 * Calls on one batch must be serialised on one stream.
 */
typedef struct rt_batch rt_batch;

/* One backward image of a batch: the arguments of rt_trace_backward. */
typedef struct {
  int32_t nx, ny;
  double incl_rad, dist_over_R, bmax_over_R, Lc_cut_km;
} rt_image_desc;

rt_status rt_init_batch(const rt_star* const* stars, int32_t nstars, const int64_t* counts,
                        rt_batch** out);
void rt_destroy_batch(rt_batch* batch);
rt_status rt_sample_batch(rt_batch* batch, const double* d_uniforms, double* d_state,
                          double* d_weight, uint8_t* d_status, void* stream);
/*
 * rt_batch_set_norm - host: the weight normalisation of each star's samples
 *   in rt_sample_batch (and in graphs created afterwards): n_norm[s] >=
 *   counts[s] samples in place of counts[s], as rt_sample_conversion_surface_part
 *   does for one star, so that batches holding contiguous parts of one
 *   workload on different GPUs carry the weights of the whole.  NULL restores
 *   the counts.  RT_EINVAL if some n_norm[s] < max(counts[s], 1) (the earlier
 *   setting is kept).
 */
rt_status rt_batch_set_norm(rt_batch* batch, const int64_t* n_norm);
rt_status rt_trace_batch(rt_batch* batch, double* d_state, uint8_t* d_status, int32_t* d_nacc,
                         int32_t* d_nrej, int64_t* d_counters, const rt_trace_opts* opts,
                         void* stream);
rt_status rt_bin_batch(rt_batch* batch, const double* d_state, const double* d_weight,
                       const uint8_t* d_status, int32_t nth, int32_t nph, int32_t nnu,
                       double nu_lo, double nu_hi, double* d_hist, double* d_out_of_range,
                       void* stream);
/*
 * rt_batch_set_images - host, synchronous: the backward images that
 *   rt_trace_batch traces together with the batch's rays (Sec. 2.1, Eq.
 *   BackPower; the geometry and estimator of rt_trace_backward).  Image j of
 *   star stars[j] (handles outlive the batch) and geometry descs[j] writes its
 *   ny x nx pixels at offset P_j = sum_{i<j} nx_i ny_i of the caller-owned
 *   device buffers d_image (float64, W / sr), d_img_status (u8) and d_ncross
 *   (int32, may be NULL), each of total length P = sum nx_j ny_j <= 2^31.
 *   Uploads a table of the images (about 300 B each) and a 4 B-per-pixel list
 *   for the mixed-precision hand-over, replacing any earlier images; nimg = 0
 *   removes them.  RT_EINVAL on any invalid geometry (the earlier images are
 *   kept); RT_ENOMEM leaves the batch without images.
 */
rt_status rt_batch_set_images(rt_batch* batch, int32_t nimg, const rt_star* const* stars,
                              const rt_image_desc* descs, double* d_image, uint8_t* d_img_status,
                              int32_t* d_ncross);

/*
 * CUDA graph of one batch step.  rt_batch_graph_create captures, on a stream
 * of its own, exactly what rt_sample_batch, rt_trace_batch (with d_counters
 * and opts) and rt_bin_batch enqueue for these buffers -- plus a reset of
 * d_counters (may be NULL) and of opts->timestamps (if set) -- and
 * instantiates it (host, synchronous; the launch shape is fixed at capture,
 * so autotune first).  rt_graph_launch replays it on `stream` (the buffers'
 * contents at replay time are used).  The graph holds the batch's handles:
 * destroy it before them.
 */
typedef struct rt_graph rt_graph;
rt_status rt_batch_graph_create(rt_batch* batch, const double* d_uniforms, double* d_state,
                                double* d_weight, uint8_t* d_status, int64_t* d_counters,
                                const rt_trace_opts* opts, int32_t nth, int32_t nph, int32_t nnu,
                                double nu_lo, double nu_hi, double* d_hist,
                                double* d_out_of_range, rt_graph** out);
rt_status rt_graph_launch(rt_graph* graph, void* stream);
void rt_graph_destroy(rt_graph* graph);

/*
 * rt_batch_autotune - choose, for this batch and opts->precision, the trace
 * launch's shape (threads per block, resident blocks per SM), its refill
 * threshold and its rays per claim (rt_trace_opts.refill_min,
 * rays_per_claim) by timing candidates on a sample, in three rounds: every
 * shape the kernel's register budget allows (refill 1, 1 ray per claim), then
 * refill thresholds 2, 4, 8, 16 at the best shape, then 2, 4, 8 rays per
 * claim at the best threshold.  The sample: the first rays_per_star sampled
 * rays of every star (d_state/d_status as left by rt_sample_batch; copied,
 * not modified) and, when images are set (rt_batch_set_images), a coarse copy
 * of every image -- the same plane in at most side x side pixels, side =
 * ceil(sqrt(rays_per_star)), traced into scratch -- so that the launch tuned
 * is the one rt_trace_batch runs (rays and pixels in one queue).  One warm-up
 * run, then one timed run per candidate (CUDA events).  The choice is stored
 * in the batch per precision and per kind of launch (rays only, or with
 * images) and used by rt_trace_batch for the fields of opts left at 0.
 * Synchronous; allocates and frees scratch for the sample.
 *   block_out, bps_out, refill_out, claim_out, ms_out (host, may be NULL):
 *   the winner and its time
 *   ncand_out (may be NULL): candidates timed; cand_ms (may be NULL): their
 *   times in ms in the order above, at most cand_cap of them
 */
rt_status rt_batch_autotune(rt_batch* batch, const double* d_state, const uint8_t* d_status,
                            const rt_trace_opts* opts, int32_t rays_per_star, int32_t* block_out,
                            int32_t* bps_out, int32_t* refill_out, int32_t* claim_out,
                            double* ms_out, int32_t* ncand_out, double* cand_ms,
                            int32_t cand_cap, void* stream);

/*
 * rt_bin_spectrum_noalloc - rt_bin_spectrum for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is a service of the
 * library.  Some callers run under a device-memory budget that someone else
 * manages (a framework's caching allocator, a fixed pool shared through MPS)
 * or cannot afford the device-wide synchronisation that cudaMalloc and
 * cudaFree can imply (a real-time pipeline); rt_bin_spectrum would allocate
 * its fixed-point accumulator on first use.  This entry point allocates
 * nothing: its accumulator is a file-scope device array of
 * RT_BIN_NOALLOC_MAX_ENTRIES int64 (4 MiB) that every GPU which loads the
 * library holds until the process exits.  It takes the star parameters by
 * value (no rt_star handle) and otherwise has the arguments, outputs and
 * fixed-point semantics of rt_bin_spectrum.
 *   Limit: 2 + nth*nph*nnu + nth*nph + nnu <= RT_BIN_NOALLOC_MAX_ENTRIES,
 *   else RT_EINVAL (message in rt_last_error()).
 *   Checks: params must pass rt_init_star's validation, and every array must
 *   be device (or managed) memory of the current device; RT_EINVAL
 *   otherwise, before anything is enqueued.
 *   Set-up: the first call on a device looks up the device address of the
 *   array (cudaGetSymbolAddress, with that device current); make that first
 *   call before any stream capture.  The address is cached for the life of
 *   the process: after cudaDeviceReset on a device, do not call this entry
 *   point on that device again in the same process.
 *   Sharing: every call on a device uses the same array; each call clears
 *   the part it uses (an asynchronous memset on `stream`) and leaves its sums
 *   there afterwards.  Calls that overlap on the GPU (different streams, or
 *   different host threads without ordering) race and corrupt each other's
 *   results: order them on one stream.
 */
#define RT_BIN_NOALLOC_MAX_ENTRIES (1 << 19)
rt_status rt_bin_spectrum_noalloc(const rt_star_params* params, int64_t n, const double* d_state,
                                  const double* d_weight, const uint8_t* d_status, int32_t nth,
                                  int32_t nph, int32_t nnu, double nu_lo, double nu_hi,
                                  double* d_hist, double* d_sky, double* d_spec,
                                  double* d_out_of_range, void* stream);

/*
 * rt_hamilton_rhs - Hamilton's equations (Eq. Hamilton) of the strong-field
 * Hamiltonian (Eq. StrongBHam; the model of the star's switches) at n given
 * photon phase-space points: exactly the right-hand side that the FP64
 * integrators step with, for checks and for callers that integrate rays
 * themselves.  The Goldreich-Julian density |2 Omega.B / e| (Eq. GJDensity)
 * is differentiated on the side of its null cone where the point lies.
 *   d_state  RT_STATE_ROWS x n, as rt_trace_forward's state (x [km], k [eV],
 *            delta = omega_inf / m_a - 1, psi)
 *   d_H      out (may be NULL): n values of H / m_a^2
 *   d_dydl   out: 6 x n, d(x/R)/dl and d(k/m_a)/dl, rows x0 x1 x2 k0 k1 k2,
 *            with l the integrators' parameter (H scaled by m_a^2, x by R)
 * RT_EUNSUPPORTED for RT_ROTATION_RIGID stars.  Asynchronous on stream.
 */
rt_status rt_hamilton_rhs(const rt_star* star, int64_t n, const double* d_state, double* d_H,
                          double* d_dydl, void* stream);

/*
 * rt_count_status - histogram of per-ray status codes (synchronises the
 * stream).  counts: host array of RT_RAY_NSTATUS int64.  Returns RT_EPARTIAL
 * if any ray ended in MAXSTEPS, NAN or STIFF, else RT_OK.
 */
rt_status rt_count_status(int64_t n, const uint8_t* d_status, int64_t* counts, void* stream);

/*
 * rt_flops_per_step - algorithmic operation counts of the integrator (host
 * only), for roofline reports: out4[0] flops of one evaluation of the
 * analytic right-hand side of Hamilton's equations, out4[1] flops of one
 * Dormand-Prince step attempt (6 evaluations + stage combinations + error
 * norm + controller), out4[2] flops of the initial-step heuristic, out4[3]
 * divisions, square roots and powers per attempt.  A fused multiply-add
 * counts 2 flops; each division or square root counts 1.  RT_EINVAL for
 * unknown model switches.
 */
rt_status rt_flops_per_step(int32_t dispersion, int32_t plasma, double* out4);

/*
 * rt_flops_per_step_df - the same for RT_PREC_DF, in the FP32 operations the
 * double-float kernel executes (host only): out2[0] per right-hand side
 * evaluation, out2[1] per step attempt.  A double-float sum counts 11, a
 * product 10, a reciprocal square root 24 (rt_df.cuh); FMA = 2.  RT_EINVAL
 * for unknown model switches.
 */
rt_status rt_flops_per_step_df(int32_t dispersion, int32_t plasma, double* out2);

/*
 * rt_measure_alu_peak - measured FP64 and FP32 CUDA-core throughput of the
 * current device, the denominators of the roofline fractions (the tracing
 * kernels are bound by the fused multiply-add pipes; the paper reports no
 * throughput, Sec. 2.4 names only its CPU clusters).  A kernel in which every
 * thread runs 8 independent chains x <- x b + c (32 multiply-adds per
 * iteration) on a grid that fills every SM, one warm-up launch and one launch
 * timed with CUDA events on stream, first in FP64 (iters64 iterations), then
 * in FP32 (iters32).
 *   out4  host: [0] FP64 flop/s, [1] FP32 flop/s (a multiply-add counts 2),
 *         [2] FP64 kernel ms, [3] FP32 kernel ms
 * Synchronous; allocates and frees a result buffer of 2 KB per SM.  The rate
 * follows the SM clock of the moment: sample it alongside.
 */
rt_status rt_measure_alu_peak(int64_t iters64, int64_t iters32, double* out4, void* stream);

/* Thread-local message describing the last error of this thread. */
const char* rt_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch (2.0.0: rt_trace_opts
 * gained refill_min and rays_per_claim, rt_batch_autotune their outputs). */
int32_t rt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RT_AXION_H */
