// Persistent forward ray-tracing kernel: one thread per ray, Dormand-Prince
// 5(4) adaptive integration of Hamilton's equations (Eq. Hamilton) with the
// analytic right-hand side of rt_device.cuh, warp-level refill of finished
// lanes from a global work queue (ballot + popc prefix, one atomic per warp
// refill).  Termination (Sec. 2.2): r = r_out located on the dense output,
// capture at r <= r_capture, lambda_max, or the step bounds.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_backward.cuh"
#include "rt_device.cuh"
#include "rt_integrator.cuh"
#include "rt_internal.h"
#include "rt_tail.cuh"

namespace rtk {

namespace {

__device__ __forceinline__ int find_star(const TraceParams& p, int64_t i) {
  if (p.nstars <= 1) return 0;
  int lo = 0, hi = p.nstars - 1;   // offsets[s] <= i < offsets[s + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.offsets[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ void load_lane(const TraceParams& p, int64_t i, Lane& L) {
  const StarDev& s = p.stars[find_star(p, i)];
  const int64_t n = p.n;
  L.R_km = s.R_km;
  L.ma_eV = s.ma_eV;
  const double iR = 1.0 / s.R_km, im = 1.0 / s.ma_eV;
  L.y[0] = p.state[i] * iR;
  L.y[1] = p.state[n + i] * iR;
  L.y[2] = p.state[2 * n + i] * iR;
  L.y[3] = p.state[3 * n + i] * im;
  L.y[4] = p.state[4 * n + i] * im;
  L.y[5] = p.state[5 * n + i] * im;
  const double om = 1.0 + p.state[6 * n + i];
  const double psi = p.state[7 * n + i];
  double sp, cpsi;
  sincos(psi, &sp, &cpsi);
  L.c.rs = s.rs_prop;
  L.c.cp = s.cp;
  L.c.pa = s.plasma_a;
  L.c.W2 = om * om;
  L.c.iW2 = 1.0 / (om * om);
  L.c.m0 = s.sin_tm * cpsi;
  L.c.m1 = s.sin_tm * sp;
  L.c.m2 = s.cos_tm;
  L.c.disp = s.dispersion;
  L.c.plasma = s.plasma;
  L.c.sig = gj_side<double>(L.c.m0, L.c.m1, L.c.m2, L.y[0], L.y[1], L.y[2]);
  L.switching = false;
  L.h_resume = 0.0;
  rhs64(L.c, L.y, L.f0);
  const double hmax = (p.lambda_max > 0.0) ? p.lambda_max : 1e30;
  L.h = initial_step(L.c, L.y, L.f0, p.rtol, p.atol, hmax);
  L.lam = 0.0;
  L.na = 0;
  L.nr = 0;
  if (p.claim_status == RAY_PROMOTED) {   // resume a ray handed over by the FP32 pass
    if (p.nacc) L.na = p.nacc[i];
    if (p.nrej) L.nr = p.nrej[i];
  }
  L.last_rej = false;
}

__device__ void store_lane(const TraceParams& p, int64_t i, const Lane& L, int st) {
  const int64_t n = p.n;
  p.state[i] = L.y[0] * L.R_km;
  p.state[n + i] = L.y[1] * L.R_km;
  p.state[2 * n + i] = L.y[2] * L.R_km;
  p.state[3 * n + i] = L.y[3] * L.ma_eV;
  p.state[4 * n + i] = L.y[4] * L.ma_eV;
  p.state[5 * n + i] = L.y[5] * L.ma_eV;
  status_after_state(p, i, st);
  if (p.nacc) p.nacc[i] = L.na;
  if (p.nrej) p.nrej[i] = L.nr;
}

// Express lane, step 1: the READY rays of cost bucket 0 as (key, ray) pairs,
// key = the bits of the squared null-cone distance (ordered as the distance).
__global__ void express_select_kernel(TraceParams p) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (p.status[i] != RAY_READY) continue;
    const double d2 = cone_dist2(p.stars[find_star(p, i)], p.state, p.n, i);
    if (!(d2 < 1e-6)) continue;                     // cost bucket 0 only
    const unsigned long long slot = atomicAdd(p.xcount, 1ull);
    if (slot < (unsigned long long)p.xcap) {
      p.xcand[2 * slot] = (unsigned long long)__double_as_longlong(d2);
      p.xcand[2 * slot + 1] = (unsigned long long)i;
    }
  }
}

// Express lane, step 2: candidate k goes to record slot rank(k) (ascending
// distance, ties by ray index: nearest the cone first) as a fresh park record
// (the start of load_lane), and its ray leaves the queue (RAY_EXPRESS).
__global__ void express_rank_kernel(TraceParams p) {
  const unsigned long long K = *p.xcount < (unsigned long long)p.xcap
                                   ? *p.xcount : (unsigned long long)p.xcap;
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < K;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long key = p.xcand[2 * k], ray = p.xcand[2 * k + 1];
    unsigned long long rank = 0;
    for (unsigned long long j = 0; j < K; ++j) {
      const unsigned long long kj = p.xcand[2 * j], rj = p.xcand[2 * j + 1];
      rank += (kj < key || (kj == key && rj < ray)) ? 1ull : 0ull;
    }
    Lane L;
    load_lane(p, (int64_t)ray, L);
    double* pe = p.xrec + rank * PARKREC;
#pragma unroll
    for (int j = 0; j < 6; ++j) pe[j] = L.y[j];
    pe[6] = L.h;
    pe[7] = 0.0;
    pe[8] = L.c.sig;
    pe[9] = 0.0;
    pe[10] = 0.0;
    pe[11] = 0.0;
    pe[12] = (double)ray;
    pe[13] = 0.0;
    p.status[ray] = RAY_EXPRESS;
  }
}

__device__ __forceinline__ unsigned sm_id() {
  unsigned r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// Wait of an express SM's other blocks: 20 us naps, at most ~20 s, then on.
constexpr int XWAIT_NS = 20000;
constexpr int XWAIT_MAX = 1000000;

__global__ void __launch_bounds__(128) trace_fp64_kernel(TraceParams p) {
  const int lane = threadIdx.x & 31;
  int64_t ray = -1;   // -1: needs a ray, -2: queue exhausted
  Lane L;
  long long acc = 0, rej = 0, traced = 0, esc = 0;
  int na0 = 0, nr0 = 0;   // steps a resumed ray had already taken in FP32
  // the queue: one pass over the rays, or COST_BUCKETS passes (pass b claims
  // the rays of cost bucket b)
  const int64_t nq = p.order ? (int64_t)COST_BUCKETS * p.n : p.n;
  if (p.ts && threadIdx.x == 0) atomicMin(p.ts, global_ns());
  if (p.xrec) {
    // express lane: the first block on each of the first xs SMs continues the
    // K express records six lanes per ray from the start -- its warps 0 and 1
    // the first S = 2 xs records (the rays nearest the cone) one group at a
    // time, then, like its other warps, the rest five groups at a time; the
    // SM's other blocks nap until every record is claimed, so that each
    // express warp has its sub-partition to itself
    const unsigned long long K = *p.xcount < (unsigned long long)p.xcap
                                     ? *p.xcount : (unsigned long long)p.xcap;
    const unsigned long long xs = express_sms(K);
    const unsigned long long S = express_solo(K);
    __shared__ int role;
    if (threadIdx.x == 0) {
      const unsigned sm = sm_id();
      role = (sm < xs && sm < (unsigned)XSLOTS) ? atomicAdd(p.xslot + sm, 1) : -1;
    }
    __syncthreads();
    if (role == 0) {
      GroupCounts gc;
      if ((threadIdx.x >> 5) < 2) tail_groups(p, p.xrec, 0, S, p.xcount + 2, 1, gc);
      tail_groups(p, p.xrec, S, K, p.xcount + 1, GROUPS_PER_WARP, gc);
      acc += gc.acc;
      rej += gc.rej;
      traced += gc.traced;
      esc += gc.esc;
    } else if (role > 0) {
      for (int it = 0; it < XWAIT_MAX; ++it) {
        if (*(volatile unsigned long long*)(p.xcount + 2) >= S &&
            *(volatile unsigned long long*)(p.xcount + 1) >= K - S)
          break;
        __nanosleep(XWAIT_NS);
      }
    }
  }
  ClaimChunk ch;
  for (;;) {
    claim_items(p.queue, nq, p.refill_min, p.claim_size, ray, ch, [&](int64_t idx) -> int64_t {
      const int pass = p.order ? (int)(idx / p.n) : 0;
      const int64_t i = idx - (int64_t)pass * p.n;
      if (p.status[i] != p.claim_status ||
          (p.order && (cost_bucket(p.stars[find_star(p, i)], p.state, p.n, i) != pass ||
                       !status_still(p, i, p.claim_status))))
        return -1;
      load_lane(p, i, L);
      na0 = L.na;
      nr0 = L.nr;
      return i;
    });
    const unsigned live = __ballot_sync(FULL, ray != -2);
    if (live == 0) break;
    if (p.park) {
      // the queue has drained and this warp holds few rays: park them for the
      // six-lanes-per-ray tail kernel (the complete integrator state)
      const unsigned has = __ballot_sync(FULL, ray >= 0);
      const unsigned drained = __ballot_sync(FULL, ray == -2);
      if (drained && has && __popc(has) <= p.park_live && ray >= 0) {
        const unsigned long long slot = atomicAdd(p.park_count, 1ull);
        if (slot < (unsigned long long)p.park_cap) {
          double* pe = p.park + slot * PARKREC;
#pragma unroll
          for (int j = 0; j < 6; ++j) pe[j] = L.y[j];
          pe[6] = L.h;
          pe[7] = L.h_resume;
          pe[8] = L.c.sig;
          pe[9] = (double)((L.last_rej ? 1 : 0) | (L.switching ? 2 : 0));
          pe[10] = (double)L.na;
          pe[11] = (double)L.nr;
          pe[12] = (double)ray;
          pe[13] = L.lam;
          acc += L.na - na0;
          rej += L.nr - nr0;
          ray = -2;
        }
      }
    }
    if (ray >= 0) {
      NoHook nh;
      const int st = advance(p, L, nh);
      if (st >= 0) {
        store_lane(p, ray, L, st);
        if (p.ts) atomicMax(p.ts + 1 + find_star(p, ray), global_ns());
        acc += L.na - na0;
        rej += L.nr - nr0;
        traced += 1;
        esc += (st == RAY_ESCAPED);
        ray = -1;
      }
    }
  }
  if (p.counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_down_sync(FULL, acc, o);
      rej += __shfl_down_sync(FULL, rej, o);
      traced += __shfl_down_sync(FULL, traced, o);
      esc += __shfl_down_sync(FULL, esc, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&p.counters[CTR_ACC], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&p.counters[CTR_REJ], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&p.counters[CTR_RAYS], (unsigned long long)traced);
      atomicAdd((unsigned long long*)&p.counters[CTR_ESC], (unsigned long long)esc);
      if (p.claim_status == RAY_PROMOTED)
        atomicAdd((unsigned long long*)&p.counters[CTR_PROMOTED_STEPS],
                  (unsigned long long)(acc + rej));
    }
  }
}

// ---------------------------------------------------------------------------
// Backward image plane, FP64 integrator (crossing search in rt_backward.cuh).

// Passes every accepted step, with its FP64 continuous extension, to the
// crossing search.
struct CrossingHook {
  bool on;           // false: a forward ray of a mixed batch (no crossing search)
  CrossingAcc acc;
  __device__ void on_accept(const Lane& L, const double* y, const double* yn, const double* k1,
                            const double*, const double* k3, const double* k4, const double* k5,
                            const double* k6, const double* k7, double h) {
    if (!on) return;
    double r2[6], r3[6], r4[6], r5[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      r2[i] = yn[i] - y[i];
      r3[i] = h * k1[i] - r2[i];
      r4[i] = r2[i] - h * k7[i] - r3[i];
      r5[i] = h * (DP::d1 * k1[i] + DP::d3 * k3[i] + DP::d4 * k4[i] + DP::d5 * k5[i] +
                   DP::d6 * k6[i] + DP::d7 * k7[i]);
    }
    acc.scan_step(L.c, y, yn, r2, r3, r4, r5);
  }
};

__device__ void load_pixel(const BackParams& bp, int64_t p, Lane& L, double rtol, double atol) {
  pixel_init(bp, p, L.y, L.c);
  L.R_km = bp.s.R_km;
  L.ma_eV = bp.s.ma_eV;
  L.switching = false;
  L.h_resume = 0.0;
  rhs64(L.c, L.y, L.f0);
  L.h = initial_step(L.c, L.y, L.f0, rtol, atol, 1e30);
  L.lam = 0.0;
  L.na = 0;
  L.nr = 0;
  L.last_rej = false;
}

__global__ void __launch_bounds__(128) backward_kernel(BackParams bp) {
  const int lane = threadIdx.x & 31;
  // all pixels, or only those the mixed-precision kernel handed over
  const int64_t npix = bp.list ? (int64_t)*bp.list_n : (int64_t)bp.nx * bp.ny;
  TraceParams tp;
  tp.rtol = bp.rtol;
  tp.atol = bp.atol;
  tp.r_out = 0.0;
  tp.lambda_max = 0.0;
  tp.r_capture = bp.r_capture;
  tp.max_steps = bp.max_steps;
  tp.ts = nullptr;
  tp.park = nullptr;
  int64_t pix = -1;
  Lane L;
  CrossingHook hk;
  hk.on = true;
  long long acc = 0, rej = 0, done = 0, esc = 0, nc = 0, srch = 0;
  if (bp.ts && threadIdx.x == 0) atomicMin(bp.ts, global_ns());
  for (;;) {
    const bool need = (pix == -1);
    const unsigned mneed = __ballot_sync(FULL, need);
    if (mneed) {
      const int leader = __ffs(mneed) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(bp.queue, (unsigned long long)__popc(mneed));
      base = __shfl_sync(FULL, base, leader);
      if (need) {
        const int64_t idx = (int64_t)base + __popc(mneed & ((1u << lane) - 1u));
        if (idx >= npix) {
          pix = -2;
        } else {
          pix = bp.list ? (int64_t)bp.list[idx] : idx;
          load_pixel(bp, pix, L, bp.rtol, bp.atol);
          // escaped once back at the distance the ray started from
          tp.r_out = sqrt(L.y[0] * L.y[0] + L.y[1] * L.y[1] + L.y[2] * L.y[2]);
          hk.acc.reset(&bp.s, bp.W, bp.Lc_cut);
        }
      }
    }
    if (__ballot_sync(FULL, pix != -2) == 0) break;
    if (pix >= 0) {
      const int st = advance(tp, L, hk);
      if (st >= 0) {
        bp.image[pix] = bp.img_scale * hk.acc.sum;
        if (bp.ts) atomicMax(bp.ts + 1, global_ns());
        bp.status[pix] = (uint8_t)st;
        if (bp.ncross) bp.ncross[pix] = hk.acc.ncross - hk.acc.ncut;
        acc += L.na;
        rej += L.nr;
        done += 1;
        esc += (st == RAY_ESCAPED);
        nc += hk.acc.ncross - hk.acc.ncut;
        srch += hk.acc.nsearch;
        pix = -1;
      }
    }
  }
  if (bp.counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_down_sync(FULL, acc, o);
      rej += __shfl_down_sync(FULL, rej, o);
      done += __shfl_down_sync(FULL, done, o);
      esc += __shfl_down_sync(FULL, esc, o);
      nc += __shfl_down_sync(FULL, nc, o);
      srch += __shfl_down_sync(FULL, srch, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&bp.counters[CTR_ACC], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&bp.counters[CTR_REJ], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&bp.counters[CTR_RAYS], (unsigned long long)done);
      atomicAdd((unsigned long long*)&bp.counters[CTR_ESC], (unsigned long long)esc);
      atomicAdd((unsigned long long*)&bp.counters[CTR_CROSS], (unsigned long long)nc);
      atomicAdd((unsigned long long*)&bp.counters[CTR_SEARCH], (unsigned long long)srch);
    }
  }
}

// Forward rays and backward pixels of a batch in one persistent launch (FP64,
// one lane per item, no tail mode): a lane that finishes claims the next item
// of the common queue, whichever kind it is.
__global__ void __launch_bounds__(128) batch_fp64_kernel(TraceParams p, ImgTable t) {
  const int lane = threadIdx.x & 31;
  const int64_t nf = p.n;
  const int64_t total = nf + (t.list ? (int64_t)*t.list_n : t.npix);
  TraceParams tp = p;          // r_out per item
  tp.park = nullptr;
  int64_t item = -1;           // -1: needs an item, -2: queue exhausted
  int64_t ray = 0, pix = 0;
  int img = 0;
  bool isp = false;
  Lane L;
  CrossingHook hk;
  hk.on = false;
  long long acc = 0, rej = 0, done = 0, esc = 0, nc = 0;
  int na0 = 0, nr0 = 0;
  if (p.ts && threadIdx.x == 0) atomicMin(p.ts, global_ns());
  ClaimChunk ch;
  for (;;) {
    claim_items(p.queue, total, p.refill_min, p.claim_size, item, ch,
                [&](int64_t idx) -> int64_t {
      if (idx < nf) {
        if (p.status[idx] != p.claim_status) return -1;
        isp = false;
        ray = idx;
        load_lane(tp, idx, L);
        na0 = L.na;
        nr0 = L.nr;
        tp.r_out = p.r_out;
        hk.on = false;
        return idx;
      }
      const int64_t q = idx - nf;
      const int64_t g = t.list ? (int64_t)t.list[q] : q;
      img = find_image(t, g);
      pix = g - t.off[img];
      const BackParams& bp = t.img[img];
      load_pixel(bp, pix, L, p.rtol, p.atol);
      na0 = nr0 = 0;
      // escaped once back at the distance the ray started from
      tp.r_out = sqrt(L.y[0] * L.y[0] + L.y[1] * L.y[1] + L.y[2] * L.y[2]);
      hk.on = true;
      hk.acc.reset(&bp.s, bp.W, bp.Lc_cut);
      isp = true;
      return idx;
    });
    if (__ballot_sync(FULL, item != -2) == 0) break;
    if (item >= 0) {
      const int st = advance(tp, L, hk);
      if (st >= 0) {
        if (!isp) {
          store_lane(tp, ray, L, st);
          if (p.ts) atomicMax(p.ts + 1 + find_star(p, ray), global_ns());
        } else {
          const BackParams& bp = t.img[img];
          bp.image[pix] = bp.img_scale * hk.acc.sum;
          bp.status[pix] = (uint8_t)st;
          if (bp.ncross) bp.ncross[pix] = hk.acc.ncross - hk.acc.ncut;
          if (t.ts) atomicMax(t.ts + img, global_ns());
          nc += hk.acc.ncross - hk.acc.ncut;
        }
        acc += L.na - na0;
        rej += L.nr - nr0;
        done += 1;
        esc += (st == RAY_ESCAPED);
        item = -1;
      }
    }
  }
  if (p.counters) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc += __shfl_down_sync(FULL, acc, o);
      rej += __shfl_down_sync(FULL, rej, o);
      done += __shfl_down_sync(FULL, done, o);
      esc += __shfl_down_sync(FULL, esc, o);
      nc += __shfl_down_sync(FULL, nc, o);
    }
    if (lane == 0) {
      atomicAdd((unsigned long long*)&p.counters[CTR_ACC], (unsigned long long)acc);
      atomicAdd((unsigned long long*)&p.counters[CTR_REJ], (unsigned long long)rej);
      atomicAdd((unsigned long long*)&p.counters[CTR_RAYS], (unsigned long long)done);
      atomicAdd((unsigned long long*)&p.counters[CTR_ESC], (unsigned long long)esc);
      atomicAdd((unsigned long long*)&p.counters[CTR_CROSS], (unsigned long long)nc);
      if (p.claim_status == RAY_PROMOTED)
        atomicAdd((unsigned long long*)&p.counters[CTR_PROMOTED_STEPS],
                  (unsigned long long)(acc + rej));
    }
  }
}

}  // namespace

cudaError_t launch_batch_fp64(const TraceParams& p, const ImgTable& t, int block,
                              int blocks_per_sm, cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (block <= 0) block = 128;
  if (block > 128) block = 128;
  block = (block / 32) * 32;
  if (block < 32) block = 32;
  if (blocks_per_sm <= 0) {
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_fp64_kernel, block, 0);
    if (e != cudaSuccess) return e;
    blocks_per_sm = occ > 0 ? occ : 1;
  }
  const int64_t items = p.n + t.npix;
  int64_t grid = (int64_t)nsm * blocks_per_sm;
  const int64_t max_useful = (items + block - 1) / block;
  if (grid > max_useful) grid = max_useful;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  batch_fp64_kernel<<<(unsigned)grid, block, 0, stream>>>(p, t);
  return cudaGetLastError();
}

cudaError_t launch_backward(const BackLaunch& b, cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  BackParams bp;
  bp.s = *b.star;
  bp.nx = b.nx;
  bp.ny = b.ny;
  bp.incl = b.incl;
  bp.D = b.D;
  bp.bmax = b.bmax;
  bp.W = b.W;
  bp.Lc_cut = b.Lc_cut;
  bp.img_scale = b.img_scale;
  bp.image = b.image;
  bp.status = b.status;
  bp.ncross = b.ncross;
  bp.counters = b.counters;
  bp.queue = b.queue;
  bp.rtol = b.rtol;
  bp.atol = b.atol;
  bp.r_capture = b.r_capture;
  bp.ts = b.ts;
  bp.max_steps = b.max_steps;
  bp.promo = nullptr;
  bp.promo_n = nullptr;
  bp.list = nullptr;
  bp.list_n = nullptr;
  if (b.prec == PREC_MIXED) {
    // FP32-stage pass over every pixel, then the FP64 kernel over the pixels
    // it handed over (the list's length is read on the device)
    bp.promo = b.promo;
    bp.promo_n = b.promo_n;
    e = cudaMemsetAsync(b.promo_n, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    e = launch_backward_mixed(bp, stream);
    if (e != cudaSuccess) return e;
    bp.list = b.promo;
    bp.list_n = b.promo_n;
  }
  const int block = 128;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, backward_kernel, block, 0);
  if (e != cudaSuccess) return e;
  const int64_t npix = (int64_t)b.nx * b.ny;
  int64_t grid = (int64_t)nsm * (occ > 0 ? occ : 1);
  const int64_t max_useful = (npix + block - 1) / block;
  if (grid > max_useful) grid = max_useful;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(b.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  backward_kernel<<<(unsigned)grid, block, 0, stream>>>(bp);
  return cudaGetLastError();
}

namespace {
__global__ void ts_reset_kernel(unsigned long long* ts, int n) {
  for (int i = threadIdx.x; i <= n; i += blockDim.x) ts[i] = (i == 0) ? ~0ull : 0ull;
}
}  // namespace

cudaError_t launch_ts_reset(unsigned long long* ts, int n, cudaStream_t stream) {
  ts_reset_kernel<<<1, 256, 0, stream>>>(ts, n);
  return cudaGetLastError();
}

cudaError_t occupancy_fp64(int block, int* occ) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, trace_fp64_kernel, block, 0);
}

cudaError_t occupancy_batch_fp64(int block, int* occ) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_fp64_kernel, block, 0);
}

cudaError_t launch_trace_fp64(const TraceParams& p, int block, int blocks_per_sm,
                              cudaStream_t stream) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (block <= 0) block = 128;
  if (block > 128) block = 128;            // __launch_bounds__(128)
  block = (block / 32) * 32;
  if (block < 32) block = 32;
  if (blocks_per_sm <= 0) {
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trace_fp64_kernel, block, 0);
    if (e != cudaSuccess) return e;
    blocks_per_sm = occ > 0 ? occ : 1;
  }
  const int64_t warps_needed = (p.n + 31) / 32;
  int64_t grid = (int64_t)nsm * blocks_per_sm;
  const int64_t max_useful = (warps_needed * 32 + block - 1) / block;
  if (grid > max_useful) grid = max_useful;
  if (grid < 1) grid = 1;
  e = cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  if (p.park) {
    e = cudaMemsetAsync(p.park_count, 0, 2 * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
  }
  TraceParams q = p;
  if (p.xrec) {
    // express lane: select and rank the bucket-0 rays; the persistent launch
    // then traces the rest one lane per ray, parking only when xpark is set
    e = cudaMemsetAsync(p.xcount, 0, 64 + XSLOTS * sizeof(int), stream);
    if (e != cudaSuccess) return e;
    const int64_t sel_grid = (p.n + 255) / 256 < (int64_t)nsm * 8 ? (p.n + 255) / 256
                                                                   : (int64_t)nsm * 8;
    express_select_kernel<<<(unsigned)(sel_grid > 0 ? sel_grid : 1), 256, 0, stream>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    express_rank_kernel<<<(unsigned)((XCAP + 127) / 128), 128, 0, stream>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!p.xpark) q.park = nullptr;
  }
  trace_fp64_kernel<<<(unsigned)grid, block, 0, stream>>>(q);
  e = cudaGetLastError();
  if (e != cudaSuccess || !p.park) return e;
  return launch_tail_fp64(p, stream);
}

}  // namespace rtk
