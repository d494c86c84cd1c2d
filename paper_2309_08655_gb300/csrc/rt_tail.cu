// Tail mode of the FP64 forward integrator: six lanes per ray (the group code,
// and why it pays on GB300, is in rt_tail.cuh).  This launch continues the
// rays that the persistent kernel parked once its queue had drained, and any
// express record (cost-ordered tracing) that no express group had claimed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_device.cuh"
#include "rt_integrator.cuh"
#include "rt_internal.h"
#include "rt_tail.cuh"

namespace rtk {

namespace {

__global__ void __launch_bounds__(128) tail_fp64_kernel(TraceParams p) {
  const int lane = threadIdx.x & 31;
  GroupCounts gc;
  if (p.xrec) {   // express records that no express group claimed
    const unsigned long long K = *p.xcount < (unsigned long long)p.xcap
                                     ? *p.xcount : (unsigned long long)p.xcap;
    const unsigned long long S = express_solo(K);
    tail_groups(p, p.xrec, 0, S, p.xcount + 2, GROUPS_PER_WARP, gc);
    tail_groups(p, p.xrec, S, K, p.xcount + 1, GROUPS_PER_WARP, gc);
  }
  const unsigned long long nparked = *p.park_count < (unsigned long long)p.park_cap
                                         ? *p.park_count
                                         : (unsigned long long)p.park_cap;
  tail_groups(p, p.park, 0, nparked, p.park_next, GROUPS_PER_WARP, gc);
  if (p.counters && (lane % GROUP) == 0 && lane / GROUP < GROUPS_PER_WARP) {
    atomicAdd((unsigned long long*)&p.counters[CTR_ACC], (unsigned long long)gc.acc);
    atomicAdd((unsigned long long*)&p.counters[CTR_REJ], (unsigned long long)gc.rej);
    atomicAdd((unsigned long long*)&p.counters[CTR_RAYS], (unsigned long long)gc.traced);
    atomicAdd((unsigned long long*)&p.counters[CTR_ESC], (unsigned long long)gc.esc);
    if (p.claim_status == RAY_PROMOTED)
      atomicAdd((unsigned long long*)&p.counters[CTR_PROMOTED_STEPS],
                (unsigned long long)(gc.acc + gc.rej));
  }
}

}  // namespace

cudaError_t launch_tail_fp64(const TraceParams& p, cudaStream_t stream) {
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tail_fp64_kernel, 128, 0);
  if (e != cudaSuccess) return e;
  // enough groups for every possible parked ray to start at once
  const int64_t groups_per_block = 4 * GROUPS_PER_WARP;
  int64_t grid = (p.park_cap + groups_per_block - 1) / groups_per_block;
  const int64_t cap = (int64_t)nsm * (occ > 0 ? occ : 1);
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  tail_fp64_kernel<<<(unsigned)grid, 128, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace rtk
