// dsm_reduce.cuh -- deterministic block reductions that keep FP64 accuracy
// without FP64 arithmetic inside a warp.
//
// GB300's FP64 rate is a small fraction of its FP32 rate, so a warp-level tree
// of FP64 additions costs far more than the memory traffic of the kernels that
// reduce.  Here each warp adds FP32 values as unevaluated pairs hi + lo with
// Knuth's TwoSum (the exact rounding error of every addition is carried along),
// and only the per-warp results are converted and added in FP64.
#pragma once

#include <cuda_runtime.h>

namespace dsm {

struct FF {
  float hi, lo;
};

// s + e = a + b exactly (Knuth, TAOCP vol. 2, Sec. 4.2.2)
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = two_sum(x.hi, y.hi);
  const float t = s.lo + (x.lo + y.lo);
  return two_sum(s.hi, t);
}

// Sum over the block of NV per-thread FP32 values; kinds[k] = 1 takes the
// maximum instead.  Thread k < NV of the block receives result k in out[k]
// (FP64).  Fixed reduction order: the result does not depend on timing.
template <int NV>
__device__ __forceinline__ void block_reduce_ff(const float (&v)[NV], const int (&is_max)[NV],
                                                double *out) {
  __shared__ double sh[NV][32];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
  const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    if (is_max[k]) {
      float m = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
      if (lane == 0) sh[k][warp] = (double)m;
    } else {
      FF s = {v[k], 0.0f};
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        FF t;
        t.hi = __shfl_down_sync(0xffffffffu, s.hi, o);
        t.lo = __shfl_down_sync(0xffffffffu, s.lo, o);
        s = ff_add(s, t);
      }
      if (lane == 0) sh[k][warp] = (double)s.hi + (double)s.lo;
    }
  }
  __syncthreads();
  if (tid < NV) {
    double r = sh[tid][0];
    for (int w = 1; w < nw; w++) r = is_max[tid] ? fmax(r, sh[tid][w]) : r + sh[tid][w];
    out[tid] = r;
  }
}

}  // namespace dsm
