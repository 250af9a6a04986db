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

// p + e = a * b exactly (the product's rounding error from one FMA)
__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

// Sum over the block of NV per-thread values given as FP32 pairs (hi + lo);
// is_max[k] = 1 takes the maximum of the hi parts instead.  Thread k < NV of
// the block writes result k to out[k] as one FP64 value.  The whole reduction
// runs on the FP32 pipes: on GB300 a warp-wide FP64 instruction occupies the
// FP64 pipe for many cycles even when one lane is active, so FP64 appears only
// in the final conversion.  Fixed order: the result does not depend on timing.
template <int NV>
__device__ __forceinline__ void block_reduce_ff(const FF (&v)[NV], const int (&is_max)[NV],
                                                double *out) {
  __shared__ float shh[NV][32], shl[NV][32];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int lane = tid & 31, warp = tid >> 5;
  const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) {
    FF s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      FF t;
      t.hi = __shfl_down_sync(0xffffffffu, s.hi, o);
      t.lo = __shfl_down_sync(0xffffffffu, s.lo, o);
      s = is_max[k] ? FF{fmaxf(s.hi, t.hi), 0.0f} : ff_add(s, t);
    }
    if (lane == 0) {
      shh[k][warp] = s.hi;
      shl[k][warp] = s.lo;
    }
  }
  __syncthreads();
  if (tid < NV) {
    FF r = {shh[tid][0], shl[tid][0]};
    for (int w = 1; w < nw; w++)
      r = is_max[tid] ? FF{fmaxf(r.hi, shh[tid][w]), 0.0f} : ff_add(r, FF{shh[tid][w], shl[tid][w]});
    out[tid] = (double)r.hi + (double)r.lo;
  }
}

template <int NV>
__device__ __forceinline__ void block_reduce_ff(const float (&v)[NV], const int (&is_max)[NV],
                                                double *out) {
  FF p[NV];
#pragma unroll
  for (int k = 0; k < NV; k++) p[k] = FF{v[k], 0.0f};
  block_reduce_ff<NV>(p, is_max, out);
}

}  // namespace dsm
