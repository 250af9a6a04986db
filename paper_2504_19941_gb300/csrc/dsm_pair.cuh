// dsm_pair.cuh -- arithmetic on pairs of reals that undergo the same
// operation (the two populations of opposite directions, the two stencil sums
// of one neighbour).  In FP32 each pair operation is one packed two-wide
// instruction (the FP32x2 add, multiply and fused multiply-add of sm_100 and
// later): one issue slot for two results, each rounded as its scalar
// counterpart would be.  In FP64 it is two scalar operations.
#pragma once

#include <cuda_runtime.h>

namespace dsm {

template <class T>
struct Pr {
  T a, b;
};

__device__ __forceinline__ Pr<float> pr_fma(Pr<float> x, Pr<float> y, Pr<float> z) {
  const float2 r = __ffma2_rn(make_float2(x.a, x.b), make_float2(y.a, y.b), make_float2(z.a, z.b));
  return {r.x, r.y};
}
__device__ __forceinline__ Pr<float> pr_add(Pr<float> x, Pr<float> y) {
  const float2 r = __fadd2_rn(make_float2(x.a, x.b), make_float2(y.a, y.b));
  return {r.x, r.y};
}
__device__ __forceinline__ Pr<float> pr_mul(Pr<float> x, Pr<float> y) {
  const float2 r = __fmul2_rn(make_float2(x.a, x.b), make_float2(y.a, y.b));
  return {r.x, r.y};
}

__device__ __forceinline__ Pr<double> pr_fma(Pr<double> x, Pr<double> y, Pr<double> z) {
  return {fma(x.a, y.a, z.a), fma(x.b, y.b, z.b)};
}
__device__ __forceinline__ Pr<double> pr_add(Pr<double> x, Pr<double> y) {
  return {x.a + y.a, x.b + y.b};
}
__device__ __forceinline__ Pr<double> pr_mul(Pr<double> x, Pr<double> y) {
  return {x.a * y.a, x.b * y.b};
}

template <class T>
__device__ __forceinline__ Pr<T> pr(T a, T b) {
  return {a, b};
}

}  // namespace dsm
