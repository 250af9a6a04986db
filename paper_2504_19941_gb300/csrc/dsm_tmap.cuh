// dsm_tmap.cuh -- host side of the single-pass steps' staging: tensor maps
// over the padded planes (layout in dsm_zstep.cuh), encoded through the
// driver's cuTensorMapEncodeTiled, looked up once through the runtime (no link
// against the driver library).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "dsm_lb_impl.cuh"

namespace dsm {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return (EncodeTiledFn)f;
  }();
  return fn;
}

// A 3-D tensor map over padded planes of `comp` interleaved reals per node
// (dims comp * nxp, nyp, nz) whose box is comp * ZB_X wide and `rows` high.
// nz may count several stacked plane sets (the N-fluid pairs).
inline bool encode_plane_map(CUtensorMap *m, void *base, int real_bytes, int comp, int nxp,
                             int nyp, int nz, int rows) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dim[3] = {(cuuint64_t)comp * nxp, (cuuint64_t)nyp, (cuuint64_t)nz};
  const cuuint64_t stride[2] = {(cuuint64_t)comp * nxp * real_bytes,
                                (cuuint64_t)comp * nxp * nyp * real_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)(comp * ZB_X), (cuuint32_t)rows, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  return enc(m, real_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
             3, base, dim, stride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace dsm
