// dsm_lb_bf16.cu -- lattice Boltzmann kernels instantiated for __nv_bfloat16 storage
// and float arithmetic (one translation unit per precision, compiled in parallel).
#include "dsm_lb_impl.cuh"

namespace dsm {

LBTable lb_table_bf16(int kind) {
  return kind == 0 ? LBOps<0, float, __nv_bfloat16>::table() : LBOps<1, float, __nv_bfloat16>::table();
}

}  // namespace dsm
