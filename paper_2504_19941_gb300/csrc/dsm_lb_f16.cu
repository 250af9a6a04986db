// dsm_lb_f16.cu -- lattice Boltzmann kernels instantiated for __half storage
// and float arithmetic (one translation unit per precision, compiled in parallel).
#include "dsm_lb_impl.cuh"

namespace dsm {

LBTable lb_table_f16(int kind) {
  return kind == 0 ? LBOps<0, float, __half>::table() : LBOps<1, float, __half>::table();
}

}  // namespace dsm
