// dsm_lb_f32.cu -- lattice Boltzmann kernels instantiated for float storage
// and float arithmetic (one translation unit per precision, compiled in parallel).
#include "dsm_lb_impl.cuh"

namespace dsm {

LBTable lb_table_f32(int kind) {
  return kind == 0 ? LBOps<0, float, float>::table() : LBOps<1, float, float>::table();
}

}  // namespace dsm
