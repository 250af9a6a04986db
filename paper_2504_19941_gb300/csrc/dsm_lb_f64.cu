// dsm_lb_f64.cu -- lattice Boltzmann kernels instantiated for double storage
// and double arithmetic (one translation unit per precision, compiled in parallel).
#include "dsm_lb_impl.cuh"

namespace dsm {

LBTable lb_table_f64(int kind) {
  return kind == 0 ? LBOps<0, double, double>::table() : LBOps<1, double, double>::table();
}

}  // namespace dsm
