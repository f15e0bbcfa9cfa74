// DOUBLE instantiation of the box solver kernels (see dst_impl.cuh).
#include "dst_impl.cuh"

namespace kfbi {

kfbi_status box_solve_f64(Ctx& c, const double* rhs, double* work) {
  return dst::box_solve_dispatch<double>(c, rhs, work,
                                      reinterpret_cast<const dst::cx<double>*>(c.t64.tw), c.t64.lam);
}

// picks the faster column-pass variant on the (scratch) work grid; called by setup
kfbi_status autotune_f64(Ctx& c) {
  return dst::autotune_dispatch<double>(c, c.V64, reinterpret_cast<const dst::cx<double>*>(c.t64.tw),
                                     c.t64.lam);
}

}  // namespace kfbi
