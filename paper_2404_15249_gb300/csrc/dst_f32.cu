// FLOAT instantiation of the box solver kernels (see dst_impl.cuh).
#include "dst_impl.cuh"

namespace kfbi {

kfbi_status box_solve_f32(Ctx& c, const float* rhs, float* work) {
  return dst::box_solve_dispatch<float>(c, rhs, work,
                                      reinterpret_cast<const dst::cx<float>*>(c.t32.tw), c.t32.lam);
}

// picks the faster column-pass variant on the (scratch) work grid; called by setup
kfbi_status autotune_f32(Ctx& c) {
  return dst::autotune_dispatch<float>(c, c.V32, reinterpret_cast<const dst::cx<float>*>(c.t32.tw),
                                     c.t32.lam);
}

}  // namespace kfbi
