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

kfbi_status x_pass_f32(Ctx& c, const float* X, float* V) {
  return dst::x_pass_dispatch<float>(c, X, V, reinterpret_cast<const dst::cx<float>*>(c.t32.tw));
}

kfbi_status ylines_f32(Ctx& c, float* X) {
  return dst::ylines_dispatch<float>(c, X, reinterpret_cast<const dst::cx<float>*>(c.t32.tw),
                                     c.t32.lam);
}

kfbi_status box_solve_after_rows_f32(Ctx& c, float* work) {
  return dst::box_after_rows_dispatch<float>(c, work,
                                             reinterpret_cast<const dst::cx<float>*>(c.t32.tw),
                                             c.t32.lam);
}

kfbi_status rows_pass_f32(Ctx& c, const float* in, float* out) {
  return dst::rows_dispatch<float>(c, in, out, reinterpret_cast<const dst::cx<float>*>(c.t32.tw));
}

kfbi_status ycol_lines_f32(Ctx& c, const float* V, float* Y, int ncols) {
  return dst::ycol_lines_dispatch<float>(c, V, Y, reinterpret_cast<const dst::cx<float>*>(c.t32.tw),
                                         c.t32.lam, ncols);
}


}  // namespace kfbi
