// Box solve of (Lap_h - kappa^2) v = b on the N^3 work grid (x fastest, index 0 along
// every axis zero), v = 0 on the box boundary (Alg. 4 in 3-D): DST-I along x, y and z with
// the division by lambda_i + lambda_j + lambda_k - kappa^2 between the forward and the
// inverse z-transforms.  Every transform runs on contiguous lines; the y- and z-lines
// are made contiguous by tile transposes:
//   A[k][j][i] -x-> A -> X[k][i][j] -y-> X -> A[(i,j)][k] -z, divide, z-> A
//   -> X[k][i][j] -y-> X -> A[k][j][i] -x-> A
// A is the work grid, X the context's second grid of the same size.
#include "dst_impl.cuh"

namespace kfbi {
namespace dst {

template <typename T, int N>
kfbi_status box_solve3_n(Ctx& c, const T* rhs, T* A, const cx<T>* tw, const T* lam) {
  constexpr int E = default_ept(N);
  constexpr CPlan P = cplan(N, E);
  constexpr int lpc = yline_lpc<T, N, E>();
  T* X = reinterpret_cast<T*>(c.XT);
  const int n2 = N * N;
  KFBI_TRY((launch_rows<T, N, E>(c, rhs, A, tw, T(1), n2)));
  KFBI_TRY(launch_transpose<T>(c, A, X, N, N, N));
  KFBI_TRY((launch_rows<T, N, E>(c, X, X, tw, T(1), n2)));
  KFBI_TRY(launch_transpose<T>(c, X, A, N, n2, 1));
  {
    const cx<T>* stw = nullptr;
    KFBI_TRY((stage_table<T, N, E>(c, tw, &stw)));
    const int threads = lpc * P.tpl;
    const size_t smem = yline_smem<T, N, E>();
    KFBI_TRY(set_smem_limit((const void*)yline_kernel<T, N, E, 3>, smem));
    int per_sm = 0;
    KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, yline_kernel<T, N, E, 3>,
                                                                threads, smem));
    if (per_sm < 1) per_sm = 1;
    int blocks = (n2 + lpc - 1) / lpc;
    blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
    const T scale = T((2.0 / N) * (2.0 / N) * (2.0 / N));
    const int pr = prof_begin(c, sizeof(T) == 4 ? ST_COLS32 : ST_COLS64);
    yline_kernel<T, N, E, 3><<<blocks, threads, smem, c.stream>>>(A, stw, tw, lam, T(c.kappa2),
                                                                  scale, n2, c.err_flag + 2,
                                                                  c.poll_limit);
    prof_end(c, pr);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  KFBI_TRY(launch_transpose<T>(c, A, X, n2, N, 1));
  KFBI_TRY((launch_rows<T, N, E>(c, X, X, tw, T(1), n2)));
  KFBI_TRY(launch_transpose<T>(c, X, A, N, N, N));
  KFBI_TRY((launch_rows<T, N, E>(c, A, A, tw, T(1), n2)));
  return KFBI_OK;
}

template <typename T>
kfbi_status box_solve3_dispatch(Ctx& c, const T* rhs, T* work, const cx<T>* tw, const T* lam) {
  switch (c.N) {
#define KFBI_CASE(n) \
  case n: return box_solve3_n<T, n>(c, rhs, work, tw, lam);
    KFBI_CASE(32) KFBI_CASE(48) KFBI_CASE(64) KFBI_CASE(96) KFBI_CASE(128) KFBI_CASE(192)
    KFBI_CASE(256) KFBI_CASE(384) KFBI_CASE(512)
#undef KFBI_CASE
  }
  set_error("3-D box solve: no compiled plan for N = %d", c.N);
  return KFBI_ERR_UNSUPPORTED;
}

}  // namespace dst

kfbi_status box_solve3_f32(Ctx& c, const float* rhs, float* work) {
  return dst::box_solve3_dispatch<float>(c, rhs, work, reinterpret_cast<const dst::cx<float>*>(c.t32.tw),
                                         c.t32.lam);
}

kfbi_status box_solve3_f64(Ctx& c, const double* rhs, double* work) {
  return dst::box_solve3_dispatch<double>(c, rhs, work,
                                          reinterpret_cast<const dst::cx<double>*>(c.t64.tw), c.t64.lam);
}

}  // namespace kfbi
