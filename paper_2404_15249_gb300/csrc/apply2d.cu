// One application of the layer potential (Alg. 1 steps 4-6) and the interface solves
// built from the same stages:
//   correction  b_p = F~_p + sum over crossed arms of sigma/h^2 (Taylor jump)  (Alg. 2)
//   box solve   (Lap_h - kappa^2) v = b, v = 0 on the box boundary            (Alg. 4)
//   interpolation  v^+(z_k) = sum_p w_p v_p + jump Taylor terms               (Alg. 3)
// The correction is a gather over the compacted irregular-node list with precomputed
// FP64 weights (one thread per irregular node, consecutive nodes per warp); for the
// double-layer apply the right-hand side is nonzero only at irregular nodes, so those
// entries of a persistent zero grid are overwritten in place and nothing else is touched.
#include "kfbi_internal.cuh"

namespace kfbi {

__device__ __forceinline__ int wrap(int k, int M) { return k < 0 ? k + M : (k >= M ? k - M : k); }

// b[irr_node[k]] = (add ? b : 0) + sum_arms sum_r (wD dens + wS psi + wF f)
template <typename T>
__global__ void correction_kernel(int nirr, int M, const int* __restrict__ irr_node,
                                  const int* __restrict__ arm_ptr, const int* __restrict__ arm_seg,
                                  const double* __restrict__ wD, const double* __restrict__ wS,
                                  const double* __restrict__ wF, const double* __restrict__ dens,
                                  const double* __restrict__ psi, const double* __restrict__ fctl,
                                  T* __restrict__ B, int add) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nirr) return;
  double acc = 0.0;
  for (int a = arm_ptr[k]; a < arm_ptr[k + 1]; ++a) {
    const int s = arm_seg[a];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      const int m = wrap(s - 2 + r, M);
      if (dens) acc += wD[6 * a + r] * dens[m];
      if (psi) acc += wS[6 * a + r] * psi[m];
      if (fctl) acc += wF[6 * a + r] * fctl[m];
    }
  }
  const int node = irr_node[k];
  B[node] = add ? (T)((double)B[node] + acc) : (T)acc;
}

// dense right-hand side on the N x N work grid: F at inside interior nodes, else 0
template <typename T>
__global__ void rhs_dense_kernel(int N, const double* __restrict__ F,
                                 const uint8_t* __restrict__ inside, T* __restrict__ W) {
  const long n = (long)N * N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / N), i = (int)(idx - (long)j * N);
    T v = T(0);
    if (F && i > 0 && j > 0) {
      const long g = (long)j * (N + 1) + i;
      if (inside[g]) v = (T)F[g];
    }
    W[idx] = v;
  }
}

// grid (N+1)^2 -> work grid N x N (interior entries; row/col 0 zero)
template <typename T>
__global__ void grid_to_work_kernel(int N, const double* __restrict__ G, T* __restrict__ W) {
  const long n = (long)N * N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n;
       idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / N), i = (int)(idx - (long)j * N);
    W[idx] = (i > 0 && j > 0) ? (T)G[(long)j * (N + 1) + i] : T(0);
  }
}

// work grid N x N -> (N+1)^2 grid; mask (optional) keeps inside nodes only
template <typename T>
__global__ void work_to_grid_kernel(int N, const T* __restrict__ W, const uint8_t* __restrict__ mask,
                                    double* __restrict__ G) {
  const long n = (long)(N + 1) * (N + 1);
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n;
       g += (long)gridDim.x * blockDim.x) {
    const int j = (int)(g / (N + 1)), i = (int)(g - (long)j * (N + 1));
    double v = (i < N && j < N) ? (double)W[(long)j * N + i] : 0.0;
    if (mask && !mask[g]) v = 0.0;
    G[g] = v;
  }
}

// out_k = sum_p w_p v(node_p) + sum_r (cD dens + cS psi) + eF f_k
template <typename T>
__global__ void interp_kernel(int M, const int* __restrict__ node, const double* __restrict__ w,
                              const double* __restrict__ cD, const double* __restrict__ cS,
                              const double* __restrict__ eF, const T* __restrict__ V,
                              const double* __restrict__ dens, const double* __restrict__ psi,
                              const double* __restrict__ fctl, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  double acc = 0.0;
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int nd = node[6 * k + p];
    if (nd >= 0) acc += w[6 * k + p] * (double)V[nd];
  }
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    const int m = wrap(k - 2 + r, M);
    if (dens) acc += cD[6 * k + r] * dens[m];
    if (psi) acc += cS[6 * k + r] * psi[m];
  }
  if (fctl) acc += eF[k] * fctl[k];
  out[k] = acc;
}

static inline int gs_blocks(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

template <typename T>
static kfbi_status correct(Ctx& c, const double* dens, const double* psi, const double* fctl,
                           T* B, int add) {
  if (c.nirr == 0) return KFBI_OK;
  const int pr = prof_begin(c, ST_CORR);
  correction_kernel<T><<<(c.nirr + 127) / 128, 128, 0, c.stream>>>(
      c.nirr, c.M, c.irr_node, c.arm_ptr, c.arm_seg, c.arm_wD, c.arm_wS, c.arm_wF, dens, psi,
      fctl, B, add);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T>
static kfbi_status interp(Ctx& c, const T* V, const double* dens, const double* psi,
                          const double* fctl, double* out) {
  const int pr = prof_begin(c, ST_INTERP);
  interp_kernel<T><<<(c.M + 127) / 128, 128, 0, c.stream>>>(c.M, c.ctrl_node, c.ctrl_w,
                                                            c.ctrl_cD, c.ctrl_cS, c.ctrl_eF, V,
                                                            dens, psi, fctl, out);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

static kfbi_status box(Ctx& c, int precision, const void* rhs, void* work) {
  if (precision == KFBI_FP64) return box_solve_f64(c, (const double*)rhs, (double*)work);
  return box_solve_f32(c, (const float*)rhs, (float*)work);
}

kfbi_status apply_potential(Ctx& c, Layer layer, int precision, const double* dens, double* out) {
  const double* d = layer == Layer::Double ? dens : nullptr;
  const double* s = layer == Layer::Single ? dens : nullptr;
  if (precision == KFBI_FP64) {
    KFBI_TRY(correct<double>(c, d, s, nullptr, c.B64, 0));
    KFBI_TRY(box_solve_f64(c, c.B64, c.V64));
    return interp<double>(c, c.V64, d, s, nullptr, out);
  }
  KFBI_TRY(correct<float>(c, d, s, nullptr, c.B32, 0));
  KFBI_TRY(box_solve_f32(c, c.B32, c.V32));
  return interp<float>(c, c.V32, d, s, nullptr, out);
}

template <typename T>
static kfbi_status interface_solve_t(Ctx& c, int precision, T* W, const double* dens,
                                     const double* f_grid, const double* f_ctrl,
                                     double* rhs_grid, double* v_grid, double* out) {
  prof_count(c, ST_GRID);
  rhs_dense_kernel<T><<<gs_blocks((long)c.N * c.N), 256, 0, c.stream>>>(c.N, f_grid, c.inside, W);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_TRY(correct<T>(c, dens, nullptr, f_ctrl, W, 1));
  if (rhs_grid) {
    prof_count(c, ST_GRID);
    work_to_grid_kernel<T><<<gs_blocks((long)(c.N + 1) * (c.N + 1)), 256, 0, c.stream>>>(
        c.N, W, nullptr, rhs_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  KFBI_TRY(box(c, precision, W, W));
  if (v_grid) {
    prof_count(c, ST_GRID);
    work_to_grid_kernel<T><<<gs_blocks((long)(c.N + 1) * (c.N + 1)), 256, 0, c.stream>>>(
        c.N, W, nullptr, v_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  if (out) KFBI_TRY(interp<T>(c, W, dens, nullptr, f_ctrl, out));
  return KFBI_OK;
}

kfbi_status interface_solve(Ctx& c, int precision, const double* dens, const double* f_grid,
                            const double* f_ctrl, double* rhs_grid, double* v_grid,
                            double* out) {
  if (precision == KFBI_FP64)
    return interface_solve_t<double>(c, precision, c.V64, dens, f_grid, f_ctrl, rhs_grid, v_grid,
                                     out);
  return interface_solve_t<float>(c, precision, c.V32, dens, f_grid, f_ctrl, rhs_grid, v_grid,
                                  out);
}

// u on the grid: inside nodes of the combined solve, zero elsewhere (FP64 path)
kfbi_status combined_u(Ctx& c, const double* dens, const double* f_grid, const double* f_ctrl,
                       double* u_grid) {
  double* W = c.V64;
  prof_count(c, ST_GRID);
  rhs_dense_kernel<double><<<gs_blocks((long)c.N * c.N), 256, 0, c.stream>>>(c.N, f_grid,
                                                                             c.inside, W);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_TRY(correct<double>(c, dens, nullptr, f_ctrl, W, 1));
  KFBI_TRY(box_solve_f64(c, W, W));
  prof_count(c, ST_GRID);
  work_to_grid_kernel<double><<<gs_blocks((long)(c.N + 1) * (c.N + 1)), 256, 0, c.stream>>>(
      c.N, W, c.inside, u_grid);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T>
static kfbi_status box_grid_t(Ctx& c, int precision, T* W, const double* b_grid, double* v_grid) {
  prof_count(c, ST_GRID);
  grid_to_work_kernel<T><<<gs_blocks((long)c.N * c.N), 256, 0, c.stream>>>(c.N, b_grid, W);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_TRY(box(c, precision, W, W));
  prof_count(c, ST_GRID);
  work_to_grid_kernel<T><<<gs_blocks((long)(c.N + 1) * (c.N + 1)), 256, 0, c.stream>>>(
      c.N, W, nullptr, v_grid);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status box_solve_grid(Ctx& c, int precision, const double* b_grid, double* v_grid) {
  if (precision == KFBI_FP64) return box_grid_t<double>(c, precision, c.V64, b_grid, v_grid);
  return box_grid_t<float>(c, precision, c.V32, b_grid, v_grid);
}

__global__ void copy_mask_kernel(long n, const uint8_t* in, uint8_t* out) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
       k += (long)gridDim.x * blockDim.x)
    out[k] = in[k];
}

kfbi_status inside_mask(Ctx& c, uint8_t* mask) {
  const long n = (long)(c.N + 1) * (c.N + 1);
  prof_count(c, ST_GRID);
  copy_mask_kernel<<<gs_blocks(n), 256, 0, c.stream>>>(n, c.inside, mask);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace kfbi
