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

// same sums written to an FP64 grid and its FP32 rounding (right-hand side of a
// refined FP32 box solve)
__global__ void correction_dual_kernel(int nirr, int M, const int* __restrict__ irr_node,
                                       const int* __restrict__ arm_ptr,
                                       const int* __restrict__ arm_seg,
                                       const double* __restrict__ wD, const double* __restrict__ wS,
                                       const double* __restrict__ dens,
                                       const double* __restrict__ psi, double* __restrict__ B64,
                                       float* __restrict__ B32) {
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
    }
  }
  const int node = irr_node[k];
  B64[node] = acc;
  B32[node] = (float)acc;
}

// One step of iterative refinement of the box solve (Lap_h - kappa^2) v = b:
//   v_new = v_old + c  (c: FP32 correction from the last FP32 box solve, v_old FP64 or 0),
//   r = b - (Lap_h - kappa^2) v_new in FP64, stored as FP32 for the next FP32 solve.
// Work-grid layout N x N with row/column 0 and the implicit row/column N equal to zero.
__global__ void refine_step_kernel(int N, double inv_h2, double kappa2,
                                   const double* __restrict__ b, const double* __restrict__ v_old,
                                   const float* __restrict__ c, double* __restrict__ v_new,
                                   float* __restrict__ r) {
  const int j = blockIdx.y;                          // one grid row per blockIdx.y
  const long base = (long)j * N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const long idx = base + i;
    if (i == 0 || j == 0) {
      v_new[idx] = 0.0;
      r[idx] = 0.f;
      continue;
    }
    const double vc = (v_old ? v_old[idx] : 0.0) + (double)c[idx];
    const double e = (i + 1 < N) ? (v_old ? v_old[idx + 1] : 0.0) + (double)c[idx + 1] : 0.0;
    const double w = (v_old ? v_old[idx - 1] : 0.0) + (double)c[idx - 1];
    const double nn = (j + 1 < N) ? (v_old ? v_old[idx + N] : 0.0) + (double)c[idx + N] : 0.0;
    const double so = (v_old ? v_old[idx - N] : 0.0) + (double)c[idx - N];
    const double Lv = (e + w + nn + so - 4.0 * vc) * inv_h2 - kappa2 * vc;
    v_new[idx] = vc;
    r[idx] = (float)(b[idx] - Lv);
  }
}

// v = v_old + c (final refinement update) written to the (N+1)^2 grid, optional mask
__global__ void refine_out_kernel(int N, const double* __restrict__ v_old,
                                  const float* __restrict__ c, const uint8_t* __restrict__ mask,
                                  double* __restrict__ G) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= N; i += gridDim.x * blockDim.x) {
    const long g = (long)j * (N + 1) + i;
    double v = 0.0;
    if (i < N && j < N) {
      const long q = (long)j * N + i;
      v = v_old[q] + (double)c[q];
    }
    if (mask && !mask[g]) v = 0.0;
    G[g] = v;
  }
}

// FP64 grid -> FP32 copy (dense right-hand side of a refined solve)
__global__ void round_kernel(long n, const double* __restrict__ a, float* __restrict__ b) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
       k += (long)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}

// dense right-hand side on the N x N work grid: F at inside interior nodes, else 0
template <typename T>
__global__ void rhs_dense_kernel(int N, const double* __restrict__ F,
                                 const uint8_t* __restrict__ inside, T* __restrict__ W) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const long idx = (long)j * N + i;
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
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const long idx = (long)j * N + i;
    W[idx] = (i > 0 && j > 0) ? (T)G[(long)j * (N + 1) + i] : T(0);
  }
}

// work grid N x N -> (N+1)^2 grid; mask (optional) keeps inside nodes only
template <typename T>
__global__ void work_to_grid_kernel(int N, const T* __restrict__ W, const uint8_t* __restrict__ mask,
                                    double* __restrict__ G) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= N; i += gridDim.x * blockDim.x) {
    const long g = (long)j * (N + 1) + i;
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

// interpolation from a refined solution v = v_old + c
__global__ void interp_refined_kernel(int M, const int* __restrict__ node,
                                      const double* __restrict__ w, const double* __restrict__ cD,
                                      const double* __restrict__ cS, const double* __restrict__ eF,
                                      const double* __restrict__ v_old, const float* __restrict__ c,
                                      const double* __restrict__ dens,
                                      const double* __restrict__ psi,
                                      const double* __restrict__ fctl, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  double acc = 0.0;
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int nd = node[6 * k + p];
    if (nd >= 0) acc += w[6 * k + p] * (v_old[nd] + (double)c[nd]);
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

static inline dim3 rows_grid(int cols, int rows) {
  return dim3((unsigned)((cols + 255) / 256 < 8 ? (cols + 255) / 256 : 8), (unsigned)rows);
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

// Refined FP32 box solve: rhs b64 (FP64) and its FP32 rounding b32 (work-grid layout).
// Leaves v = X64[final] + V32; returns the index of X64 holding the FP64 part.
static kfbi_status refined_solve(Ctx& c, const double* b64, const float* b32, int* which,
                                 int steps) {
  const long n = (long)c.N * c.N;
  KFBI_TRY(box_solve_f32(c, b32, c.V32));
  const double* v_old = nullptr;
  int cur = 0;
  for (int it = 0; it < steps; ++it) {
    const int pr = prof_begin(c, ST_REFINE);
    refine_step_kernel<<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, 1.0 / (c.h * c.h), c.kappa2, b64,
                                                           v_old, c.V32, c.X64[cur], c.W32);
    prof_end(c, pr);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(box_solve_f32(c, c.W32, c.V32));
    v_old = c.X64[cur];
    cur ^= 1;
  }
  *which = cur ^ 1;
  if (steps == 0) {
    // no refinement: FP64 part is zero
    KFBI_CUDA_TRY(cudaMemsetAsync(c.X64[0], 0, sizeof(double) * n, c.stream));
    *which = 0;
  }
  return KFBI_OK;
}

static kfbi_status interp_refined(Ctx& c, int which, const double* dens, const double* psi,
                                  const double* fctl, double* out) {
  const int pr = prof_begin(c, ST_INTERP);
  interp_refined_kernel<<<(c.M + 127) / 128, 128, 0, c.stream>>>(
      c.M, c.ctrl_node, c.ctrl_w, c.ctrl_cD, c.ctrl_cS, c.ctrl_eF, c.X64[which], c.V32, dens,
      psi, fctl, out);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status apply_potential(Ctx& c, Layer layer, int precision, const double* dens, double* out) {
  const double* d = layer == Layer::Double ? dens : nullptr;
  const double* s = layer == Layer::Single ? dens : nullptr;
  if (precision == KFBI_FP64) {
    KFBI_TRY(correct<double>(c, d, s, nullptr, c.B64, 0));
    KFBI_TRY(box_solve_f64(c, c.B64, c.V64));
    return interp<double>(c, c.V64, d, s, nullptr, out);
  }
  if (precision == KFBI_FP32_REFINED || precision == PREC_REFINED1) {
    if (c.nirr > 0) {
      const int pr = prof_begin(c, ST_CORR);
      correction_dual_kernel<<<(c.nirr + 127) / 128, 128, 0, c.stream>>>(
          c.nirr, c.M, c.irr_node, c.arm_ptr, c.arm_seg, c.arm_wD, c.arm_wS, d, s, c.B64, c.B32);
      prof_end(c, pr);
      KFBI_CUDA_TRY(cudaGetLastError());
    }
    int which = 0;
    KFBI_TRY(refined_solve(c, c.B64, c.B32, &which, precision == PREC_REFINED1 ? 1 : c.refine_steps));
    return interp_refined(c, which, d, s, nullptr, out);
  }
  KFBI_TRY(correct<float>(c, d, s, nullptr, c.B32, 0));
  KFBI_TRY(box_solve_f32(c, c.B32, c.V32));
  return interp<float>(c, c.V32, d, s, nullptr, out);
}

// dense right-hand side F~ + corrections in FP64 in V64 (work layout)
static kfbi_status dense_rhs64(Ctx& c, const double* dens, const double* f_grid,
                               const double* f_ctrl) {
  prof_count(c, ST_GRID);
  rhs_dense_kernel<double><<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, f_grid, c.inside,
                                                                             c.V64);
  KFBI_CUDA_TRY(cudaGetLastError());
  return correct<double>(c, dens, nullptr, f_ctrl, c.V64, 1);
}

template <typename T>
static kfbi_status interface_solve_t(Ctx& c, int precision, T* W, const double* dens,
                                     const double* f_grid, const double* f_ctrl,
                                     double* rhs_grid, double* v_grid, double* out) {
  prof_count(c, ST_GRID);
  rhs_dense_kernel<T><<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, f_grid, c.inside, W);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_TRY(correct<T>(c, dens, nullptr, f_ctrl, W, 1));
  if (rhs_grid) {
    prof_count(c, ST_GRID);
    work_to_grid_kernel<T><<<rows_grid(c.N + 1, c.N + 1), 256, 0, c.stream>>>(
        c.N, W, nullptr, rhs_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  KFBI_TRY(box(c, precision, W, W));
  if (v_grid) {
    prof_count(c, ST_GRID);
    work_to_grid_kernel<T><<<rows_grid(c.N + 1, c.N + 1), 256, 0, c.stream>>>(
        c.N, W, nullptr, v_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  if (out) KFBI_TRY(interp<T>(c, W, dens, nullptr, f_ctrl, out));
  return KFBI_OK;
}

static kfbi_status interface_solve_refined(Ctx& c, const double* dens, const double* f_grid,
                                           const double* f_ctrl, double* rhs_grid,
                                           double* v_grid, double* out, const uint8_t* mask) {
  KFBI_TRY(dense_rhs64(c, dens, f_grid, f_ctrl));
  const long n = (long)c.N * c.N;
  if (rhs_grid) {
    prof_count(c, ST_GRID);
    work_to_grid_kernel<double><<<rows_grid(c.N + 1, c.N + 1), 256, 0, c.stream>>>(
        c.N, c.V64, nullptr, rhs_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  prof_count(c, ST_GRID);
  round_kernel<<<gs_blocks(n), 256, 0, c.stream>>>(n, c.V64, c.W32);
  KFBI_CUDA_TRY(cudaGetLastError());
  int which = 0;
  KFBI_TRY(refined_solve(c, c.V64, c.W32, &which, c.refine_steps));
  if (v_grid) {
    prof_count(c, ST_GRID);
    refine_out_kernel<<<rows_grid(c.N + 1, c.N + 1), 256, 0, c.stream>>>(
        c.N, c.X64[which], c.V32, mask, v_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  if (out) KFBI_TRY(interp_refined(c, which, dens, nullptr, f_ctrl, out));
  return KFBI_OK;
}

kfbi_status interface_solve(Ctx& c, int precision, const double* dens, const double* f_grid,
                            const double* f_ctrl, double* rhs_grid, double* v_grid,
                            double* out) {
  if (precision == KFBI_FP64)
    return interface_solve_t<double>(c, precision, c.V64, dens, f_grid, f_ctrl, rhs_grid, v_grid,
                                     out);
  if (precision == KFBI_FP32_REFINED)
    return interface_solve_refined(c, dens, f_grid, f_ctrl, rhs_grid, v_grid, out, nullptr);
  return interface_solve_t<float>(c, precision, c.V32, dens, f_grid, f_ctrl, rhs_grid, v_grid,
                                  out);
}

// u on the grid: inside nodes of the combined solve (Phi = phi, F = f~), zero elsewhere
kfbi_status combined_u(Ctx& c, int precision, const double* dens, const double* f_grid,
                       const double* f_ctrl, double* u_grid) {
  if (precision != KFBI_FP64)
    return interface_solve_refined(c, dens, f_grid, f_ctrl, nullptr, u_grid, nullptr, c.inside);
  double* W = c.V64;
  KFBI_TRY(dense_rhs64(c, dens, f_grid, f_ctrl));
  KFBI_TRY(box_solve_f64(c, W, W));
  prof_count(c, ST_GRID);
  work_to_grid_kernel<double><<<rows_grid(c.N + 1, c.N + 1), 256, 0, c.stream>>>(
      c.N, W, c.inside, u_grid);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T>
static kfbi_status box_grid_t(Ctx& c, int precision, T* W, const double* b_grid, double* v_grid) {
  prof_count(c, ST_GRID);
  grid_to_work_kernel<T><<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, b_grid, W);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_TRY(box(c, precision, W, W));
  prof_count(c, ST_GRID);
  work_to_grid_kernel<T><<<rows_grid(c.N + 1, c.N + 1), 256, 0, c.stream>>>(
      c.N, W, nullptr, v_grid);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status box_solve_grid(Ctx& c, int precision, const double* b_grid, double* v_grid) {
  if (precision == KFBI_FP64) return box_grid_t<double>(c, precision, c.V64, b_grid, v_grid);
  if (precision == KFBI_FP32_REFINED) {
    const long n = (long)c.N * c.N;
    prof_count(c, ST_GRID, 2);
    grid_to_work_kernel<double><<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, b_grid, c.V64);
    round_kernel<<<gs_blocks(n), 256, 0, c.stream>>>(n, c.V64, c.W32);
    KFBI_CUDA_TRY(cudaGetLastError());
    int which = 0;
    KFBI_TRY(refined_solve(c, c.V64, c.W32, &which, c.refine_steps));
    prof_count(c, ST_GRID);
    refine_out_kernel<<<rows_grid(c.N + 1, c.N + 1), 256, 0, c.stream>>>(
        c.N, c.X64[which], c.V32, nullptr, v_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
    return KFBI_OK;
  }
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
