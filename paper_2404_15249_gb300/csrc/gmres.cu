// Restarted GMRES for K_D phi = g_hat (Alg. 5) with every vector operation on the GPU in
// FP64: Arnoldi by classical Gram-Schmidt applied twice (CGS2), Givens rotations and the
// triangular least-squares solve on the device (the paper moves the least-squares step
// to the host every iteration; here only the residual estimate, 16 bytes, is read back).
// Mixed precision (GMRES-IR): the outer loop forms the true residual r = g_hat - K_D phi
// with an FP64 apply, an inner GMRES with FP32 box solves (FP64 Arnoldi) solves
// K_D d = r to a loose tolerance, and phi += d, until ||r|| <= tol ||g_hat||.
#include <cmath>

#include "kfbi_internal.cuh"

namespace kfbi {

constexpr int RED_T = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;   // valid in thread 0
}

// h[b] = <V_b, w> for b < blocks
__global__ void multidot_kernel(const double* __restrict__ V, int ld, int M,
                                const double* __restrict__ w, double* __restrict__ h) {
  __shared__ double sh[32];
  const double* v = V + (size_t)blockIdx.x * ld;
  double s = 0.0;
  for (int x = threadIdx.x; x < M; x += blockDim.x) s += v[x] * w[x];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) h[blockIdx.x] = s;
}

// w += sign * sum_{b < cnt} h[b] V_b
__global__ void mv_update_kernel(double* __restrict__ w, const double* __restrict__ V, int ld,
                                 int M, const double* __restrict__ h, int cnt, double sign) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= M) return;
  double s = 0.0;
  for (int b = 0; b < cnt; ++b) s += h[b] * V[(size_t)b * ld + x];
  w[x] += sign * s;
}

// scal[slot] = ||v||
__global__ void norm_kernel(const double* __restrict__ v, int M, double* scal, int slot) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int x = threadIdx.x; x < M; x += blockDim.x) s += v[x] * v[x];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) scal[slot] = sqrt(s);
}

// r = a - b ; optional scaled copy of r into dst by 1/scal[slot]
__global__ void sub_kernel(double* r, const double* a, const double* b, int M) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < M) r[x] = a[x] - (b ? b[x] : 0.0);
}

__global__ void axpy_kernel(double* y, const double* x, double a, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < M) y[k] += a * x[k];
}

__global__ void scale_kernel(double* dst, const double* src, int M, const double* scal, int slot) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < M) dst[x] = src[x] / scal[slot];
}

// Start of a cycle: V_0 = r / beta, g = beta e_1.  scal: [0] |g_{j+1}|, [1] breakdown,
// [2] beta, [3] NaN seen.
__global__ void cycle_start_kernel(double* V0, const double* r, int M, double* gvec, int m,
                                   double* scal) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const double beta = scal[2];
  if (x < M) V0[x] = r[x] / beta;
  if (x <= m) gvec[x] = (x == 0) ? beta : 0.0;
}

// Finish Arnoldi step j: column j of the Hessenberg matrix (h1 + h2 from the two CGS
// passes), its subdiagonal ||w||, V_{j+1} = w / ||w||, Givens rotation of the column and
// update of the least-squares right-hand side g.
__global__ void finish_kernel(int j, int m, int M, const double* __restrict__ w, double* V, int ld,
                              const double* __restrict__ h1, const double* __restrict__ h2,
                              double* hess, double* giv, double* gvec, double* scal) {
  __shared__ double sh[32];
  __shared__ double nrm_s;
  double s = 0.0;
  for (int x = threadIdx.x; x < M; x += blockDim.x) s += w[x] * w[x];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) nrm_s = sqrt(s);
  __syncthreads();
  const double nrm = nrm_s;
  const double beta = scal[2];
  const bool breakdown = !(nrm > 1e-14 * beta);
  if (!breakdown)
    for (int x = threadIdx.x; x < M; x += blockDim.x) V[(size_t)(j + 1) * ld + x] = w[x] / nrm;
  if (threadIdx.x == 0) {
    double* col = hess + (size_t)j * (m + 1);
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
    col[j + 1] = nrm;
    for (int i = 0; i < j; ++i) {
      const double cs = giv[2 * i], sn = giv[2 * i + 1];
      const double t = cs * col[i] + sn * col[i + 1];
      col[i + 1] = -sn * col[i] + cs * col[i + 1];
      col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    const double cs = col[j] / den, sn = col[j + 1] / den;
    giv[2 * j] = cs;
    giv[2 * j + 1] = sn;
    col[j] = den;
    col[j + 1] = 0.0;
    gvec[j + 1] = -sn * gvec[j];
    gvec[j] = cs * gvec[j];
    scal[0] = fabs(gvec[j + 1]);
    scal[1] = breakdown ? 1.0 : 0.0;
    scal[3] = (isfinite(nrm) && isfinite(den)) ? 0.0 : 1.0;
  }
}

// back substitution R y = g (k x k, R upper triangular in hess)
__global__ void lsq_kernel(int k, int m, const double* hess, const double* gvec, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = gvec[i];
    for (int l = i + 1; l < k; ++l) s -= hess[(size_t)l * (m + 1) + i] * y[l];
    y[i] = s / hess[(size_t)i * (m + 1) + i];
  }
}

// --------------------------------------------------------------------------- host side
struct Counters {
  int iters = 0, applies64 = 0, applies32 = 0;
};

static inline int vb(int M) { return (M + 255) / 256; }

kfbi_status alloc_gmres(Ctx& c, int m) {
  if (c.gm_m >= m && c.basis) return KFBI_OK;
  if (c.basis) {
    cudaFree(c.basis); cudaFree(c.hess); cudaFree(c.givens); cudaFree(c.gvec);
    cudaFree(c.hcol); cudaFree(c.yvec);
  }
  const int M = c.M;
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.basis, sizeof(double) * (size_t)(m + 1) * M));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.hess, sizeof(double) * (size_t)(m + 1) * m));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.givens, sizeof(double) * 2 * m));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.gvec, sizeof(double) * (m + 1)));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.hcol, sizeof(double) * 2 * (m + 1)));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.yvec, sizeof(double) * m));
  c.gm_m = m;
  return KFBI_OK;
}

static kfbi_status apply_K(Ctx& c, int precision, const double* x, double* y, Counters& cnt) {
  if (precision == KFBI_MIXED_FP32) ++cnt.applies32; else ++cnt.applies64;   // FP64-accurate
  return apply_potential(c, Layer::Double, precision, x, y);
}

static kfbi_status read_scal(Ctx& c, int n) {
  KFBI_CUDA_TRY(cudaMemcpyAsync(c.h_pinned, c.scal, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                c.stream));
  KFBI_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return KFBI_OK;
}

// Matvec precision of an Arnoldi step by the current residual estimate (inexact Krylov
// relaxation: once the residual is small a matvec may be as inaccurate as tol / ||r||
// relative).  tier[0] while est > th[0], tier[1] while est > th[1], tier[2] below.
struct Relax {
  int tier[3];
  double th[2];
  int pick(double est) const { return est > th[0] ? tier[0] : (est > th[1] ? tier[1] : tier[2]); }
};

// GMRES(m) on K_D for rhs, x in/out (x_zero: start from 0), FP64 Arnoldi, matvec
// precision chosen per step by `relax`.  Every cycle ends with the true residual formed
// with the FP64-accurate apply prec_true (an iterative-refinement step).  Stops when the
// residual is <= tol_abs; *res_out = last true residual norm.
static kfbi_status gmres_run(Ctx& c, const Relax& relax, int prec_true, const double* rhs,
                             double* x, bool x_zero, double tol_abs, int max_cycles,
                             Counters& cnt, double* res_out, int* cycles_out) {
  const int M = c.M, m = c.gm_m;
  cudaStream_t st = c.stream;
  double* r = c.vecs;            // residual
  double* w = c.vecs + M;        // Krylov image
  double* tmp = c.vecs + 2 * M;
  double* h1 = c.hcol;
  double* h2 = c.hcol + (m + 1);
  if (x_zero) {
    KFBI_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * M, st));
    KFBI_CUDA_TRY(cudaMemcpyAsync(r, rhs, sizeof(double) * M, cudaMemcpyDeviceToDevice, st));
  } else {
    KFBI_TRY(apply_K(c, prec_true, x, tmp, cnt));
    prof_count(c, ST_KRYLOV);
    sub_kernel<<<vb(M), 256, 0, st>>>(r, rhs, tmp, M);
  }
  prof_count(c, ST_KRYLOV);
  norm_kernel<<<1, 1024, 0, st>>>(r, M, c.scal, 2);
  KFBI_TRY(read_scal(c, 4));
  double beta = c.h_pinned[2];
  if (!std::isfinite(beta)) return KFBI_ERR_NUMERIC;
  int cyc = 0;
  for (; cyc < max_cycles && beta > tol_abs; ++cyc) {
    prof_count(c, ST_KRYLOV);
    cycle_start_kernel<<<vb(M > m + 1 ? M : m + 1), 256, 0, st>>>(c.basis, r, M, c.gvec, m, c.scal);
    int k = 0;
    double est = beta;
    for (int j = 0; j < m; ++j) {
      const int prec = relax.pick(est);
      KFBI_TRY(apply_K(c, prec, c.basis + (size_t)j * M, w, cnt));
      ++cnt.iters;
      prof_count(c, ST_KRYLOV, 5);
      multidot_kernel<<<j + 1, RED_T, 0, st>>>(c.basis, M, M, w, h1);
      mv_update_kernel<<<vb(M), 256, 0, st>>>(w, c.basis, M, M, h1, j + 1, -1.0);
      multidot_kernel<<<j + 1, RED_T, 0, st>>>(c.basis, M, M, w, h2);
      mv_update_kernel<<<vb(M), 256, 0, st>>>(w, c.basis, M, M, h2, j + 1, -1.0);
      finish_kernel<<<1, 1024, 0, st>>>(j, m, M, w, c.basis, M, h1, h2, c.hess, c.givens,
                                        c.gvec, c.scal);
      KFBI_CUDA_TRY(cudaGetLastError());
      KFBI_TRY(read_scal(c, 4));
      k = j + 1;
      if (c.h_pinned[3] != 0.0) return KFBI_ERR_NUMERIC;
      est = c.h_pinned[0];
      if (est <= tol_abs || c.h_pinned[1] != 0.0) break;
    }
    prof_count(c, ST_KRYLOV, 2);
    lsq_kernel<<<1, 32, 0, st>>>(k, m, c.hess, c.gvec, c.yvec);
    mv_update_kernel<<<vb(M), 256, 0, st>>>(x, c.basis, M, M, c.yvec, k, 1.0);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(apply_K(c, prec_true, x, tmp, cnt));
    prof_count(c, ST_KRYLOV, 2);
    sub_kernel<<<vb(M), 256, 0, st>>>(r, rhs, tmp, M);
    norm_kernel<<<1, 1024, 0, st>>>(r, M, c.scal, 2);
    KFBI_TRY(read_scal(c, 4));
    beta = c.h_pinned[2];
    if (!std::isfinite(beta)) return KFBI_ERR_NUMERIC;
  }
  *res_out = beta;
  if (cycles_out) *cycles_out = cyc;
  return KFBI_OK;
}

kfbi_status solve_bvp(Ctx& c, const double* f_grid, const double* f_ctrl, const double* g_ctrl,
                      double* u_grid, double* dens_out, kfbi_solve_info* info) {
  const int M = c.M;
  cudaStream_t st = c.stream;
  KFBI_TRY(alloc_gmres(c, c.opt.gmres_m));
  // precision of every step that must be FP64-accurate: FP64 transforms in the plain FP64
  // solver, FP32 transforms with FP64 residual refinement otherwise
  const int acc = c.opt.precision == KFBI_FP64 ? KFBI_FP64 : KFBI_FP32_REFINED;
  double* ghat = c.vecs + 3 * M;
  double* phi = c.vecs + 4 * M;
  double* d = c.vecs + 5 * M;
  Counters cnt;
  // g_hat = g - (Y f)^+
  KFBI_TRY(interface_solve(c, acc, nullptr, f_grid, f_ctrl, nullptr, nullptr, d));
  ++cnt.applies64;
  prof_count(c, ST_KRYLOV, 2);
  sub_kernel<<<vb(M), 256, 0, st>>>(ghat, g_ctrl, d, M);
  norm_kernel<<<1, 1024, 0, st>>>(ghat, M, c.scal, 4);
  KFBI_TRY(read_scal(c, 5));
  const double gnorm = c.h_pinned[4];
  const double tol_abs = c.opt.tol * gnorm;
  double res = 0.0;
  int cycles = 0;
  if (c.opt.precision == KFBI_MIXED_FP32) {
    // twice-refined applies (about 1e-13) while the residual is above tol / 1e-9,
    // once-refined (about 1e-10 at the largest grids) down to tol / inner_tol, plain FP32
    // below (inner_tol: the assumed relative accuracy of an FP32 apply)
    const Relax relax{{KFBI_FP32_REFINED, KFBI_FP32_REFINED_ONCE, KFBI_MIXED_FP32},
                      {tol_abs / 1e-9, tol_abs / c.opt.inner_tol}};
    KFBI_TRY(gmres_run(c, relax, acc, ghat, phi, true, tol_abs, c.opt.max_restarts + 1, cnt,
                       &res, &cycles));
  } else {
    const Relax relax{{acc, acc, acc}, {0.0, 0.0}};
    KFBI_TRY(gmres_run(c, relax, acc, ghat, phi, true, tol_abs, c.opt.max_restarts + 1, cnt,
                       &res, &cycles));
  }
  // u = W phi + Y f on inside nodes
  if (u_grid) {
    KFBI_TRY(combined_u(c, acc, phi, f_grid, f_ctrl, u_grid));
    ++cnt.applies64;
  }
  if (dens_out)
    KFBI_CUDA_TRY(cudaMemcpyAsync(dens_out, phi, sizeof(double) * M, cudaMemcpyDeviceToDevice, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  const double rel = gnorm > 0 ? res / gnorm : 0.0;
  if (info) {
    info->iterations = cnt.iters;
    info->outer_iterations = cycles;
    info->applies_fp64 = cnt.applies64;
    info->applies_low = cnt.applies32;
    info->rel_residual = rel;
    info->converged = rel <= c.opt.tol;
  }
  return rel <= c.opt.tol ? KFBI_OK : KFBI_ERR_NOT_CONVERGED;
}

// Batched BVPs: problems in turn on one stream, every right-hand side solved with the
// context's own options.
kfbi_status batch_solve(kfbi_ctx* ctxs, int count, int nrhs, const double* const* f_grid,
                        const double* const* f_ctrl, const double* const* g_ctrl,
                        double* const* u_grid, kfbi_solve_info* info, cudaStream_t stream) {
  kfbi_status worst = KFBI_OK;
  for (int p = 0; p < count; ++p) {
    Ctx& c = ctxs[p]->c;
    c.stream = stream;
    for (int r = 0; r < nrhs; ++r) {
      const int q = p * nrhs + r;
      kfbi_status s = solve_bvp(c, f_grid[q], f_ctrl[q], g_ctrl[q], u_grid[q], nullptr,
                                info ? info + q : nullptr);
      if (s != KFBI_OK && s != KFBI_ERR_NOT_CONVERGED) return s;
      if (s != KFBI_OK) worst = s;
    }
  }
  return worst;
}

}  // namespace kfbi
