// Restarted GMRES for K_D phi = g_hat (Alg. 5) with every vector operation on the GPU in
// FP64: Arnoldi by classical Gram-Schmidt applied twice (CGS2), Givens rotations and the
// triangular least-squares solve on the device (the paper moves the least-squares step
// to the host every iteration; here only 32 bytes of flags per step are read back, one
// step behind the device).  Mixed precision: one FP64 Arnoldi process whose matvec
// precision is relaxed as the residual drops (inexact Krylov), every restart cycle ending
// with the true residual from an FP64-accurate apply (an iterative-refinement step).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>
#include <string>
#include <thread>
#include <vector>
#include <cstdlib>

#include "kfbi_internal.cuh"

namespace kfbi {

constexpr int RED_T = 256;
constexpr int kBatchWorkers = 16;    // concurrent problems of a batch (8: 798 ms, 16: 729 ms,
                                     // 32: 778 ms for the 1024 solves of the batched workload)

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

// h[b] = <V_b, w> for b < nb.  Block (s, b) forms the partial dot product of V_b and w
// over the chunk [s DOT_CHUNK, (s+1) DOT_CHUNK) (eight independent loads per thread), the
// partial sums part[s * pld + b] are added in chunk order by the last block to finish (a
// counter, reset by that block), so the result does not depend on scheduling.
constexpr int DOT_CHUNK = 2048;
constexpr int DOT_T = 256;

static inline int dot_blocks(int M) { return (M + DOT_CHUNK - 1) / DOT_CHUNK; }

// With jp (the Arnoldi step index in device memory, so that one captured launch serves
// every step) nb = *jp + 1 and the grid covers the largest nb: blocks b >= nb return at once
// and the last of the gridDim.x * nb active blocks to finish adds the partial sums.
__global__ void __launch_bounds__(DOT_T) multidot_kernel(const double* __restrict__ V, int ld,
                                                         int M, int nb, const int* jp,
                                                         const double* __restrict__ w,
                                                         double* part, int pld,
                                                         unsigned* counter,
                                                         double* __restrict__ h) {
  __shared__ double sh[32];
  __shared__ bool last;
  if (jp) nb = *jp + 1;
  const int b = blockIdx.y, x0 = blockIdx.x * DOT_CHUNK;
  if (b >= nb) return;                       // uniform per block; only active blocks count
  const double* v = V + (size_t)b * ld;
  double a[DOT_CHUNK / DOT_T];
#pragma unroll
  for (int q = 0; q < DOT_CHUNK / DOT_T; ++q) {
    const int x = x0 + threadIdx.x + q * DOT_T;
    a[q] = x < M ? v[x] * w[x] : 0.0;
  }
  double t = 0.0;
#pragma unroll
  for (int q = 0; q < DOT_CHUNK / DOT_T; ++q) t += a[q];
  t = block_sum(t, sh);
  if (threadIdx.x == 0) {                    // the writer fences, then counts the block
    part[(size_t)blockIdx.x * pld + b] = t;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x * (unsigned)nb - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int bb = threadIdx.x; bb < nb; bb += blockDim.x) {
    double u = 0.0;
    for (int s = 0; s < (int)gridDim.x; ++s) u += __ldcg(part + (size_t)s * pld + bb);
    h[bb] = u;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// w += sign * sum_{b < cnt} h[b] V_b.  A CTA takes 32 consecutive x (one per lane) and
// MVU_SLICES warps: warp s accumulates the b = s, s + MVU_SLICES, ... (four independent
// partial sums, every load independent of the others), and the slices' partial sums are
// added in slice order through shared memory, so a thread waits for about cnt / MVU_SLICES
// loads instead of cnt and the grid has M / 32 CTAs.  With nrm_out: also ||w||_2 of the
// updated w, from per-CTA partial sums added in a fixed order by the last CTA to finish.
// (cnt = *jp + 1 when jp is given: the Arnoldi step index in device memory)
constexpr int MVU_X = 32;
constexpr int MVU_SLICES = 8;

static inline int mvu_blocks(int M) { return (M + MVU_X - 1) / MVU_X; }

__global__ void __launch_bounds__(MVU_X * MVU_SLICES)
    mv_update_kernel(double* __restrict__ w, const double* __restrict__ V, int ld, int M,
                     const double* __restrict__ h, int cnt, const int* jp, double sign,
                     double* part, unsigned* counter, double* nrm_out) {
  __shared__ double sp[MVU_SLICES][MVU_X];
  if (jp) cnt = *jp + 1;
  const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int x = blockIdx.x * MVU_X + lane;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  if (x < M) {
    constexpr int S = MVU_SLICES;
    int b = sl;
    for (; b + 3 * S < cnt; b += 4 * S) {
      a0 += __ldg(h + b) * V[(size_t)b * ld + x];
      a1 += __ldg(h + b + S) * V[(size_t)(b + S) * ld + x];
      a2 += __ldg(h + b + 2 * S) * V[(size_t)(b + 2 * S) * ld + x];
      a3 += __ldg(h + b + 3 * S) * V[(size_t)(b + 3 * S) * ld + x];
    }
    for (; b < cnt; b += S) a0 += __ldg(h + b) * V[(size_t)b * ld + x];
  }
  sp[sl][lane] = (a0 + a1) + (a2 + a3);
  __syncthreads();
  if (sl != 0) return;
  double wn = 0.0;
  if (x < M) {
    double t = sp[0][lane];
#pragma unroll
    for (int q = 1; q < MVU_SLICES; ++q) t += sp[q][lane];
    wn = w[x] + sign * t;
    w[x] = wn;
  }
  if (!nrm_out) return;                      // uniform over the grid
  double s2 = wn * wn;
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_down_sync(0xffffffffu, s2, o);
  unsigned last = 0;
  if (lane == 0) {
    part[blockIdx.x] = s2;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  // last CTA: lane l adds the partials l, l + 32, ... in order, then a fixed shuffle tree
  // (short FP64 dependency chains; the same order on every run)
  __threadfence();
  double u = 0.0;
  for (int q = lane; q < (int)gridDim.x; q += 32) u += __ldcg(part + q);
  for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
  if (lane == 0) {
    *nrm_out = sqrt(u);
    *counter = 0u;
  }
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

// Start of a cycle: V_0 = r / beta (also into vin, the input of the next apply), g = beta
// e_1, step index 0.  scal: [0] |g_{j+1}|, [1] breakdown, [2] beta, [3] NaN seen.
__global__ void cycle_start_kernel(double* V0, double* vin, const double* r, int M, double* gvec,
                                   int m, double* scal, int* jp) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const double beta = scal[2];
  if (x < M) {
    const double v = r[x] / beta;
    V0[x] = v;
    vin[x] = v;
  }
  if (x <= m) gvec[x] = (x == 0) ? beta : 0.0;
  if (x == 0) *jp = 0;
}

// Finish Arnoldi step j (nrm = ||w||, formed by the second update): V_{j+1} = w / nrm
// by every block; block 0 also forms column j of the Hessenberg matrix (h1 + h2 from the
// two CGS passes, subdiagonal nrm), applies the earlier Givens rotations and the new one,
// and updates the least-squares right-hand side g.  The column and the rotations are
// staged in shared memory (dynamic: (m + 1) + 2m doubles) so the sequential rotation loop
// runs on shared-memory operands.
// The step index j is read from device memory (jp); the flags scal[0..3] of the step are
// also written into host-mapped memory flags[4 (j mod 2) + 0..3] for the host to read one
// step behind, and V_{j+1} into vin, the input of the next apply.
__global__ void finish_kernel(int* jp, int m, int M, const double* __restrict__ w, double* V,
                              int ld, const double* __restrict__ h1, const double* __restrict__ h2,
                              const double* __restrict__ nrm_in, double* hess, double* giv,
                              double* gvec, double* scal, double* vin, double* flags,
                              unsigned* counter) {
  extern __shared__ double dyn[];
  const int j = *jp;
  // the last CTA to arrive advances the step index (every CTA has read it by then)
  auto advance = [&] {
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(counter, 1u) == gridDim.x - 1) {
        *jp = j + 1;
        *counter = 0u;
      }
    }
  };
  const double nrm = *nrm_in;
  const double beta = scal[2];
  const bool breakdown = !(nrm > 1e-14 * beta);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (!breakdown && x < M) {
    const double v = w[x] / nrm;
    V[(size_t)(j + 1) * ld + x] = v;
    vin[x] = v;
  }
  if (blockIdx.x != 0) {
    advance();
    return;
  }
  double* col = dyn;                 // m + 1
  double* gs = dyn + (m + 1);        // 2m
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = h1[i] + h2[i];
  for (int i = threadIdx.x; i < 2 * j; i += blockDim.x) gs[i] = giv[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    // the earlier rotations, in order; the entry that each rotation passes on to the next
    // stays in a register (two dependent FP64 operations per rotation)
    double carry = col[0];
    for (int i = 0; i < j; ++i) {
      const double cs = gs[2 * i], sn = gs[2 * i + 1], b = col[i + 1];
      col[i] = cs * carry + sn * b;
      carry = -sn * carry + cs * b;
    }
    col[j] = carry;
    col[j + 1] = nrm;
    const double den = hypot(col[j], col[j + 1]);
    const double cs = col[j] / den, sn = col[j + 1] / den;
    giv[2 * j] = cs;
    giv[2 * j + 1] = sn;
    col[j] = den;
    col[j + 1] = 0.0;
    const double gj = gvec[j];
    gvec[j + 1] = -sn * gj;
    gvec[j] = cs * gj;
    scal[0] = fabs(sn * gj);
    scal[1] = breakdown ? 1.0 : 0.0;
    scal[3] = (isfinite(nrm) && isfinite(den)) ? 0.0 : 1.0;
    // host-mapped slot: the host reads it after an event recorded behind this kernel,
    // whose completion makes the writes visible (no fence needed here)
    double* f = flags + 4 * (j & 1);
    f[0] = scal[0];
    f[1] = scal[1];
    f[2] = scal[2];
    f[3] = scal[3];
  }
  __syncthreads();
  double* hc = hess + (size_t)j * (m + 1);
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) hc[i] = col[i];
  advance();
}

// back substitution R y = g (k x k, R upper triangular in hess: column l at hess + l (m + 1)),
// column by column across the CTA: y_i = g_i / R_ii, then every thread updates its entries
// g_r -= R_ri y_i (r < i) of column i.  The reciprocals 1 / R_ii are formed in parallel
// first, so the serial chain holds one multiplication per column instead of an FP64
// division (the columns of R staged in shared memory when they fit; dynamic shared memory:
// k (k + 1) doubles if staged, else 2k)
__global__ void lsq_kernel(int k, int m, const double* hess, const double* gvec, double* y,
                           int staged) {
  extern __shared__ double dyn[];
  const double* R = hess;
  int ldr = m + 1;
  double* g;
  double* rinv;
  if (staged) {
    double* Rs = dyn;                 // k x k, column l at Rs[l * k]
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
      const int l = e / k, i = e - l * k;
      Rs[e] = hess[(size_t)l * (m + 1) + i];
    }
    R = Rs;
    ldr = k;
    g = dyn + (size_t)k * k;
  } else {
    g = dyn;
  }
  rinv = g + k;                       // the reciprocals after g
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    g[i] = gvec[i];
    rinv[i] = 1.0 / R[(size_t)i * ldr + i];
  }
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double yi = g[i] * rinv[i];
    if (threadIdx.x == 0) y[i] = yi;
    const double* col = R + (size_t)i * ldr;
    for (int r = threadIdx.x; r < i; r += blockDim.x) g[r] -= col[r] * yi;
    __syncthreads();
  }
}

// --------------------------------------------------------------------------- host side
struct Counters {
  int iters = 0, applies64 = 0, applies32 = 0;
};

static inline int vb(int M) { return (M + 255) / 256; }

void drop_step_graphs(Ctx& c) {
  for (int o = 0; o < kOps; ++o)
    for (int p = 0; p < kStepGraphs; ++p)
      if (c.step_exec[o][p]) {
        cudaGraphExecDestroy(c.step_exec[o][p]);
        c.step_exec[o][p] = nullptr;
      }
}

kfbi_status alloc_gmres(Ctx& c, int m) {
  if (!c.gm_j) KFBI_CUDA_TRY(cudaMalloc((void**)&c.gm_j, sizeof(int)));
  if (!c.d_flags) {
    void* p = nullptr;
    KFBI_CUDA_TRY(cudaHostGetDevicePointer(&p, c.h_pinned, 0));
    c.d_flags = static_cast<double*>(p) + 8;
  }
  if (c.gm_m >= m && c.basis) return KFBI_OK;
  drop_step_graphs(c);           // captured with the old workspace
  if (c.basis) {
    cudaFree(c.basis); cudaFree(c.hess); cudaFree(c.givens); cudaFree(c.gvec);
    cudaFree(c.hcol); cudaFree(c.yvec); cudaFree(c.gm_part); cudaFree(c.gm_counter);
  }
  const int M = c.M;
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.basis, sizeof(double) * (size_t)(m + 1) * M));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.hess, sizeof(double) * (size_t)(m + 1) * m));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.givens, sizeof(double) * 2 * m));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.gvec, sizeof(double) * (m + 1)));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.hcol, sizeof(double) * 2 * (m + 1)));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.yvec, sizeof(double) * m));
  const size_t nparts = std::max((size_t)dot_blocks(M) * (m + 1), (size_t)mvu_blocks(M));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.gm_part, sizeof(double) * nparts));
  KFBI_CUDA_TRY(cudaMalloc((void**)&c.gm_counter, sizeof(unsigned)));
  KFBI_CUDA_TRY(cudaMemset(c.gm_counter, 0, sizeof(unsigned)));
  for (int i = 0; i < 2; ++i)
    if (!c.gm_ev[i]) KFBI_CUDA_TRY(cudaEventCreateWithFlags(&c.gm_ev[i], cudaEventDisableTiming));
  c.gm_m = m;
  return KFBI_OK;
}

// The operator of the BIE being solved: K_D = v^+ of the double layer (Dirichlet BVP) or
// K_N = d_n v^+ of the single layer (Neumann BVP)
static kfbi_status op_apply(Ctx& c, int precision, const double* x, double* y) {
  if (c.gm_op == kOpNeumann) return apply_potential(c, Layer::Single, precision, x, y, true);
  return apply_potential(c, Layer::Double, precision, x, y);
}

static kfbi_status apply_K(Ctx& c, int precision, const double* x, double* y, Counters& cnt) {
  if (precision == KFBI_MIXED_FP32 || precision == KFBI_TF32X3) ++cnt.applies32;
  else ++cnt.applies64;   // FP64-accurate
  return op_apply(c, precision, x, y);
}

static kfbi_status read_scal(Ctx& c, int n) {
  KFBI_CUDA_TRY(cudaMemcpyAsync(c.h_pinned, c.scal, sizeof(double) * n, cudaMemcpyDeviceToHost,
                                c.stream));
  KFBI_CUDA_TRY(cudaStreamSynchronize(c.stream));
  return KFBI_OK;
}

// Arnoldi-step flags through two host-mapped slots (h_pinned[8..11], [12..15], written by
// finish_kernel) and two events
static kfbi_status post_flags(Ctx& c, int j) {
  KFBI_CUDA_TRY(cudaEventRecord(c.gm_ev[j & 1], c.stream));
  return KFBI_OK;
}

static kfbi_status wait_flags(Ctx& c, int j, const double** flags) {
  KFBI_CUDA_TRY(cudaEventSynchronize(c.gm_ev[j & 1]));
  *flags = c.h_pinned + 8 + 4 * (j & 1);
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

// One Arnoldi step with the matvec in precision `prec`: the apply of vin (V_j) into w, the
// two classical Gram-Schmidt passes against V_0..V_j, the normalisation into V_{j+1} (and
// vin) with the Givens update, and the step index advance.  j lives in device memory, so
// this launch sequence is the same at every step.
static kfbi_status arnoldi_step(Ctx& c, int prec) {
  const int M = c.M, m = c.opt.gmres_m;
  cudaStream_t st = c.stream;
  double* w = c.vecs + M;
  double* vin = c.vecs + 6 * M;
  double* h1 = c.hcol;
  double* h2 = c.hcol + (m + 1);
  KFBI_TRY(op_apply(c, prec, vin, w));
  const int pk = prof_begin(c, ST_KRYLOV);
  prof_count(c, ST_KRYLOV, 4);
  const dim3 dg(dot_blocks(M), m + 1);
  const int ub = mvu_blocks(M), ut = MVU_X * MVU_SLICES;
  multidot_kernel<<<dg, DOT_T, 0, st>>>(c.basis, M, M, 0, c.gm_j, w, c.gm_part, m + 1,
                                        c.gm_counter, h1);
  mv_update_kernel<<<ub, ut, 0, st>>>(w, c.basis, M, M, h1, 0, c.gm_j, -1.0, nullptr, nullptr,
                                      nullptr);
  multidot_kernel<<<dg, DOT_T, 0, st>>>(c.basis, M, M, 0, c.gm_j, w, c.gm_part, m + 1,
                                        c.gm_counter, h2);
  mv_update_kernel<<<ub, ut, 0, st>>>(w, c.basis, M, M, h2, 0, c.gm_j, -1.0, c.gm_part,
                                      c.gm_counter, c.scal + 5);
  finish_kernel<<<vb(M), 256, sizeof(double) * (3 * m + 1), st>>>(
      c.gm_j, m, M, w, c.basis, M, h1, h2, c.scal + 5, c.hess, c.givens, c.gvec, c.scal, vin,
      c.d_flags, c.gm_counter);
  prof_end(c, pk);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

// The Arnoldi step as one CUDA graph per matvec precision, captured on first use (the
// kernels and their arguments are the same at every step of every cycle of this context),
// launched with one call; direct launches while the stage timers run or if capture is not
// possible.  A graph's kernel launches are added to the launch counters at every replay.
static kfbi_status launch_step(Ctx& c, int prec) {
  if (c.prof.on || !c.graphs_ok || prec < 0 || prec >= kStepGraphs) return arnoldi_step(c, prec);
  if (c.graph_m != c.opt.gmres_m) {   // captured with another restart length
    drop_step_graphs(c);
    c.graph_m = c.opt.gmres_m;
  }
  cudaGraphExec_t& exec = c.step_exec[c.gm_op][prec];
  long long* counts = c.step_launches[c.gm_op][prec];
  if (!exec) {
    long long before[KFBI_NSTAGES];
    for (int s = 0; s < KFBI_NSTAGES; ++s) before[s] = c.prof.launches[s];
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      c.graphs_ok = false;
      return arnoldi_step(c, prec);
    }
    const kfbi_status body = arnoldi_step(c, prec);
    const cudaError_t ec = cudaStreamEndCapture(c.stream, &g);
    for (int s = 0; s < KFBI_NSTAGES; ++s) {   // captured, not run: counted per replay
      counts[s] = c.prof.launches[s] - before[s];
      c.prof.launches[s] = before[s];
    }
    cudaGraphExec_t ex = nullptr;
    const bool ok = body == KFBI_OK && ec == cudaSuccess && g &&
                    cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {                   // nothing ran: take the step with direct launches
      cudaGetLastError();
      c.graphs_ok = false;
      return arnoldi_step(c, prec);
    }
    exec = ex;
  }
  KFBI_CUDA_TRY(cudaGraphLaunch(exec, c.stream));
  for (int s = 0; s < KFBI_NSTAGES; ++s) c.prof.launches[s] += counts[s];
  return KFBI_OK;
}

// GMRES(m) on K_D for rhs, x in/out (x_zero: start from 0), FP64 Arnoldi, matvec
// precision chosen per step by `relax`.  Every cycle ends with the true residual formed
// with the FP64-accurate apply prec_true (an iterative-refinement step).  Stops when the
// residual is <= tol_abs; *res_out = last true residual norm.
static kfbi_status gmres_run(Ctx& c, const Relax& relax, int prec_true, const double* rhs,
                             double* x, bool x_zero, double tol_abs, int max_cycles,
                             Counters& cnt, double* res_out, int* cycles_out) {
  const int M = c.M, m = c.opt.gmres_m;   // workspace is sized for c.gm_m >= m
  cudaStream_t st = c.stream;
  double* r = c.vecs;            // residual
  double* tmp = c.vecs + 2 * M;
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
  if (!std::isfinite(beta)) {
    set_error("GMRES: non-finite residual norm (NaN or Inf in the data or the iteration)");
    return KFBI_ERR_NUMERIC;
  }
  int cyc = 0;
  for (; cyc < max_cycles && beta > tol_abs; ++cyc) {
    prof_count(c, ST_KRYLOV);
    cycle_start_kernel<<<vb(M > m + 1 ? M : m + 1), 256, 0, st>>>(c.basis, c.vecs + 6 * M, r, M,
                                                                   c.gvec, m, c.scal, c.gm_j);
    // The host runs one Arnoldi step ahead of the device: the flags of step j (residual
    // estimate, breakdown, NaN) are copied to a pinned slot behind step j's kernels and
    // read only after step j + 1 has been enqueued, so the device never idles on a host
    // round trip.  The matvec precision of step j is picked from the estimate of step
    // j - 2 (estimates only decrease, so an older one errs towards higher precision).
    // When step p reports convergence or breakdown, the step p + 1 already enqueued is
    // kept if it is finite and did not break down itself (one more Arnoldi step only
    // lowers the GMRES residual).
    int k = 0;
    double est = beta;
    int pending = -1;
    for (int j = 0; j < m; ++j) {
      const int prec = relax.pick(est);
      if (prec == KFBI_MIXED_FP32 || prec == KFBI_TF32X3) ++cnt.applies32;
      else ++cnt.applies64;   // FP64-accurate
      KFBI_TRY(launch_step(c, prec));
      ++cnt.iters;
      KFBI_TRY(post_flags(c, j));
      k = j + 1;
      if (pending >= 0) {
        const double* f = nullptr;
        KFBI_TRY(wait_flags(c, pending, &f));
        if (f[3] != 0.0) {
          set_error("GMRES: non-finite Arnoldi vector");
          return KFBI_ERR_NUMERIC;
        }
        est = f[0];
        if (est <= tol_abs || f[1] != 0.0) {
          const bool broke = f[1] != 0.0;
          KFBI_TRY(wait_flags(c, j, &f));
          k = (!broke && f[3] == 0.0 && f[1] == 0.0) ? j + 1 : j;
          pending = -1;
          break;
        }
      }
      pending = j;
    }
    if (pending >= 0) {             // the last step's flags (cycle ended at m steps)
      const double* f = nullptr;
      KFBI_TRY(wait_flags(c, pending, &f));
      if (f[3] != 0.0) {
          set_error("GMRES: non-finite Arnoldi vector");
          return KFBI_ERR_NUMERIC;
        }
    }
    prof_count(c, ST_KRYLOV, 2);
    const size_t lsm = sizeof(double) * (size_t)k * (k + 2);
    const bool staged = lsm <= 48 * 1024;
    lsq_kernel<<<1, 256, staged ? lsm : sizeof(double) * 2 * k, st>>>(k, m, c.hess, c.gvec, c.yvec,
                                                                       staged ? 1 : 0);
    mv_update_kernel<<<mvu_blocks(M), MVU_X * MVU_SLICES, 0, st>>>(x, c.basis, M, M, c.yvec, k,
                                                                  nullptr, 1.0, nullptr, nullptr,
                                                                  nullptr);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(apply_K(c, prec_true, x, tmp, cnt));
    prof_count(c, ST_KRYLOV, 2);
    sub_kernel<<<vb(M), 256, 0, st>>>(r, rhs, tmp, M);
    norm_kernel<<<1, 1024, 0, st>>>(r, M, c.scal, 2);
    KFBI_TRY(read_scal(c, 4));
    beta = c.h_pinned[2];
    if (!std::isfinite(beta)) {
      set_error("GMRES: non-finite residual norm (NaN or Inf in the data or the iteration)");
      return KFBI_ERR_NUMERIC;
    }
  }
  *res_out = beta;
  if (cycles_out) *cycles_out = cyc;
  return KFBI_OK;
}

static kfbi_status solve_bvp_on(Ctx& c, int op, const double* f_grid, const double* f_ctrl,
                                const double* g_ctrl, double* u_grid, double* dens_out,
                                kfbi_solve_info* info);

// The solve runs on the context's own non-blocking stream (the captured Arnoldi-step graphs
// need a stream that can be captured; the legacy default stream cannot), joined to the
// caller's stream at both ends: it starts after the work already queued there, and the
// caller's stream waits for it.  op: kOpDirichlet (g = u on Gamma, double-layer density)
// or kOpNeumann (g = d_n u on Gamma, single-layer density).
kfbi_status solve_bvp(Ctx& c, const double* f_grid, const double* f_ctrl, const double* g_ctrl,
                      double* u_grid, double* dens_out, kfbi_solve_info* info, int op) {
  const cudaStream_t caller = c.stream;
  if (!c.own) return solve_bvp_on(c, op, f_grid, f_ctrl, g_ctrl, u_grid, dens_out, info);
  KFBI_CUDA_TRY(cudaEventRecord(c.own_in, caller));
  KFBI_CUDA_TRY(cudaStreamWaitEvent(c.own, c.own_in, 0));
  c.stream = c.own;
  const kfbi_status s = solve_bvp_on(c, op, f_grid, f_ctrl, g_ctrl, u_grid, dens_out, info);
  c.stream = caller;
  KFBI_CUDA_TRY(cudaEventRecord(c.own_out, c.own));
  KFBI_CUDA_TRY(cudaStreamWaitEvent(caller, c.own_out, 0));
  return s;
}

static kfbi_status solve_bvp_on(Ctx& c, int op, const double* f_grid, const double* f_ctrl,
                                const double* g_ctrl, double* u_grid, double* dens_out,
                                kfbi_solve_info* info) {
  const int M = c.M;
  const bool neumann = op == kOpNeumann;
  if (neumann && c.dim != 2) {
    set_error("Neumann BVP: 2-D only");
    return KFBI_ERR_UNSUPPORTED;
  }
  c.gm_op = op;
  cudaStream_t st = c.stream;
  KFBI_TRY(alloc_gmres(c, c.opt.gmres_m));
  // precision of every step that must be FP64-accurate: FP64 transforms in the plain FP64
  // solver, FP32 transforms with FP64 residual refinement otherwise
  const int acc = c.opt.precision == KFBI_FP64 ? KFBI_FP64 : KFBI_FP32_REFINED;
  double* ghat = c.vecs + 3 * M;
  double* phi = c.vecs + 4 * M;
  double* d = c.vecs + 5 * M;
  Counters cnt;
  // bounded waits that give up during this solve are reported by this solve
  KFBI_CUDA_TRY(cudaMemsetAsync(c.err_flag + 2, 0, sizeof(int), st));
  // g_hat = g - (Y f)^+  (Neumann: g - d_n (Y f)^+)
  KFBI_TRY(interface_solve(c, acc, nullptr, f_grid, f_ctrl, nullptr, nullptr, d, nullptr, neumann));
  ++cnt.applies64;
  prof_count(c, ST_KRYLOV, 2);
  sub_kernel<<<vb(M), 256, 0, st>>>(ghat, g_ctrl, d, M);
  norm_kernel<<<1, 1024, 0, st>>>(ghat, M, c.scal, 4);
  KFBI_TRY(read_scal(c, 5));
  const double gnorm = c.h_pinned[4];
  const double tol_abs = c.opt.tol * gnorm;
  double res = 0.0;
  int cycles = 0;
  if (c.opt.precision == KFBI_MIXED_FP32 || c.opt.precision == KFBI_TF32X3) {
    // twice-refined applies (about 1e-13) while the residual is above tol / 1e-9,
    // once-refined (about 1e-10 at the largest grids) down to tol / inner_tol, plain FP32
    // (FFT or tensor-core transforms) below (inner_tol: the assumed relative accuracy of
    // an FP32 apply)
    const Relax relax{{KFBI_FP32_REFINED, KFBI_FP32_REFINED_ONCE, c.opt.precision},
                      {tol_abs / 1e-9, tol_abs / c.opt.inner_tol}};
    KFBI_TRY(gmres_run(c, relax, acc, ghat, phi, true, tol_abs, c.opt.max_restarts + 1, cnt,
                       &res, &cycles));
  } else {
    const Relax relax{{acc, acc, acc}, {0.0, 0.0}};
    KFBI_TRY(gmres_run(c, relax, acc, ghat, phi, true, tol_abs, c.opt.max_restarts + 1, cnt,
                       &res, &cycles));
  }
  // u = W phi + Y f (Neumann: V psi + Y f) on inside nodes
  if (u_grid) {
    if (neumann) KFBI_TRY(combined_u(c, acc, nullptr, f_grid, f_ctrl, u_grid, phi));
    else KFBI_TRY(combined_u(c, acc, phi, f_grid, f_ctrl, u_grid));
    ++cnt.applies64;
  }
  if (dens_out)
    KFBI_CUDA_TRY(cudaMemcpyAsync(dens_out, phi, sizeof(double) * M, cudaMemcpyDeviceToDevice, st));
  int timeout = 0;           // a bounded wait of a transform kernel that gave up
  KFBI_CUDA_TRY(cudaMemcpyAsync(&timeout, c.err_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  if (timeout) {
    set_error("BVP solve: a staged line copy did not complete (bounded wait expired)");
    return KFBI_ERR_TIMEOUT;
  }
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

// Batched BVPs: a pool of host workers, each with its own CUDA stream, takes problems from
// a shared queue in decreasing order of cost ((N+1)^dim log N per apply; longest first)
// and solves all right-hand sides of a problem in turn.  Problems never share a context,
// so their solves run concurrently on the device; the caller's stream is joined at both
// ends (the batch starts after work already on it and is complete when the call returns).
kfbi_status batch_solve(kfbi_ctx* ctxs, int count, int nrhs, const double* const* f_grid,
                        const double* const* f_ctrl, const double* const* g_ctrl,
                        double* const* u_grid, double* const* dens_out, kfbi_solve_info* info,
                        cudaStream_t stream) {
  int dev = 0;
  KFBI_CUDA_TRY(cudaGetDevice(&dev));
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  auto cost = [&](int p) {
    const Ctx& c = ctxs[p]->c;
    const double n = c.N + 1.0;
    return (c.dim == 3 ? n * n * n : n * n) * std::log2((double)c.N);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  // KFBI_BATCH_WORKERS (1..64) overrides the number of concurrent problems
  int nw = kBatchWorkers;
  if (const char* e = std::getenv("KFBI_BATCH_WORKERS")) {
    const int v = std::atoi(e);
    if (v >= 1 && v <= 64) nw = v;
  }
  const int workers = std::max(1, std::min(count, nw));
  cudaEvent_t start;
  KFBI_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  KFBI_CUDA_TRY(cudaEventRecord(start, stream));
  std::atomic<int> next{0};
  std::vector<kfbi_status> wstatus(workers, KFBI_OK);
  std::vector<std::string> wmsg(workers);
  std::vector<int> not_converged(workers, 0);
  auto work = [&](int w) {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(st, start, 0) != cudaSuccess) {
      wstatus[w] = KFBI_ERR_CUDA;
      wmsg[w] = "kfbi_batch_solve: stream creation failed";
      if (st) cudaStreamDestroy(st);
      return;
    }
    for (int k = next.fetch_add(1); k < count; k = next.fetch_add(1)) {
      const int p = order[k];
      Ctx& c = ctxs[p]->c;
      c.stream = st;
      for (int r = 0; r < nrhs; ++r) {
        const int q = p * nrhs + r;
        const kfbi_status s = solve_bvp(c, f_grid[q], f_ctrl[q], g_ctrl[q], u_grid[q],
                                        dens_out ? dens_out[q] : nullptr,
                                        info ? info + q : nullptr, kOpDirichlet);
        if (s == KFBI_ERR_NOT_CONVERGED) {
          not_converged[w] = 1;
        } else if (s != KFBI_OK) {
          wstatus[w] = s;
          wmsg[w] = last_error_message();
          next.store(count);               // stop the other workers at their next problem
          break;
        }
      }
      c.stream = stream;
      if (wstatus[w] != KFBI_OK) break;
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(work, w);
  work(0);
  for (auto& t : pool) t.join();
  cudaEventDestroy(start);
  for (int w = 0; w < workers; ++w)
    if (wstatus[w] != KFBI_OK) {
      set_error("%s", wmsg[w].c_str());
      return wstatus[w];
    }
  for (int w = 0; w < workers; ++w)
    if (not_converged[w]) return KFBI_ERR_NOT_CONVERGED;
  return KFBI_OK;
}

}  // namespace kfbi
