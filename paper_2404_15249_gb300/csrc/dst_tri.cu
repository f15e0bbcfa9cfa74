// y-direction solve of the 2-D box solve for the well-conditioned x-modes, in FP32.
//
// After the x-transform, line k of the transposed work grid (x-mode k) needs the solution of
//     (T_y + lambda_k - kappa^2) v = x_k,   T_y = tridiag(1, -2, 1) / h^2,  v_0 = v_N = 0,
// which the FFT pass computes as (2/N) S diag(1 / (lambda_k + lambda_l - kappa^2)) S x_k
// (Alg. 4, the sine transform along y).  For modes with |lambda_k| well above 1/N^2 of the
// spectrum the system is strictly and strongly diagonally dominant, so the tridiagonal
// solve of Alg. 4's form (elimination along the line, here along y) is accurate in FP32
// and costs a few operations per point instead of two transforms.  The elimination
// coefficients converge geometrically to the fixed point c* of c = A / (D - A c) (A = 1/h^2,
// D = -2/h^2 + lambda_k - kappa^2, |c*| < 1): a line is split into 32 (64 from N = 2048)
// chunks, one per thread; each thread starts its forward and backward recursions w points
// early (inside the neighbouring chunk, |c*|^w <= 1e-8, w <= TRI_W) from a zero state, an
// error that decays like |c*|^w, and the first TRI_EXACT coefficients of the line are the
// exact ones, from the closed form
// c'_j = c* (1 - c*^2j) / (1 - c*^(2j+2)) of the recursion with c'_0 = 0.  The modes used
// here are those with |c*| <= TRI_CMAX; the lower modes stay on the FFT pass.
#include <atomic>
#include <cmath>

#include "kfbi_internal.cuh"

namespace kfbi {
namespace {

constexpr int TRI_W = 96;          // longest warm-up of a chunk's recursions
constexpr double TRI_CMAX = 0.825; // |c*| <= 0.825: |c*|^96 <= 1e-8
constexpr int TRI_THREADS = 128;   // threads per block: 128 / CH lines of CH chunks each
constexpr int TRI_EXACT = 64;      // leading coefficients computed exactly (|c*|^128 < 1e-10)

// padded shared-memory index of point j: chunk L (M points) starts at L (M + 1), so the
// lanes walking their chunks in step hit 32 different banks
template <int N, int CH>
__device__ __forceinline__ int tpad(int j) {
  constexpr int M = N / CH;
  return j + j / M;
}

// CH chunks (threads) per line; the block's lines advance together (block barriers)
template <int N, int CH>
__global__ void __launch_bounds__(TRI_THREADS)
    ytri_kernel(float* __restrict__ X, int k0, const float* __restrict__ lam, float kappa2,
                float inv_h2, float scale) {
  constexpr int M = N / CH, LPB = TRI_THREADS / CH;
  constexpr int LINE = N + CH + 2 * TRI_EXACT;     // padded line + exact coefficients
  static_assert(M >= 1 && LPB >= 1, "chunking");
  extern __shared__ float sm[];
  const int sub = threadIdx.x / CH, lane = threadIdx.x % CH;
  float* buf = sm + sub * LINE;
  float* cpx = buf + N + CH;                        // exact c'_j, j < TRI_EXACT
  float* idx = cpx + TRI_EXACT;                     // exact 1 / den_j
  const float A = inv_h2;
  for (int kb = k0 + blockIdx.x * LPB; kb < N; kb += gridDim.x * LPB) {
    const int k = kb + sub;
    const bool act = k < N;
    float* line = X + (size_t)(act ? k : kb) * N;
    // load the line (16-byte loads, padded stores)
    if (act)
      for (int q = lane; q < N / 4; q += CH) {
        const float4 v = reinterpret_cast<const float4*>(line)[q];
        const int j = 4 * q;
        buf[tpad<N, CH>(j)] = v.x;
        buf[tpad<N, CH>(j + 1)] = v.y;
        buf[tpad<N, CH>(j + 2)] = v.z;
        buf[tpad<N, CH>(j + 3)] = v.w;
      }
    const float D = fmaf(-2.f, A, lam[act ? k : kb] - kappa2);
    // fixed point c* = 2A / (D - sqrt(D^2 - 4A^2)) (no cancellation: D < 0), 1/den = c*/A
    const float disc = sqrtf(fmaf(D, D, -4.f * A * A));
    const float cs = 2.f * A / (D - disc);
    const float gs = cs / A;
    // warm-up of this line: |c*|^w <= 1e-8 (at most TRI_W)
    const int w = min(TRI_W, (int)ceilf(-18.42f / logf(fabsf(cs))) + 1);
    const float lc2 = 2.f * log2f(fabsf(cs));    // log2 c*^2
    for (int j = lane; j < TRI_EXACT; j += CH) {
      const float q = exp2f(lc2 * (float)j);      // c*^2j
      const float c = cs * (1.f - q) / fmaf(-q, cs * cs, 1.f);
      cpx[j] = c;
      idx[j] = c / A;                             // 1 / den_j = c'_j / A
    }
    __syncthreads();
    const int s = lane * M, e = s + M;
    const int s1 = s < 1 ? 1 : s;                  // point 0 is the boundary
    // the thread's chunk in registers: the recursions' dependency chains then run on
    // register operands, shared memory is only read by the warm-ups and the final store
    float r[M];
#pragma unroll
    for (int i = 0; i < M; ++i) r[i] = buf[tpad<N, CH>(s + i)];
    // forward elimination y_j = (x_j - A y_{j-1}) / den_j: warm-up on the previous
    // chunk's values, then the own chunk
    float y = 0.f;
#pragma unroll 4
    for (int j = (s1 - w > 1 ? s1 - w : 1); j < s1; ++j)
      y = (buf[tpad<N, CH>(j)] - A * y) * (j < TRI_EXACT ? idx[j] : gs);
#pragma unroll
    for (int i = 0; i < M; ++i) {
      const int j = s + i;
      if (j >= 1) {
        y = (r[i] - A * y) * (j < TRI_EXACT ? idx[j] : gs);
        r[i] = y;
      }
    }
    __syncthreads();                               // every warm-up read the input values
#pragma unroll
    for (int i = 0; i < M; ++i) buf[tpad<N, CH>(s + i)] = r[i];
    __syncthreads();
    // back substitution v_j = y_j - c'_j v_{j+1} (v_N = 0): warm-up on the next chunk's
    // y, then the own chunk, scaled
    float v = 0.f;
#pragma unroll 4
    for (int j = (e - 1 + w < N - 1 ? e - 1 + w : N - 1); j >= e; --j)
      v = buf[tpad<N, CH>(j)] - (j < TRI_EXACT ? cpx[j] : cs) * v;
#pragma unroll
    for (int i = M - 1; i >= 0; --i) {
      const int j = s + i;
      if (j >= 1) {
        v = r[i] - (j < TRI_EXACT ? cpx[j] : cs) * v;
        r[i] = v * scale;
      } else {
        r[i] = 0.f;
      }
    }
    __syncthreads();                               // every warm-up read the y values
#pragma unroll
    for (int i = 0; i < M; ++i) buf[tpad<N, CH>(s + i)] = r[i];
    __syncthreads();
    if (act)
      for (int q = lane; q < N / 4; q += CH) {
        const int j = 4 * q;
        reinterpret_cast<float4*>(line)[q] =
            make_float4(buf[tpad<N, CH>(j)], buf[tpad<N, CH>(j + 1)], buf[tpad<N, CH>(j + 2)],
                        buf[tpad<N, CH>(j + 3)]);
      }
    __syncthreads();
  }
}

// 64 chunks per line from N = 2048 (shorter recursions per thread), 32 below
template <int N>
kfbi_status launch_tri(Ctx& c, float* X, int k0) {
  constexpr int CH = N >= 4096 ? 128 : (N >= 2048 ? 64 : 32);
  constexpr int LPB = TRI_THREADS / CH;
  constexpr size_t smem = (size_t)LPB * (N + CH + 2 * TRI_EXACT) * sizeof(float);
  static_assert(smem <= 227 * 1024, "tridiagonal pass exceeds shared memory");
  KFBI_TRY(set_smem_limit((const void*)ytri_kernel<N, CH>, smem));
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ytri_kernel<N, CH>,
                                                              TRI_THREADS, smem));
  int dev = 0, sms = 0;
  KFBI_CUDA_TRY(cudaGetDevice(&dev));
  KFBI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int lines = N - k0;
  int blocks = (lines + LPB - 1) / LPB;
  const int cap = (per_sm < 1 ? 1 : per_sm) * sms;
  if (blocks > cap) blocks = cap;
  const int pr = prof_begin(c, ST_TRI);
  ytri_kernel<N, CH><<<blocks, TRI_THREADS, smem, c.stream>>>(
      X, k0, c.t32.lam, (float)c.kappa2, (float)(1.0 / (c.h * c.h)), (float)(2.0 / N));
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace

// the smallest x-mode k >= 1 with |c*(k)| <= cmax, in FP64 on the host, rounded up to a
// multiple of 32 (N: none); KFBI_TRI=0 keeps every mode on the FFT pass
static int first_mode_below(const Ctx& c, double cmax) {
  if (const char* e = std::getenv("KFBI_TRI"))
    if (e[0] == '0') return c.N;
  if (c.dim != 2 || c.N < 64) return c.N;
  const double h2 = c.h * c.h;
  for (int k = 1; k < c.N; ++k) {
    const double sk = std::sin(M_PI * k / (2.0 * c.N));
    const double mu = 4.0 * sk * sk + h2 * c.kappa2;           // -D h^2 - 2
    const double cst = 2.0 / ((2.0 + mu) + std::sqrt((2.0 + mu) * (2.0 + mu) - 4.0));
    // rounded up to a multiple of 32: the filter pass then moves whole 128-byte rows of
    // 32 modes (the extra modes take the transform pair, accurate for every mode)
    if (cst <= cmax) return ((k + 31) / 32) * 32 < c.N ? ((k + 31) / 32) * 32 : c.N;
  }
  return c.N;
}

// first x-mode of the tridiagonal pass (transposed layout): |c*(k)| <= TRI_CMAX
int tri_first_mode(const Ctx& c) { return first_mode_below(c, TRI_CMAX); }

// first x-mode of the recursive filters of the row-layout y-pass: |c*(k)| <= 0.9 (warm-ups
// of at most 176 rows; the filters' FP32 error for the mode at the threshold is 4.7e-7 of
// its amplitude, modelled in numpy at N = 4096, against 3.4e-7 at 0.825 and 9.9e-7 at 0.95;
// 0.9 to 0.95 gave the same solve time at N = 4096, 0.88 and 0.97 slower)
int ypass_first_mode(const Ctx& c) { return first_mode_below(c, 0.9); }

kfbi_status ytri_f32(Ctx& c, float* X, int k0) {
  if (k0 >= c.N) return KFBI_OK;
  switch (c.N) {
#define KFBI_TRI_CASE(n) \
  case n: return launch_tri<n>(c, X, k0);
    KFBI_TRI_CASE(64) KFBI_TRI_CASE(96) KFBI_TRI_CASE(128) KFBI_TRI_CASE(192)
    KFBI_TRI_CASE(256) KFBI_TRI_CASE(384) KFBI_TRI_CASE(512) KFBI_TRI_CASE(768)
    KFBI_TRI_CASE(1024) KFBI_TRI_CASE(1536) KFBI_TRI_CASE(2048) KFBI_TRI_CASE(3072)
    KFBI_TRI_CASE(4096) KFBI_TRI_CASE(6144) KFBI_TRI_CASE(8192)
#undef KFBI_TRI_CASE
    default:
      set_error("tridiagonal y-pass: unsupported N = %d", c.N);
      return KFBI_ERR_UNSUPPORTED;
  }
}

}  // namespace kfbi
