// y-direction pass of the FP32 2-D box solve on the row layout (Alg. 4 with the axes of the
// transform and of the tridiagonal solve swapped): after the sine transform along x, column
// k of the work grid V (node (i, j) at j N + i, so column k is x-mode k along y) needs
//     (T_y + lambda_k - kappa^2) v = x,   T_y = tridiag(1, -2, 1) / h^2,  v_0 = v_N = 0,
// then the inverse x-transform's scale 2/N.
//
// Well-conditioned modes (k >= k0, the elimination coefficient |c| <= 0.9): the operator
// of the scaled system  v_{j-1} - mu v_j + v_{j+1} = h^2 x_j,  mu = 2 + h^2 (kappa^2 - lambda_k),
// factors on infinite sequences as -(1/c) (I - c S-)(I - c S+) with c + 1/c = mu, 0 < c < 1
// (S-, S+ the shifts), so v = -c h^2 F+ F- x with the causal filter F-: u_j = x_j + c u_{j-1}
// and the anticausal filter F+: z_j = u_j + c z_{j+1}, which commute.  Extending x as an odd,
// 2N-periodic sequence (x_{-j} = -x_j, x_{N+j} = -x_{N-j}, x_0 = x_N = 0) makes the bounded
// solution odd about 0 and N, so it is the finite system's solution with v_0 = v_N = 0.
// A thread owns one mode (consecutive modes across a warp: every row access is one
// coalesced 128-byte segment) and one chunk of MC rows: it runs F+ down from w rows past its
// chunk (the truncated tail weighs c^w <= 1e-8; w <= 176), keeps the chunk's values in registers,
// continues F+ over the w rows before the chunk while summing the causal state
// u_{s-1} = sum_m c^m z_{s-1-m}, then runs F- forward over the chunk.  The warm-ups read
// rows of the neighbouring chunks, which other warps own, so the pass is out of place: it
// reads V and writes the result grid Y.  Low modes (k < k0) take the sine-transform pair
// along y on a side stream while the filters run, gathering their columns of V and
// scattering them into Y directly (ycol_lines_kernel).
#include <cmath>
#include <cstdint>

#include "kfbi_internal.cuh"

namespace kfbi {
namespace {

constexpr int YC_W = 176;           // longest warm-up (before rounding up to 16): 0.9^176 < 1e-8
constexpr int YC_WARPS = 8;         // warps per CTA: 8 consecutive chunks of the same 32 modes
constexpr int YC_THREADS = 32 * YC_WARPS;

// c of mode k: the root in (0, 1) of c^2 - mu c + 1, mu = 2 + h^2 (kappa^2 - lambda_k)
__device__ __forceinline__ float filter_c(const float* lam, int k, float h2, float h2k2) {
  const float mu = 2.f + (h2k2 - h2 * lam[k]);
  return 2.f / (mu + sqrtf(fmaf(mu, mu, -4.f)));
}

// The filters of one chunk [s, s + MC) of one mode (column col, coefficient c) with W rows
// of warm-up each side; INNER: every row read lies in [0, N) (row 0 holds zeros), else rows
// outside follow the odd 2N-periodic extension (|j| < 2N here, so one shift by 2N and one
// mirror suffice).  Rows are read in unrolled batches of 16 so that many loads are in
// flight.  Returns the chunk's solution rows in r.
template <int MC, bool INNER>
__device__ __forceinline__ void filter_chunk(const float* __restrict__ col, int N, int s, int W,
                                             float c, float g, float (&r)[MC]) {
  constexpr int B = 16;
  const int N2 = 2 * N;
  auto load = [&](int j) -> float {
    if constexpr (INNER) {
      return col[(size_t)j * N];
    } else {
      int m = j;
      m += m < 0 ? N2 : 0;
      m -= m >= N2 ? N2 : 0;
      const bool neg = m > N;
      const int src = neg ? N2 - m : m;
      const float x = (m != 0 && m != N) ? col[(size_t)src * N] : 0.f;
      return neg ? -x : x;
    }
  };
  const int e = s + MC;
  float z = 0.f;
  for (int jb = e + W - B; jb >= e; jb -= B) {                     // F+ warm-up, far end first
    float x[B];
#pragma unroll
    for (int u = 0; u < B; ++u) x[u] = load(jb + u);
#pragma unroll
    for (int u = B - 1; u >= 0; --u) z = fmaf(c, z, x[u]);
  }
#pragma unroll
  for (int i = 0; i < MC; ++i) r[i] = col[(size_t)(s + i) * N];
#pragma unroll
  for (int i = MC - 1; i >= 0; --i) {                              // F+ over the chunk
    z = fmaf(c, z, r[i]);
    r[i] = z;
  }
  float u = 0.f, p = 1.f;                                          // causal state entering s
  for (int jb = s - B; jb >= s - W; jb -= B) {
    float x[B];
#pragma unroll
    for (int q = 0; q < B; ++q) x[q] = load(jb + q);
#pragma unroll
    for (int q = B - 1; q >= 0; --q) {
      z = fmaf(c, z, x[q]);
      u = fmaf(p, z, u);
      p *= c;
    }
  }
#pragma unroll
  for (int i = 0; i < MC; ++i) {                                   // F- over the chunk
    u = fmaf(c, u, r[i]);
    r[i] = u * g;
  }
}

// Warp w of CTA (b, g) owns modes k0 + 32 g + lane and chunk b YC_WARPS + w of MC rows; W
// comes from the group's lowest mode, whose c is the largest, rounded up to a multiple of
// 16.  Every access is one coalesced 128-byte row segment (the group's 32 modes; k0 is a
// multiple of 32).  The groups vary slowest over the grid, so the lowest modes, whose
// warm-ups are the longest, start first.
template <int MC>
__global__ void __launch_bounds__(YC_THREADS)
    ycol_filter_kernel(const float* __restrict__ V, float* __restrict__ Y, int N, int k0,
                       const float* __restrict__ lam, float h2, float h2k2, float scale) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int kb = k0 + blockIdx.y * 32;
  const int k = kb + lane;
  const int s = (blockIdx.x * YC_WARPS + warp) * MC;               // first row of the chunk
  if (s >= N) return;                                              // uniform per warp
  const bool act = k < N;
  const int kk = act ? k : N - 1;                                  // idle lanes read a valid column
  // (at most N, so every row read, warm-ups included, lies within one period each side)
  const int W = min((min(YC_W, (int)ceilf(-18.43f / logf(filter_c(lam, kb, h2, h2k2))) + 1) + 15) / 16 * 16, N);
  const float c = filter_c(lam, kk, h2, h2k2);
  const float g = -c * h2 * scale;
  float r[MC];
  if (s - W >= 0 && s + MC + W <= N) filter_chunk<MC, true>(V + kk, N, s, W, c, g, r);
  else filter_chunk<MC, false>(V + kk, N, s, W, c, g, r);
  if (!act) return;
  float* out = Y + k;
#pragma unroll
  for (int i = 0; i < MC; ++i) out[(size_t)(s + i) * N] = (s + i == 0) ? 0.f : r[i];
}

template <int MC>
kfbi_status launch_filter(Ctx& c, const float* V, float* Y, int k0) {
  const int N = c.N;
  const dim3 grid((N + YC_WARPS * MC - 1) / (YC_WARPS * MC), (N - k0 + 31) / 32);
  const int pr = prof_begin(c, ST_TRI);
  ycol_filter_kernel<MC><<<grid, YC_THREADS, 0, c.stream>>>(
      V, Y, N, k0, c.t32.lam, (float)(c.h * c.h), (float)(c.h * c.h * c.kappa2), (float)(2.0 / N));
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace

// the y-pass of the FP32 2-D box solve from V into Y (row layout, Y != V); the low modes
// k < ypass_k0 take the transform pair on the side stream
kfbi_status ypass_rows_f32(Ctx& c, const float* V, float* Y) {
  const int N = c.N, k0 = c.ypass_k0;
  if (k0 <= 0 || k0 >= N || k0 % 32 != 0 || N % 32 != 0) {
    set_error("row-layout y-pass: needs 0 < k0 < N, both multiples of 32 (N = %d, k0 = %d)", N, k0);
    return KFBI_ERR_UNSUPPORTED;
  }
  // the stage timers take the y-pass as one span on the main stream (its kernels overlap)
  struct Span {
    Ctx& c;
    int pair;
    ~Span() { prof_span_end(c, pair); }
  } span{c, prof_span_begin(c, ST_TRI)};
  // fork: the low modes on the side stream, after everything already queued on the main one
  const cudaStream_t main_st = c.stream;
  KFBI_CUDA_TRY(cudaEventRecord(c.fork_ev, main_st));
  KFBI_CUDA_TRY(cudaStreamWaitEvent(c.side, c.fork_ev, 0));
  c.stream = c.side;                                               // launches go to the side stream
  const kfbi_status st = ycol_lines_f32(c, V, Y, k0);
  c.stream = main_st;
  KFBI_TRY(st);
  KFBI_CUDA_TRY(cudaEventRecord(c.join_ev, c.side));
  // the well-conditioned modes on the main stream, concurrently
  if (N >= 1024) KFBI_TRY(launch_filter<64>(c, V, Y, k0));
  else if (N >= 256) KFBI_TRY(launch_filter<32>(c, V, Y, k0));
  else KFBI_TRY(launch_filter<16>(c, V, Y, k0));
  KFBI_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev, 0));      // join
  return KFBI_OK;
}

}  // namespace kfbi
