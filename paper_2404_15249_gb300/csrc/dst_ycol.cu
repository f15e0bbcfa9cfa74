// y-direction pass of the FP32 2-D box solve on the row layout (Alg. 4 with the axes of the
// transform and of the tridiagonal solve swapped): after the sine transform along x, column
// k of the work grid V (node (i, j) at j N + i, so column k is x-mode k along y) needs
//     (T_y + lambda_k - kappa^2) v = x,   T_y = tridiag(1, -2, 1) / h^2,  v_0 = v_N = 0,
// then the inverse x-transform's scale 2/N.
//
// Well-conditioned modes (k >= k0, the elimination coefficient |c| <= 0.825): the operator
// of the scaled system  v_{j-1} - mu v_j + v_{j+1} = h^2 x_j,  mu = 2 + h^2 (kappa^2 - lambda_k),
// factors on infinite sequences as -(1/c) (I - c S-)(I - c S+) with c + 1/c = mu, 0 < c < 1
// (S-, S+ the shifts), so v = -c h^2 F+ F- x with the causal filter F-: u_j = x_j + c u_{j-1}
// and the anticausal filter F+: z_j = u_j + c z_{j+1}, which commute.  Extending x as an odd,
// 2N-periodic sequence (x_{-j} = -x_j, x_{N+j} = -x_{N-j}, x_0 = x_N = 0) makes the bounded
// solution odd about 0 and N, so it is the finite system's solution with v_0 = v_N = 0.
// A thread owns one mode (consecutive modes across a warp: every row access is one
// coalesced 128-byte segment) and one chunk of MC rows: it runs F+ down from w rows past its
// chunk (the truncated tail weighs c^w <= 1e-8), keeps the chunk's values in registers,
// continues F+ over the w rows before the chunk while summing the causal state
// u_{s-1} = sum_m c^m z_{s-1-m}, then runs F- forward over the chunk.  Low modes (k < k0)
// are copied out by a narrow transpose, take the sine-transform pair along y (yline_kernel)
// on a side stream while the filters run, and are copied back.
#include <cmath>

#include "kfbi_internal.cuh"

namespace kfbi {
namespace {

constexpr int YC_W = 97;            // longest warm-up: 0.825^97 < 1e-8
constexpr int YC_THREADS = 256;     // 8 warps: 8 consecutive chunks of the same 32 modes

template <int MC>
__global__ void __launch_bounds__(YC_THREADS)
    ycol_filter_kernel(float* __restrict__ V, int N, int k0, const float* __restrict__ lam,
                       float h2, float h2k2, float scale) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = k0 + blockIdx.x * 32 + lane;
  const int s = (blockIdx.y * (YC_THREADS / 32) + warp) * MC;     // first row of the chunk
  if (s >= N) return;                                              // uniform per warp
  const bool act = k < N;
  const int kk = act ? k : N - 1;                                  // idle lanes read a valid column
  const float mu = 2.f + (h2k2 - h2 * lam[kk]);
  const float c = 2.f / (mu + sqrtf(fmaf(mu, mu, -4.f)));          // root of c^2 - mu c + 1 in (0, 1)
  float cw = c;                                                    // the warp's largest c sets w
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cw = fmaxf(cw, __shfl_xor_sync(0xffffffffu, cw, o));
  const int w = min(YC_W, (int)ceilf(-18.43f / logf(cw)) + 1);
  const float* col = V + kk;
  const int N2 = 2 * N;
  auto ext = [&](int j) -> float {                                 // odd 2N-periodic extension
    int m = j % N2;
    m += m < 0 ? N2 : 0;
    if (m == 0 || m == N) return 0.f;
    return m < N ? col[(size_t)m * N] : -col[(size_t)(N2 - m) * N];
  };
  const int e = s + MC;
  float z = 0.f;
  for (int j = e + w - 1; j >= e; --j) z = fmaf(c, z, ext(j));     // F+ warm-up
  float r[MC];
#pragma unroll
  for (int i = MC - 1; i >= 0; --i) {                              // F+ over the chunk
    z = fmaf(c, z, col[(size_t)(s + i) * N]);
    r[i] = z;
  }
  float u = 0.f, p = 1.f;                                          // causal state entering s
  for (int j = s - 1; j >= s - w; --j) {
    z = fmaf(c, z, ext(j));
    u = fmaf(p, z, u);
    p *= c;
  }
  const float g = -c * h2 * scale;
#pragma unroll
  for (int i = 0; i < MC; ++i) {                                   // F- over the chunk
    u = fmaf(c, u, r[i]);
    r[i] = u * g;
  }
  if (!act) return;
  float* out = V + k;
#pragma unroll
  for (int i = 0; i < MC; ++i) out[(size_t)(s + i) * N] = (s + i == 0) ? 0.f : r[i];
}

// out[c][r] = in[r][c] for r < R, c < C; in has row stride ld_in, out row stride ld_out
// (32 x 32 tiles through shared memory)
__global__ void transpose_block_kernel(const float* __restrict__ in, int ld_in,
                                       float* __restrict__ out, int ld_out, int R, int C) {
  __shared__ float tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;            // column, row of the input tile
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int y = by + r, x = bx + threadIdx.x;
    if (x < C && y < R) tile[r][threadIdx.x] = in[(size_t)y * ld_in + x];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int y = bx + r, x = by + threadIdx.x;                    // row y of out = column y of in
    if (x < R && y < C) out[(size_t)y * ld_out + x] = tile[threadIdx.x][r];
  }
}

template <int MC>
kfbi_status launch_filter(Ctx& c, float* V, int k0) {
  const int N = c.N;
  const dim3 grid((N - k0 + 31) / 32, (N / MC + YC_THREADS / 32 - 1) / (YC_THREADS / 32));
  const int pr = prof_begin(c, ST_TRI);
  ycol_filter_kernel<MC><<<grid, YC_THREADS, 0, c.stream>>>(
      V, N, k0, c.t32.lam, (float)(c.h * c.h), (float)(c.h * c.h * c.kappa2), (float)(2.0 / N));
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status transpose_block(Ctx& c, const float* in, int ld_in, float* out, int ld_out, int R,
                            int C) {
  const int pr = prof_begin(c, ST_TRANS);
  transpose_block_kernel<<<dim3((C + 31) / 32, (R + 31) / 32), dim3(32, 8), 0, c.stream>>>(
      in, ld_in, out, ld_out, R, C);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace

// the y-pass of the FP32 2-D box solve on V in place (row layout); the low modes k < tri_k0
// run the transform pair in the context's transposed scratch on the side stream
kfbi_status ypass_rows_f32(Ctx& c, float* V) {
  const int N = c.N, k0 = c.tri_k0;
  if (k0 <= 0 || k0 >= N) {
    set_error("row-layout y-pass: no well-conditioned modes at N = %d", N);
    return KFBI_ERR_UNSUPPORTED;
  }
  float* L = reinterpret_cast<float*>(c.XT);                       // k0 x N low-mode lines
  // fork: the low modes on the side stream, after everything already queued on the main one
  const cudaStream_t main_st = c.stream;
  KFBI_CUDA_TRY(cudaEventRecord(c.fork_ev, main_st));
  KFBI_CUDA_TRY(cudaStreamWaitEvent(c.side, c.fork_ev, 0));
  c.stream = c.side;                                               // launches go to the side stream
  kfbi_status st = transpose_block(c, V, N, L, N, N, k0);          // L[k][j] = V[j][k]
  if (st == KFBI_OK) st = ylines_f32_lines(c, L, k0);
  if (st == KFBI_OK) st = transpose_block(c, L, N, V, N, k0, N);   // V[j][k] = L[k][j]
  c.stream = main_st;
  KFBI_TRY(st);
  KFBI_CUDA_TRY(cudaEventRecord(c.join_ev, c.side));
  // the well-conditioned modes on the main stream, concurrently
  if (N >= 1024) KFBI_TRY(launch_filter<64>(c, V, k0));
  else if (N >= 256) KFBI_TRY(launch_filter<32>(c, V, k0));
  else KFBI_TRY(launch_filter<16>(c, V, k0));
  KFBI_CUDA_TRY(cudaStreamWaitEvent(c.stream, c.join_ev, 0));      // join
  return KFBI_OK;
}

}  // namespace kfbi
