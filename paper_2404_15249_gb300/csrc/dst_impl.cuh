// Fast box solver of (Lap_h - kappa^2) v = b with v = 0 on the box boundary (Alg. 4),
// instantiated for one precision T by dst_f32.cu / dst_f64.cu.
//
// Work grid: N x N, node (i, j) at j*N + i for 0 <= i, j < N; row 0 and column 0 are
// boundary nodes and stay zero, the interior unknowns are 1 <= i, j <= N-1 and the last
// boundary row/column (index N) is implicit.  A grid line is then exactly the length-N
// array (0, x_1, ..., x_{N-1}) that a sine transform of type I acts on.
//
// Three passes, each reading and writing every unknown once:
//   pass 1  DST-I along x of every row
//   pass 2  DST-I along y of every column, multiplication by
//           (2/N)^2 / (lambda_k + lambda_l - kappa^2), DST-I along y again
//   pass 3  DST-I along x of every row
// with lambda_k = -(4/h^2) sin^2(pi k / 2N) the eigenvalues of the 1-D second difference.
//
// DST-I of a line through one complex FFT of length N: z_m = u_{2m} + i u_{2m+1} packs the
// odd extension u of the line (u_{2N-j} = -x_j); with Z = FFT_N(z), Z_k = a + ib and
// Z_{N-k} = c + id,  X_k = [-(b - d) + cos(pi k/N)(a - c) + sin(pi k/N)(b + d)] / 4.
// The FFT is a mixed-radix (16, 8, 4, 2, 3) Stockham transform in shared memory with the
// plan fixed at compile time for each supported N, so every shared-memory offset is a
// per-thread base plus a constant.  The first stage reads the raw line and forms the
// packed odd extension on the fly; the last stage keeps its outputs in registers and the
// post-processing pairs them with the partner value Z_{N-k} from shared memory.
#pragma once

#include "kfbi_internal.cuh"

namespace kfbi {
namespace dst {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cx<T> mul_negi(cx<T> a) { return {a.y, -a.x}; }   // -i a

// cos / sin at multiples of pi/8 and pi/3 used inside the small DFTs
#define KFBI_C8 0.92387953251128675613
#define KFBI_S8 0.38268343236508977173
#define KFBI_R2 0.70710678118654752440
#define KFBI_S3 0.86602540378443864676

template <typename T>
__device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
  cx<T> t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <typename T>
__device__ __forceinline__ void dft4(cx<T>& a, cx<T>& b, cx<T>& c, cx<T>& d) {
  cx<T> t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = csub(b, d);
  a = cadd(t0, t2);
  c = csub(t0, t2);
  b = cadd(t1, mul_negi(t3));
  d = csub(t1, mul_negi(t3));
}

template <typename T>
__device__ __forceinline__ void dft3(cx<T>* v) {
  const T s3 = T(KFBI_S3);
  cx<T> a = v[0], t = cadd(v[1], v[2]), s = csub(v[1], v[2]);
  cx<T> m = {a.x - T(0.5) * t.x, a.y - T(0.5) * t.y};
  v[0] = cadd(a, t);
  v[1] = {m.x + s3 * s.y, m.y - s3 * s.x};
  v[2] = {m.x - s3 * s.y, m.y + s3 * s.x};
}

template <typename T>
__device__ __forceinline__ void dft8(cx<T>* v) {
  cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  const T r = T(KFBI_R2);
  cx<T> w1 = {(o1.x + o1.y) * r, (o1.y - o1.x) * r};
  cx<T> w2 = mul_negi(o2);
  cx<T> w3 = {(-o3.x + o3.y) * r, (-o3.y - o3.x) * r};
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1); v[5] = csub(e1, w1);
  v[2] = cadd(e2, w2); v[6] = csub(e2, w2);
  v[3] = cadd(e3, w3); v[7] = csub(e3, w3);
}

template <typename T>
__device__ __forceinline__ void dft16(cx<T>* v) {
  // 16 = 4 x 4: inputs x[4 n1 + n2]; DFT over n1, twiddle W16^{n2 k1}, DFT over n2;
  // outputs y[k1 + 4 k2]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
  const cx<T> w1 = {T(KFBI_C8), T(-KFBI_S8)}, w2 = {T(KFBI_R2), T(-KFBI_R2)},
              w3 = {T(KFBI_S8), T(-KFBI_C8)}, w6 = {T(-KFBI_R2), T(-KFBI_R2)},
              w9 = {T(-KFBI_C8), T(KFBI_S8)};
  v[5] = cmul(v[5], w1);  v[9] = cmul(v[9], w2);   v[13] = cmul(v[13], w3);
  v[6] = cmul(v[6], w2);  v[10] = mul_negi(v[10]); v[14] = cmul(v[14], w6);
  v[7] = cmul(v[7], w3);  v[11] = cmul(v[11], w6); v[15] = cmul(v[15], w9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  cx<T> y[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = y[i];
}

template <typename T, int R>
__device__ __forceinline__ void dft(cx<T>* v) {
  if constexpr (R == 2) dft2(v[0], v[1]);
  else if constexpr (R == 3) dft3(v);
  else if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8(v);
  else dft16(v);
}

// ------------------------------------------------------------------ compile-time plan
struct CPlan {
  int ept, tpl, nst;
  int radix[8];
  int ns[8];      // product of the radices of the earlier stages
};

__host__ __device__ constexpr CPlan cplan(int N) {
  CPlan p{};
  if (N % 3 == 0) {
    p.ept = 24;
    int r = N / 3;
    while (r % 8 == 0 && r > 8) { p.radix[p.nst++] = 8; r /= 8; }
    if (r > 1) p.radix[p.nst++] = r;
    p.radix[p.nst++] = 3;
  } else {
    p.ept = 16;
    int r = N;
    while (r % 16 == 0) { p.radix[p.nst++] = 16; r /= 16; }
    if (r > 1) p.radix[p.nst++] = r;
  }
  p.tpl = N / p.ept;
  int ns = 1;
  for (int s = 0; s < p.nst; ++s) { p.ns[s] = ns; ns *= p.radix[s]; }
  return p;
}

// padded shared-memory index (one spare slot per 16 complex values)
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int line_len(int N) { return N + N / 16 + 2; }   // complex slots per line

// value m of the packed odd extension, read from the raw line (T[0..N], raw[N] = 0)
template <typename T, int N>
__device__ __forceinline__ cx<T> packed(const T* raw, int m, bool upper) {
  if (!upper) return *reinterpret_cast<const cx<T>*>(raw + 2 * m);
  const int mp = N - m;                       // 0 < mp <= N/2
  return {-raw[2 * mp], -raw[2 * mp - 1]};
}

// One in-place Stockham stage S of the plan for N.  Butterfly j reads z[j + r N/R],
// multiplies input r by W_N^{(j mod Ns) r N/(Ns R)}, writes output r to
// z[(j - j mod Ns) R + j mod Ns + r Ns].  The first stage reads the raw line instead.
// The last stage leaves its outputs in v (output r of butterfly q at v[q R + r]) and
// also stores them to z.
template <typename T, int N, int S>
__device__ __forceinline__ void stage(cx<T>* z, int t, const cx<T>* __restrict__ tw,
                                      cx<T>* v) {
  constexpr CPlan P = cplan(N);
  constexpr int R = P.radix[S], Ns = P.ns[S], NB = P.ept / R, STR = N / R;
  if constexpr (S == 0) {
    const T* raw = reinterpret_cast<const T*>(z);
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r)
        v[q * R + r] = packed<T, N>(raw, t + q * P.tpl + r * STR, 2 * r >= R);
  } else {
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = z[pad(t + q * P.tpl + r * STR)];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = t + q * P.tpl;
    if constexpr (Ns > 1) {
      const int jm = j & (Ns - 1);
      const int b2 = 2 * jm * (N / (Ns * R));
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], tw[b2 * r]);
    }
    dft<T, R>(&v[q * R]);
    const int out0 = (j & ~(Ns - 1)) * R + (j & (Ns - 1));
#pragma unroll
    for (int r = 0; r < R; ++r) z[pad(out0 + r * Ns)] = v[q * R + r];
  }
  __syncthreads();
}

template <typename T, int N, int S = 0>
__device__ __forceinline__ void fft(cx<T>* z, int t, const cx<T>* __restrict__ tw, cx<T>* v) {
  constexpr CPlan P = cplan(N);
  stage<T, N, S>(z, t, tw, v);
  if constexpr (S + 1 < P.nst) fft<T, N, S + 1>(z, t, tw, v);
}

// DST-I outputs held by this thread after fft(): output e = q R + r is X_k with
// k = t + q tpl + r N/R (R the last radix), formed from v[e] = Z_k and the partner value
// Z_{N-k} in shared memory, and handed to f(e, k, X_k).
template <typename T, int N, typename F>
__device__ __forceinline__ void dst_outputs(const cx<T>* z, int t, const cx<T>* __restrict__ tw,
                                            cx<T>* v, F&& f) {
  constexpr CPlan P = cplan(N);
  constexpr int R = P.radix[P.nst - 1], NB = P.ept / R, STR = N / R;
#pragma unroll
  for (int q = 0; q < NB; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = t + q * P.tpl + r * STR;
      const cx<T> a = v[q * R + r];
      const cx<T> b = z[pad(N - k)];            // k = 0 reads a discarded slot
      const cx<T> w = tw[k];
      const T val = T(0.25) * (-(a.y - b.y) + w.x * (a.x - b.x) - w.y * (a.y + b.y));
      f(q * R + r, k, (k == 0) ? T(0) : val);
    }
}

template <typename T, int N>
__device__ __forceinline__ int out_index(int t, int e) {
  constexpr CPlan P = cplan(N);
  constexpr int R = P.radix[P.nst - 1], STR = N / R;
  return t + (e / R) * P.tpl + (e % R) * STR;
}

// ---------------------------------------------------------------------------- pass 1/3
// DST-I along every row: out[row] = scale * DST(in[row]); in may equal out.  LPC lines per
// CTA, persistent grid-stride loop; the next row is loaded into registers while the
// current one is transformed.
template <typename T, int N>
__global__ void __launch_bounds__(512) rows_kernel(const T* in, T* out,
                                                   const cx<T>* __restrict__ tw, T scale) {
  constexpr CPlan P = cplan(N);
  constexpr int H = P.ept / 2;                  // pairs of the raw line per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lpc = blockDim.x / P.tpl;
  const int line = threadIdx.x / P.tpl, t = threadIdx.x - line * P.tpl;
  cx<T>* z = reinterpret_cast<cx<T>*>(smem_raw) + line * line_len(N);
  const int step = gridDim.x * lpc;
  int row = blockIdx.x * lpc + line;
  cx<T> pre[H];
  if (row < N) {
    const cx<T>* src = reinterpret_cast<const cx<T>*>(in + (size_t)row * N);
#pragma unroll
    for (int u = 0; u < H; ++u) pre[u] = src[t + u * P.tpl];
  }
  cx<T> v[P.ept];
  for (int row0 = blockIdx.x * lpc; row0 < N; row0 += step, row += step) {
    const bool active = row < N;
#pragma unroll
    for (int u = 0; u < H; ++u) z[t + u * P.tpl] = active ? pre[u] : cx<T>{T(0), T(0)};
    if (t == 0) reinterpret_cast<T*>(z)[N] = T(0);
    const int nrow = row + step;
    if (nrow < N) {
      const cx<T>* src = reinterpret_cast<const cx<T>*>(in + (size_t)nrow * N);
#pragma unroll
      for (int u = 0; u < H; ++u) pre[u] = src[t + u * P.tpl];
    }
    __syncthreads();
    fft<T, N>(z, t, tw, v);
    T* dst = out + (size_t)row * N;
    dst_outputs<T, N>(z, t, tw, v, [&](int, int k, T x) {
      if (active) dst[k] = x * scale;
    });
    __syncthreads();
  }
}

template <int B> struct RawVec;
template <> struct RawVec<4> { typedef unsigned int type; };
template <> struct RawVec<8> { typedef uint2 type; };
template <> struct RawVec<16> { typedef uint4 type; };

__device__ __forceinline__ float recip(float d) { return __frcp_rn(d); }
__device__ __forceinline__ double recip(double d) {
  // Newton-Raphson from the FP32 reciprocal: two steps reach FP64 accuracy
  double r = (double)__frcp_rn((float)d);
  r = r * (2.0 - d * r);
  r = r * (2.0 - d * r);
  return r;
}

// column tile width: largest power of two <= 32 dividing N with L * tpl threads within
// the bound and L line buffers plus the staging tile within 220 KB of shared memory
template <typename T, int N, int MAXT>
__host__ __device__ constexpr int cols_L() {
  constexpr CPlan P = cplan(N);
  int L = 1;
  while (L < 32 && N % (2 * L) == 0 && 2 * L * P.tpl <= MAXT &&
         (size_t)(2 * L) * (line_len(N) * 2 * sizeof(T) + N * sizeof(T)) <= 220 * 1024)
    L *= 2;
  return L;
}


// ---------------------------------------------------------------------------- pass 2
// L consecutive columns (x-modes k) per CTA: DST-I along y, multiply by
// scale / (lam[k] + lam[l] - kappa^2), DST-I along y again.  The next column tile is
// copied into a shared-memory staging area with cp.async while the current one is
// transformed.
template <typename T, int N, int MAXT>
__global__ void __launch_bounds__(MAXT) cols_kernel(T* V, const cx<T>* __restrict__ tw,
                                                               const T* __restrict__ lam,
                                                               T kappa2, T scale) {
  constexpr CPlan P = cplan(N);
  constexpr int L = cols_L<T, N, MAXT>();
  constexpr int CH = (L * (int)sizeof(T) >= 16) ? L * (int)sizeof(T) / 16 : 1;
  constexpr int W = L / CH;
  constexpr int VB = W * (int)sizeof(T);
  constexpr int NCH = N * CH;                   // chunks per tile
  constexpr int LL = line_len(N);
  typedef typename RawVec<VB>::type Raw;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* lines = reinterpret_cast<cx<T>*>(smem_raw);
  Raw* stage_buf = reinterpret_cast<Raw*>(lines + L * LL);     // N rows x L values
  const int line = threadIdx.x / P.tpl, t = threadIdx.x - line * P.tpl;
  cx<T>* z = lines + line * LL;
  T* raw = reinterpret_cast<T*>(z);
  const int nthr = blockDim.x;

  auto prefetch = [&](int col0) {
    for (int g = threadIdx.x; g < NCH; g += nthr) {
      const int r = g / CH, cc = g - r * CH;
      const T* src = V + (size_t)r * N + col0 + cc * W;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(stage_buf + g);
      if constexpr (VB == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
      else if constexpr (VB == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src));
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src));
    }
    asm volatile("cp.async.commit_group;\n" ::);
  };

  int c0 = blockIdx.x * L;
  if (c0 < N) prefetch(c0);
  cx<T> v[P.ept];
  for (; c0 < N; c0 += gridDim.x * L) {
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();
    // staging tile -> raw lines
    for (int g = threadIdx.x; g < NCH; g += nthr) {
      const int r = g / CH, cc = g - r * CH;
      const Raw pk = stage_buf[g];
      const T* vals = reinterpret_cast<const T*>(&pk);
#pragma unroll
      for (int w = 0; w < W; ++w) reinterpret_cast<T*>(lines + (cc * W + w) * LL)[r] = vals[w];
    }
    if (t == 0) raw[N] = T(0);
    __syncthreads();
    if (c0 + gridDim.x * L < N) prefetch(c0 + gridDim.x * L);
    fft<T, N>(z, t, tw, v);
    const int k = c0 + line;
    const T lk = lam[k] - kappa2;
    // each output only needs its own v[e] and a partner from shared memory, so the
    // result can overwrite v[e].x
    dst_outputs<T, N>(z, t, tw, v, [&](int e, int l, T x) {
      v[e].x = (k == 0 || l == 0) ? T(0) : x * scale * recip(lk + lam[l]);
    });
    __syncthreads();
#pragma unroll
    for (int e = 0; e < P.ept; ++e) raw[out_index<T, N>(t, e)] = v[e].x;
    if (t == 0) raw[N] = T(0);
    __syncthreads();
    fft<T, N>(z, t, tw, v);
    dst_outputs<T, N>(z, t, tw, v, [&](int e, int, T x) { v[e].x = x; });
    __syncthreads();
#pragma unroll
    for (int e = 0; e < P.ept; ++e) raw[out_index<T, N>(t, e)] = v[e].x;
    __syncthreads();
    for (int g = threadIdx.x; g < NCH; g += nthr) {
      const int r = g / CH, cc = g - r * CH;
      Raw pk;
      T* vals = reinterpret_cast<T*>(&pk);
#pragma unroll
      for (int w = 0; w < W; ++w) vals[w] = reinterpret_cast<const T*>(lines + (cc * W + w) * LL)[r];
      *reinterpret_cast<Raw*>(V + (size_t)r * N + c0 + cc * W) = pk;
    }
  }
  asm volatile("cp.async.wait_group 0;\n" ::);
}

// ---------------------------------------------------------------------------- launch
inline int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <typename T, int N>
kfbi_status launch_rows(Ctx& c, const T* in, T* out, const cx<T>* tw, T scale) {
  constexpr CPlan P = cplan(N);
  const int lpc = P.tpl >= 256 ? 1 : 256 / P.tpl;
  const int threads = lpc * P.tpl;
  const size_t smem = (size_t)lpc * line_len(N) * sizeof(cx<T>);
  static bool attr = false;
  if (!attr) {
    KFBI_CUDA_TRY(cudaFuncSetAttribute(rows_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024));
    attr = true;
  }
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_kernel<T, N>, threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = (N + lpc - 1) / lpc;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_ROWS32 : ST_ROWS64);
  rows_kernel<T, N><<<blocks, threads, smem, c.stream>>>(in, out, tw, scale);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T, int N, int MAXT>
kfbi_status launch_cols(Ctx& c, T* V, const cx<T>* tw, const T* lam) {
  constexpr CPlan P = cplan(N);
  constexpr int L = cols_L<T, N, MAXT>();
  const int threads = L * P.tpl;
  const size_t smem = (size_t)L * line_len(N) * sizeof(cx<T>) + (size_t)N * L * sizeof(T);
  static bool attr = false;
  if (!attr) {
    KFBI_CUDA_TRY(cudaFuncSetAttribute(cols_kernel<T, N, MAXT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cols_kernel<T, N, MAXT>,
                                                              threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = N / L;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const T scale = T((2.0 / N) * (2.0 / N));
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_COLS32 : ST_COLS64);
  cols_kernel<T, N, MAXT><<<blocks, threads, smem, c.stream>>>(V, tw, lam, T(c.kappa2), scale);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

// column-pass variant chosen by the autotuner (0: 512-thread CTAs, 1: 1024-thread CTAs)
template <typename T, int N>
kfbi_status launch_cols_v(Ctx& c, T* V, const cx<T>* tw, const T* lam, int variant) {
  if (variant == 1 && cplan(N).tpl * 2 <= 1024) return launch_cols<T, N, 1024>(c, V, tw, lam);
  return launch_cols<T, N, 512>(c, V, tw, lam);
}

// Time both column-pass variants on the context's work grid (its contents are scratch
// at setup) and keep the faster one for this precision.
template <typename T, int N>
kfbi_status autotune_cols(Ctx& c, T* V, const cx<T>* tw, const T* lam, int* choice) {
  cudaEvent_t e[3];
  for (auto& x : e) KFBI_CUDA_TRY(cudaEventCreate(&x));
  float ms[2] = {0.f, 0.f};
  for (int v = 0; v < 2; ++v) {
    KFBI_TRY((launch_cols_v<T, N>(c, V, tw, lam, v)));           // warm-up
    KFBI_CUDA_TRY(cudaEventRecord(e[0], c.stream));
    for (int rep = 0; rep < 3; ++rep) KFBI_TRY((launch_cols_v<T, N>(c, V, tw, lam, v)));
    KFBI_CUDA_TRY(cudaEventRecord(e[1], c.stream));
    KFBI_CUDA_TRY(cudaEventSynchronize(e[1]));
    KFBI_CUDA_TRY(cudaEventElapsedTime(&ms[v], e[0], e[1]));
  }
  for (auto& x : e) cudaEventDestroy(x);
  *choice = ms[1] < ms[0] ? 1 : 0;
  return KFBI_OK;
}

template <typename T, int N>
kfbi_status box_solve_n(Ctx& c, const T* rhs, T* work, const cx<T>* tw, const T* lam) {
  const int variant = c.cols_variant[sizeof(T) == 8] > 0 ? 1 : 0;
  KFBI_TRY((launch_rows<T, N>(c, rhs, work, tw, T(1))));
  KFBI_TRY((launch_cols_v<T, N>(c, work, tw, lam, variant)));
  KFBI_TRY((launch_rows<T, N>(c, work, work, tw, T(1))));
  return KFBI_OK;
}

template <typename T>
kfbi_status autotune_dispatch(Ctx& c, T* scratch, const cx<T>* tw, const T* lam) {
  int* choice = &c.cols_variant[sizeof(T) == 8];
  switch (c.N) {
#define KFBI_CASE(n) \
  case n: return autotune_cols<T, n>(c, scratch, tw, lam, choice);
    KFBI_CASE(32) KFBI_CASE(48) KFBI_CASE(64) KFBI_CASE(96) KFBI_CASE(128) KFBI_CASE(192)
    KFBI_CASE(256) KFBI_CASE(384) KFBI_CASE(512) KFBI_CASE(768) KFBI_CASE(1024)
    KFBI_CASE(1536) KFBI_CASE(2048) KFBI_CASE(3072) KFBI_CASE(4096) KFBI_CASE(6144)
    KFBI_CASE(8192)
#undef KFBI_CASE
  }
  return KFBI_ERR_UNSUPPORTED;
}

template <typename T>
kfbi_status box_solve_dispatch(Ctx& c, const T* rhs, T* work, const cx<T>* tw, const T* lam) {
  switch (c.N) {
#define KFBI_CASE(n) \
  case n: return box_solve_n<T, n>(c, rhs, work, tw, lam);
    KFBI_CASE(32) KFBI_CASE(48) KFBI_CASE(64) KFBI_CASE(96) KFBI_CASE(128) KFBI_CASE(192)
    KFBI_CASE(256) KFBI_CASE(384) KFBI_CASE(512) KFBI_CASE(768) KFBI_CASE(1024)
    KFBI_CASE(1536) KFBI_CASE(2048) KFBI_CASE(3072) KFBI_CASE(4096) KFBI_CASE(6144)
    KFBI_CASE(8192)
#undef KFBI_CASE
  }
  set_error("box solve: no compiled plan for N = %d", c.N);
  return KFBI_ERR_UNSUPPORTED;
}

}  // namespace dst
}  // namespace kfbi
