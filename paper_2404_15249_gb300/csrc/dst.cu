// Fast box solver of (Lap_h - kappa^2) v = b with v = 0 on the box boundary (Alg. 4).
//
// The N x N work grid holds node (i, j) at j*N + i for 0 <= i, j < N; row 0 and column 0
// are boundary nodes and stay zero, the interior unknowns are 1 <= i, j <= N-1, and the
// last boundary row/column (index N) is implicit.  With that layout a grid line is exactly
// the length-N array (0, x_1, ..., x_{N-1}) that a sine transform of type I needs.
//
// Three passes, each reading and writing every unknown once:
//   pass 1  DST-I along x of every row                 (rows contiguous in memory)
//   pass 2  DST-I along y of every column, division by the eigenvalue
//           lambda_k + lambda_l - kappa^2 scaled by (2/N)^2, inverse DST-I along y
//   pass 3  DST-I along x of every row
// Both kernels stage whole lines in shared memory.  A DST-I of a length-N line is one
// complex FFT of length N: z_m = u_{2m} + i u_{2m+1} packs the odd extension u of the
// line (u_{2N-j} = -x_j), and X_k = [-(b - d) + cos(pi k/N)(a - c) + sin(pi k/N)(b + d)]/4
// with Z_k = a + ib, Z_{N-k} = c + id recovers the transform (Z = FFT_N(z)).
// The FFT is a mixed-radix (16, 8, 4, 2, 3) Stockham transform done in place in shared
// memory: every stage reads all of a thread's values into registers, synchronises, then
// writes the butterfly outputs.
#include "kfbi_internal.cuh"

namespace kfbi {

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

// Constants of the small DFTs (values of cos / sin at multiples of pi/8 and pi/3).
#define KFBI_C8 0.92387953251128675613   // cos(pi/8)
#define KFBI_S8 0.38268343236508977173   // sin(pi/8)
#define KFBI_R2 0.70710678118654752440   // sqrt(1/2)
#define KFBI_S3 0.86602540378443864676   // sin(pi/3)

template <typename T>
__device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
  cx<T> t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// forward DFT of length 4 on (a, b, c, d) in place
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
  // even / odd halves, then combine with W8^k = e^{-i pi k/4}
  cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3);
  dft4(o0, o1, o2, o3);
  const T r = T(KFBI_R2);
  cx<T> w1 = {(o1.x + o1.y) * r, (o1.y - o1.x) * r};      // (r, -r) * o1
  cx<T> w2 = mul_negi(o2);                                // -i * o2
  cx<T> w3 = {(-o3.x + o3.y) * r, (-o3.y - o3.x) * r};    // (-r, -r) * o3
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, w1); v[5] = csub(e1, w1);
  v[2] = cadd(e2, w2); v[6] = csub(e2, w2);
  v[3] = cadd(e3, w3); v[7] = csub(e3, w3);
}

template <typename T>
__device__ __forceinline__ void dft16(cx<T>* v) {
  // 16 = 4 x 4: inputs x[4 n1 + n2]; DFT over n1, twiddle W16^{n2 k1}, DFT over n2;
  // output y[k1 + 4 k2].
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
  const cx<T> w1 = {T(KFBI_C8), T(-KFBI_S8)}, w2 = {T(KFBI_R2), T(-KFBI_R2)},
              w3 = {T(KFBI_S8), T(-KFBI_C8)}, w6 = {T(-KFBI_R2), T(-KFBI_R2)},
              w9 = {T(-KFBI_C8), T(KFBI_S8)};
  // A[n2][k1] sits in v[n2 + 4 k1]
  v[1 + 4] = cmul(v[1 + 4], w1);  v[1 + 8] = cmul(v[1 + 8], w2);  v[1 + 12] = cmul(v[1 + 12], w3);
  v[2 + 4] = cmul(v[2 + 4], w2);  v[2 + 8] = mul_negi(v[2 + 8]);  v[2 + 12] = cmul(v[2 + 12], w6);
  v[3 + 4] = cmul(v[3 + 4], w3);  v[3 + 8] = cmul(v[3 + 8], w6);  v[3 + 12] = cmul(v[3 + 12], w9);
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

// One in-place Stockham stage of radix R on the line z (padded indices).  Butterfly j
// reads z[j + r N/R], multiplies input r by W_N^{(j mod Ns) r N/(Ns R)}, and writes
// output r to z[(j / Ns) Ns R + j mod Ns + r Ns].  tw[s] = e^{-i pi s / N}, s < 2N.
template <typename T, int EPT, int R>
__device__ __forceinline__ void fft_stage(cx<T>* z, int N, int Ns, int t, int tpl,
                                          const cx<T>* __restrict__ tw) {
  constexpr int NB = EPT / R;
  cx<T> v[EPT];
  const int stride = N / R;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = t + q * tpl;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = z[padi(j + r * stride)];
  }
  __syncthreads();
  const int tstep = N / (Ns * R);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = t + q * tpl;
    const int jm = j % Ns;
    if (jm != 0) {
      const int base = jm * tstep;
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], tw[2 * base * r]);
    }
    dft<T, R>(&v[q * R]);
    const int out0 = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) z[padi(out0 + r * Ns)] = v[q * R + r];
  }
  __syncthreads();
}

template <typename T, int EPT>
__device__ void fft_line(cx<T>* z, const FftPlan& p, int t, const cx<T>* __restrict__ tw) {
  int Ns = 1;
  for (int s = 0; s < p.nst; ++s) {
    const int R = p.radix[s];
    if constexpr (EPT % 16 == 0) {
      if (R == 16) fft_stage<T, EPT, 16>(z, p.N, Ns, t, p.tpl, tw);
    }
    if (R == 8) fft_stage<T, EPT, 8>(z, p.N, Ns, t, p.tpl, tw);
    else if (R == 4) fft_stage<T, EPT, 4>(z, p.N, Ns, t, p.tpl, tw);
    else if (R == 2) fft_stage<T, EPT, 2>(z, p.N, Ns, t, p.tpl, tw);
    if constexpr (EPT % 3 == 0) {
      if (R == 3) fft_stage<T, EPT, 3>(z, p.N, Ns, t, p.tpl, tw);
    }
    Ns *= R;
  }
}

// Fill the upper half of the packed sequence from the lower half (odd extension):
// z_m = (-x_{2m'}, -x_{2m'-1}) with m' = N - m, m in [N/2, N).
template <typename T>
__device__ __forceinline__ void mirror_fill(cx<T>* z, int N, int t, int tpl) {
  const int half = N >> 1;
#pragma unroll 4
  for (int m = half + t; m < N; m += tpl) {
    const int mp = N - m;
    const T re = (mp < half) ? z[padi(mp)].x : T(0);
    const T im = z[padi(mp - 1)].y;
    z[padi(m)] = {-re, -im};
  }
}

// Output pair q of the DST-I: (X_{2q}, X_{2q+1}), X_0 = 0.
template <typename T>
__device__ __forceinline__ cx<T> dst_pair(const cx<T>* z, int N, int q,
                                          const cx<T>* __restrict__ tw) {
  T o[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int k = 2 * q + e;
    if (k == 0) {
      o[e] = T(0);
    } else {
      const cx<T> a = z[padi(k)], b = z[padi(N - k)];
      const cx<T> w = tw[k];                        // (cos, -sin)(pi k / N)
      o[e] = T(0.25) * (-(a.y - b.y) + w.x * (a.x - b.x) - w.y * (a.y + b.y));
    }
  }
  return {o[0], o[1]};
}

// ---------------------------------------------------------------------------- pass 1/3
// DST-I along every row of the N x N grid: out[row] = scale * DST(in[row]).  in may equal
// out.  LPC lines per CTA (tpl threads each); persistent grid-stride loop over rows.  The
// next row is loaded into registers while the current one is transformed, so global
// latency overlaps the FFT.
template <typename T, int EPT>
__global__ void __launch_bounds__(512) dst_rows_kernel(const T* in, T* out, FftPlan p,
                                                       const cx<T>* __restrict__ tw, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  constexpr int H = EPT / 2;                 // packed pairs per thread
  const int N = p.N, tpl = p.tpl;
  const int lpc = blockDim.x / tpl;
  const int line = threadIdx.x / tpl, t = threadIdx.x - line * tpl;
  cx<T>* z = sm + line * padded_len(N);
  const int step = gridDim.x * lpc;
  int row = blockIdx.x * lpc + line;
  cx<T> pre[H];
  if (row < N) {
    const cx<T>* src = reinterpret_cast<const cx<T>*>(in + (size_t)row * N);
#pragma unroll
    for (int u = 0; u < H; ++u) pre[u] = src[t + u * tpl];
  }
  for (int row0 = blockIdx.x * lpc; row0 < N; row0 += step, row += step) {
    const bool active = row < N;
#pragma unroll
    for (int u = 0; u < H; ++u) z[padi(t + u * tpl)] = active ? pre[u] : cx<T>{T(0), T(0)};
    const int nrow = row + step;
    if (nrow < N) {
      const cx<T>* src = reinterpret_cast<const cx<T>*>(in + (size_t)nrow * N);
#pragma unroll
      for (int u = 0; u < H; ++u) pre[u] = src[t + u * tpl];
    }
    __syncthreads();
    mirror_fill(z, N, t, tpl);
    __syncthreads();
    fft_line<T, EPT>(z, p, t, tw);
    cx<T> o[H];
#pragma unroll
    for (int u = 0; u < H; ++u) o[u] = dst_pair(z, N, t + u * tpl, tw);
    if (active) {
      cx<T>* dst = reinterpret_cast<cx<T>*>(out + (size_t)row * N);
#pragma unroll
      for (int u = 0; u < H; ++u) dst[t + u * tpl] = {o[u].x * scale, o[u].y * scale};
    }
    __syncthreads();
  }
}

// raw vector of B bytes for tile loads / stores
template <int B> struct RawVec;
template <> struct RawVec<4> { typedef unsigned int type; };
template <> struct RawVec<8> { typedef uint2 type; };
template <> struct RawVec<16> { typedef uint4 type; };

// reciprocal: FP32 correctly rounded; FP64 by two Newton-Raphson steps from the FP32 one
__device__ __forceinline__ float recip(float d) { return __frcp_rn(d); }
__device__ __forceinline__ double recip(double d) {
  double r = (double)__frcp_rn((float)d);
  r = r * (2.0 - d * r);
  r = r * (2.0 - d * r);
  return r;
}

// ---------------------------------------------------------------------------- pass 2
// For L consecutive columns (x-modes k) per CTA: DST-I along y, multiply by
// scale / (lam[k] + lam[l] - kappa^2), DST-I along y again; column 0 and row 0 stay 0.
// The tile rows are moved as 16-byte (or narrower) vectors; the next tile is loaded
// into registers while the current one is transformed.
template <typename T, int EPT, int L, int MAXT>
__global__ void __launch_bounds__(MAXT) dst_cols_solve_kernel(T* V, FftPlan p,
                                                              const cx<T>* __restrict__ tw,
                                                              const T* __restrict__ lam,
                                                              T kappa2, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  constexpr int CH = (L * (int)sizeof(T) >= 16) ? L * (int)sizeof(T) / 16 : 1;  // chunks/row
  constexpr int W = L / CH;                                                        // T per chunk
  constexpr int VB = W * (int)sizeof(T);
  constexpr int NC = EPT * CH / L;                                                 // chunks/thread
  typedef typename RawVec<VB>::type Raw;
  const int N = p.N, tpl = p.tpl, PL = padded_len(N);
  const int line = threadIdx.x / tpl, t = threadIdx.x - line * tpl;
  cx<T>* z = sm + line * PL;
  const int nthr = blockDim.x;
  Raw pre[NC];
  int c0 = blockIdx.x * L;
  auto load_tile = [&](int col0) {
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int g = threadIdx.x + i * nthr;
      const int r = g / CH, cc = g - r * CH;
      pre[i] = *reinterpret_cast<const Raw*>(V + (size_t)r * N + col0 + cc * W);
    }
  };
  if (c0 < N) load_tile(c0);
  for (; c0 < N; c0 += gridDim.x * L) {
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int g = threadIdx.x + i * nthr;
      const int r = g / CH, cc = g - r * CH;
      const T* vals = reinterpret_cast<const T*>(&pre[i]);
      const int pos = 2 * padi(r >> 1) + (r & 1);
#pragma unroll
      for (int w = 0; w < W; ++w) reinterpret_cast<T*>(sm + (cc * W + w) * PL)[pos] = vals[w];
    }
    if (c0 + gridDim.x * L < N) load_tile(c0 + gridDim.x * L);
    __syncthreads();
    mirror_fill(z, N, t, tpl);
    __syncthreads();
    fft_line<T, EPT>(z, p, t, tw);
    // spectral division, repacked as the next transform's input pairs
    const int k = c0 + line;
    const T lk = lam[k] - kappa2;
    cx<T> keep[EPT / 2];
#pragma unroll
    for (int u = 0; u < EPT / 2; ++u) {
      const int q = t + u * tpl;
      cx<T> o = dst_pair(z, N, q, tw);
      const int l0 = 2 * q, l1 = 2 * q + 1;
      const T d0 = (k == 0 || l0 == 0) ? T(0) : scale * recip(lk + lam[l0]);
      const T d1 = (k == 0) ? T(0) : scale * recip(lk + lam[l1]);
      keep[u] = {o.x * d0, o.y * d1};
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < EPT / 2; ++u) z[padi(t + u * tpl)] = keep[u];
    __syncthreads();
    mirror_fill(z, N, t, tpl);
    __syncthreads();
    fft_line<T, EPT>(z, p, t, tw);
#pragma unroll
    for (int u = 0; u < EPT / 2; ++u) keep[u] = dst_pair(z, N, t + u * tpl, tw);
    __syncthreads();
    // results as reals, line c value r at z_c[2 padi(r/2) + r%2]
#pragma unroll
    for (int u = 0; u < EPT / 2; ++u) z[padi(t + u * tpl)] = keep[u];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NC; ++i) {
      const int g = threadIdx.x + i * nthr;
      const int r = g / CH, cc = g - r * CH;
      Raw out;
      T* vals = reinterpret_cast<T*>(&out);
      const int pos = 2 * padi(r >> 1) + (r & 1);
#pragma unroll
      for (int w = 0; w < W; ++w) vals[w] = reinterpret_cast<const T*>(sm + (cc * W + w) * PL)[pos];
      *reinterpret_cast<Raw*>(V + (size_t)r * N + c0 + cc * W) = out;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------- plan
bool make_fft_plan(int N, FftPlan* p) {
  if (N < 32 || N > 16384) return false;
  int rest = N, n3 = 0;
  while (rest % 3 == 0) { rest /= 3; ++n3; }
  if (n3 > 1 || (rest & (rest - 1)) != 0) return false;
  FftPlan q{};
  q.N = N;
  if (n3 == 1) {
    q.ept = 24;
    int r = N / 3;
    while (r % 8 == 0 && r > 8) { q.radix[q.nst++] = 8; r /= 8; }
    if (r > 1) q.radix[q.nst++] = r;      // 8, 4 or 2
    q.radix[q.nst++] = 3;
  } else {
    q.ept = 16;
    int r = N;
    while (r % 16 == 0) { q.radix[q.nst++] = 16; r /= 16; }
    if (r > 1) q.radix[q.nst++] = r;      // 8, 4 or 2
  }
  q.tpl = N / q.ept;
  *p = q;
  return true;
}

// ---------------------------------------------------------------------------- tables
__global__ void box_tables_kernel(int N, double h, double2* tw64, float2* tw32, double* lam64,
                                  float* lam32) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < 2 * N) {
    double sn, cs;
    sincospi((double)s / (double)N, &sn, &cs);
    tw64[s] = make_double2(cs, -sn);
    tw32[s] = make_float2((float)cs, (float)-sn);
  }
  if (s < N) {
    const double sk = sinpi((double)s / (2.0 * N));
    const double l = -(4.0 / (h * h)) * sk * sk;
    lam64[s] = l;
    lam32[s] = (float)l;
  }
}

kfbi_status init_box_tables(Ctx& c) {
  const int N = c.N;
  KFBI_TRY(alloc_bytes(c, (void**)&c.t64.tw, sizeof(double2) * 2 * N));
  KFBI_TRY(alloc_bytes(c, (void**)&c.t32.tw, sizeof(float2) * 2 * N));
  KFBI_TRY(alloc_bytes(c, (void**)&c.t64.lam, sizeof(double) * N));
  KFBI_TRY(alloc_bytes(c, (void**)&c.t32.lam, sizeof(float) * N));
  prof_count(c, ST_SETUP);
  box_tables_kernel<<<(2 * N + 255) / 256, 256, 0, c.stream>>>(N, c.h, c.t64.tw, c.t32.tw,
                                                                c.t64.lam, c.t32.lam);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

// ---------------------------------------------------------------------------- launch
static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <typename T, int EPT>
static kfbi_status launch_rows(Ctx& c, const T* in, T* out, const cx<T>* tw, T scale) {
  const FftPlan& p = c.plan;
  const int lpc = p.tpl >= 256 ? 1 : 256 / p.tpl;   // tpl <= 512 for N <= 8192
  const int threads = lpc * p.tpl;
  const size_t smem = (size_t)lpc * padded_len(p.N) * sizeof(cx<T>);
  static bool attr_done[2] = {false, false};
  if (!attr_done[sizeof(T) == 8]) {
    KFBI_CUDA_TRY(cudaFuncSetAttribute(dst_rows_kernel<T, EPT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr_done[sizeof(T) == 8] = true;
  }
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dst_rows_kernel<T, EPT>,
                                                              threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = (p.N + lpc - 1) / lpc;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_ROWS32 : ST_ROWS64);
  dst_rows_kernel<T, EPT><<<blocks, threads, smem, c.stream>>>(in, out, p, tw, scale);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T, int EPT, int L>
static kfbi_status launch_cols_L(Ctx& c, T* V, const cx<T>* tw, const T* lam) {
  constexpr int MAXT = (sizeof(T) == 4 && EPT == 16) ? 1024 : 512;
  const FftPlan& p = c.plan;
  const size_t line_bytes = (size_t)padded_len(p.N) * sizeof(cx<T>);
  const int threads = L * p.tpl;
  const size_t smem = (size_t)L * line_bytes;
  static bool attr_done = false;
  if (!attr_done) {
    KFBI_CUDA_TRY(cudaFuncSetAttribute(dst_cols_solve_kernel<T, EPT, L, MAXT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr_done = true;
  }
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, dst_cols_solve_kernel<T, EPT, L, MAXT>, threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = p.N / L;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const T scale = T((2.0 / p.N) * (2.0 / p.N));
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_COLS32 : ST_COLS64);
  dst_cols_solve_kernel<T, EPT, L, MAXT><<<blocks, threads, smem, c.stream>>>(V, p, tw, lam,
                                                                              T(c.kappa2), scale);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

// tile width: largest power of two L <= 32 dividing N with L * tpl threads within the
// kernel's bound and L lines within 160 KB of shared memory
template <typename T, int EPT>
static int cols_tile(const FftPlan& p) {
  constexpr int MAXT = (sizeof(T) == 4 && EPT == 16) ? 1024 : 512;
  const size_t line_bytes = (size_t)padded_len(p.N) * sizeof(cx<T>);
  int L = 1;
  while (L < 32 && p.N % (2 * L) == 0 && 2 * L * p.tpl <= MAXT &&
         (size_t)(2 * L) * line_bytes <= 160 * 1024)
    L *= 2;
  return L;
}

template <typename T, int EPT>
static kfbi_status launch_cols(Ctx& c, T* V, const cx<T>* tw, const T* lam) {
  switch (cols_tile<T, EPT>(c.plan)) {
    case 1: return launch_cols_L<T, EPT, 1>(c, V, tw, lam);
    case 2: return launch_cols_L<T, EPT, 2>(c, V, tw, lam);
    case 4: return launch_cols_L<T, EPT, 4>(c, V, tw, lam);
    case 8: return launch_cols_L<T, EPT, 8>(c, V, tw, lam);
    case 16: return launch_cols_L<T, EPT, 16>(c, V, tw, lam);
    default: return launch_cols_L<T, EPT, 32>(c, V, tw, lam);
  }
}

template <typename T, int EPT>
static kfbi_status box_solve_t(Ctx& c, const T* rhs, T* work, const cx<T>* tw, const T* lam) {
  KFBI_TRY((launch_rows<T, EPT>(c, rhs, work, tw, T(1))));
  KFBI_TRY((launch_cols<T, EPT>(c, work, tw, lam)));
  KFBI_TRY((launch_rows<T, EPT>(c, work, work, tw, T(1))));
  return KFBI_OK;
}

kfbi_status box_solve_f32(Ctx& c, const float* rhs, float* work) {
  const cx<float>* tw = reinterpret_cast<const cx<float>*>(c.t32.tw);
  if (c.plan.ept == 16) return box_solve_t<float, 16>(c, rhs, work, tw, c.t32.lam);
  return box_solve_t<float, 24>(c, rhs, work, tw, c.t32.lam);
}

kfbi_status box_solve_f64(Ctx& c, const double* rhs, double* work) {
  const cx<double>* tw = reinterpret_cast<const cx<double>*>(c.t64.tw);
  if (c.plan.ept == 16) return box_solve_t<double, 16>(c, rhs, work, tw, c.t64.lam);
  return box_solve_t<double, 24>(c, rhs, work, tw, c.t64.lam);
}

}  // namespace kfbi
