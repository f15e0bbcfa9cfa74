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
// In FP32 (2-D) pass 2 keeps the transform pair only for the low x-modes; the others are
// solved along y by tridiagonal elimination (dst_tri.cu), the same system without the
// transforms.
//
// DST-I of a line through one complex FFT of length N: z_m = u_{2m} + i u_{2m+1} packs the
// odd extension u of the line (u_{2N-j} = -x_j); with Z = FFT_N(z), Z_k = a + ib and
// Z_{N-k} = c + id,  X_k = [-(b - d) + cos(pi k/N)(a - c) + sin(pi k/N)(b + d)] / 4.
// The FFT is a mixed-radix (16, 8, 4, 2, 3) Stockham transform with the plan fixed at
// compile time for each supported N (every shared-memory offset is a per-thread base plus
// a constant).  Stage 0 reads the raw line (global memory for rows, shared memory for
// columns) and forms the packed odd extension on the fly; later stages ping-pong between
// two padded shared-memory buffers with one barrier per stage; twiddles come from
// per-stage tables laid out [r][j mod Ns] so a warp's loads are contiguous; the last
// stage keeps its outputs in registers and the post-processing pairs them with the
// partner value Z_{N-k} from shared memory.
#pragma once

#include <atomic>
#include <type_traits>

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
  int twoff[8];   // offset of the stage's twiddle table (stages >= 1)
  int twtotal;    // total twiddle-table entries
};

// EPT values per thread per stage: 16 or 8 for N = 2^a (radices 16/8/4/2), 24 or 12 for
// N = 3 * 2^a (radices 8/4/2 then 3).  Every radix divides EPT.
__host__ __device__ constexpr int default_ept(int N) { return N % 3 == 0 ? 24 : 16; }

__host__ __device__ constexpr CPlan cplan(int N, int EPT) {
  CPlan p{};
  p.ept = EPT;
  const int big = (EPT == 16 || EPT == 24) ? (EPT == 16 ? 16 : 8) : (EPT == 8 ? 8 : 4);
  int r = N % 3 == 0 ? N / 3 : N;
  while (r % big == 0 && r > big) { p.radix[p.nst++] = big; r /= big; }
  if (r > 1) p.radix[p.nst++] = r;
  if (N % 3 == 0) p.radix[p.nst++] = 3;
  p.tpl = N / p.ept;
  int ns = 1, off = 0;
  for (int s = 0; s < p.nst; ++s) {
    p.ns[s] = ns;
    p.twoff[s] = off;
    if (s > 0) off += (p.radix[s] - 1) * ns;
    ns *= p.radix[s];
  }
  p.twtotal = off;
  return p;
}

// padded shared-memory index (one spare slot per 16 complex values)
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int line_len(int N) { return N + N / 16 + 2; }   // complex slots

// Lines whose raw values and two ping-pong buffers would not fit in shared memory (FP64,
// N >= 6144) use one buffer: every stage then reads all its inputs into registers, waits
// at a barrier, and writes its outputs over them.
template <typename T, int N>
__host__ __device__ constexpr bool one_buffer() {
  return ((size_t)(N + 2) * sizeof(T) + 15) / 16 * 16 + 2 * (size_t)line_len(N) * 2 * sizeof(T) >
         220 * 1024;
}
template <typename T, int N>
__host__ __device__ constexpr int line_buffers() { return one_buffer<T, N>() ? 1 : 2; }

// value m of the packed odd extension z_m of a line x (x_0 = 0, x_N = 0):
// (x_{2m}, x_{2m+1}) for m < N/2, (-x_{2m'}, -x_{2m'-1}) with m' = N - m otherwise
template <typename T, int N>
__device__ __forceinline__ cx<T> packed(const T* line, int m, bool upper) {
  if (!upper) return *reinterpret_cast<const cx<T>*>(line + 2 * m);
  const int mp = N - m;                       // 0 < mp <= N/2
  const T hi = (mp < N / 2) ? line[2 * mp] : T(0);
  return {-hi, -line[2 * mp - 1]};
}

// Butterflies of stage S on the values v already loaded for this thread (input r of
// butterfly q at v[q R + r], butterfly index j = t + q tpl): twiddle by the stage table
// tws[(r - 1) Ns + j mod Ns] = W_N^{(j mod Ns) r N/(Ns R)}, DFT_R, and store output r to
// zo[(j - j mod Ns) R + j mod Ns + r Ns].
template <typename T, int N, int EPT, int S>
__device__ __forceinline__ void butterflies(cx<T>* zo, int t, const cx<T>* __restrict__ stw,
                                            cx<T>* v) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int R = P.radix[S], Ns = P.ns[S], NB = P.ept / R;
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = t + q * P.tpl;
    const int jm = j & (Ns - 1);
    if constexpr (Ns > 1) {
      const cx<T>* tws = stw + P.twoff[S] + jm;
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], tws[(r - 1) * Ns]);
    }
    dft<T, R>(&v[q * R]);
    const int out0 = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) zo[pad(out0 + r * Ns)] = v[q * R + r];
  }
}

// Stages 1..nst-1, ping-ponging between the two line buffers; stage 0 has already been
// written to z0.  Returns with the last stage's outputs in v (output r of butterfly q at
// v[q R + r]) and in buffer zbuf[(nst - 1) % 2]; one barrier per stage.
template <typename T, int N, int EPT, int S>
__device__ __forceinline__ void later_stages(cx<T>* z0, cx<T>* z1, int t,
                                             const cx<T>* __restrict__ stw, cx<T>* v) {
  constexpr CPlan P = cplan(N, EPT);
  if constexpr (S < P.nst) {
    constexpr int R = P.radix[S], NB = P.ept / R, STR = N / R;
    // stage s writes buffer s % 2: stage S reads what stage S-1 wrote, writes the other
    // (z1 == z0 in single-buffer mode)
    cx<T>* src = ((S - 1) % 2 == 0) ? z0 : z1;
    cx<T>* dst = ((S - 1) % 2 == 0) ? z1 : z0;
#pragma unroll
    for (int q = 0; q < NB; ++q)
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = src[pad(t + q * P.tpl + r * STR)];
    if constexpr (one_buffer<T, N>()) __syncthreads();
    butterflies<T, N, EPT, S>(dst, t, stw, v);
    __syncthreads();
    later_stages<T, N, EPT, S + 1>(z0, z1, t, stw, v);
  }
}

template <typename T, int N, int EPT>
__device__ __forceinline__ cx<T>* last_buffer(cx<T>* z0, cx<T>* z1) {
  return ((cplan(N, EPT).nst - 1) % 2 == 0) ? z0 : z1;
}

// DST-I outputs held by this thread after the last stage: output e = q R + r is X_k with
// k = t + q tpl + r N/R (R the last radix), formed from v[e] = Z_k and the partner
// Z_{N-k} read from the last stage's buffer zl, and handed to f(e, k, X_k).
template <typename T, int N, int EPT, typename F>
__device__ __forceinline__ void dst_outputs(const cx<T>* zl, int t, const cx<T>* __restrict__ tw,
                                            cx<T>* v, F&& f) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int R = P.radix[P.nst - 1], NB = P.ept / R, STR = N / R;
#pragma unroll
  for (int q = 0; q < NB; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int k = t + q * P.tpl + r * STR;
      const cx<T> a = v[q * R + r];
      const cx<T> b = zl[pad(N - k)];           // k = 0 reads a discarded slot
      const cx<T> w = tw[k];                    // (cos, -sin)(pi k / N)
      const T val = T(0.25) * (-(a.y - b.y) + w.x * (a.x - b.x) - w.y * (a.y + b.y));
      f(q * R + r, k, (k == 0) ? T(0) : val);
    }
}

template <typename T, int N, int EPT>
__device__ __forceinline__ int out_index(int t, int e) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int R = P.radix[P.nst - 1], STR = N / R;
  return t + (e / R) * P.tpl + (e % R) * STR;
}

// One DST-I of a line whose raw values are read by `at(i)` (i < N, at(0) = 0): stage 0 forms
// the packed odd extension from the raw values directly, the remaining stages run in
// shared memory, the outputs are handed to f(e, k, X_k).  Ends with a barrier-free read of
// the last buffer; the caller synchronises before the buffers are reused.
struct NoHook {
  __device__ void operator()() const {}
};

// after0() runs once the raw values have been consumed (after stage 0's barrier)
template <typename T, int N, int EPT, typename Raw, typename F, typename A = NoHook>
__device__ __forceinline__ void dst_line(Raw&& load_pair, cx<T>* z0, cx<T>* z1, int t,
                                         const cx<T>* __restrict__ stw,
                                         const cx<T>* __restrict__ tw, F&& f, A&& after0 = A{}) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int R = P.radix[0], NB = P.ept / R, STR = N / R;
  cx<T> v[P.ept];
#pragma unroll
  for (int q = 0; q < NB; ++q)
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = load_pair(t + q * P.tpl + r * STR, 2 * r >= R);
  butterflies<T, N, EPT, 0>(z0, t, stw, v);
  __syncthreads();
  after0();
  later_stages<T, N, EPT, 1>(z0, z1, t, stw, v);
  dst_outputs<T, N, EPT>(last_buffer<T, N, EPT>(z0, z1), t, tw, v, f);
}

// ---------------------------------------------------------------------------- line staging
// The next block of contiguous lines is brought into shared memory by one bulk
// asynchronous copy (completion counted on an mbarrier) while the current block is
// transformed.  Waits are bounded: after `polls` polls (kPollLimit unless a test lowers it)
// the kernel records a timeout in *err (when given), then waits up to kPollLimit more
// polls for its own copy in flight (so no copy into shared memory outlives the wait) and
// goes on, so a lost copy cannot hang the GPU.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void stage_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// one thread: copy `bytes` (a multiple of 16, both addresses 16-byte aligned) to dst
__device__ __forceinline__ void stage_issue(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

constexpr int kPollLimit = 1 << 20;

__device__ __forceinline__ bool stage_poll(uint32_t a, uint32_t parity, int polls) {
  for (int i = 0; i < polls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void stage_wait(uint64_t* bar, uint32_t parity, int* err, int polls) {
  const uint32_t a = smem_addr(bar);
  if (stage_poll(a, parity, polls)) return;
  if (err) atomicOr(err, 1);
  stage_poll(a, parity, kPollLimit);           // drain the copy still in flight
}

// shared-memory bytes: FFT buffers of the row pass, and whether a staging line fits
template <typename T, int N, int EPT>
__host__ __device__ constexpr int rows_lpc() {
  return cplan(N, EPT).tpl >= 256 ? 1 : 256 / cplan(N, EPT).tpl;
}
template <typename T, int N, int EPT>
__host__ __device__ constexpr size_t rows_fft_bytes() {
  return ((size_t)rows_lpc<T, N, EPT>() * line_buffers<T, N>() * line_len(N) * sizeof(cx<T>) + 15) / 16 * 16;
}
template <typename T, int N, int EPT>
__host__ __device__ constexpr bool rows_staged() {
  return rows_fft_bytes<T, N, EPT>() + (size_t)rows_lpc<T, N, EPT>() * N * sizeof(T) <= 220 * 1024;
}

// ---------------------------------------------------------------------------- pass 1/3
// DST-I along every row: out[row] = scale * DST(in[row]) for the nlines contiguous rows of
// length N (N rows of a 2-D grid, N^2 x-lines of a 3-D grid); in may equal out.  LPC lines
// per CTA, persistent grid-stride loop.  Stage 0 reads the rows from a shared-memory
// staging block filled by a bulk asynchronous copy issued while the previous block was
// transformed (straight from global memory where the staging block does not fit); the
// odd-extension mirror is address arithmetic; outputs go straight to global memory.
template <typename T, int N, int EPT>
__global__ void __launch_bounds__((cplan(N, EPT).tpl > 256 ? cplan(N, EPT).tpl : 256),
                                  ((cplan(N, EPT).tpl > 256 && EPT >= 16) ? 1 : 2))
    rows_kernel(const T* in, T* out, const cx<T>* __restrict__ stw, const cx<T>* __restrict__ tw,
                T scale, int nlines, int* err, int polls) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr bool STG = rows_staged<T, N, EPT>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  const int lpc = blockDim.x / P.tpl;
  const int line = threadIdx.x / P.tpl, t = threadIdx.x - line * P.tpl;
  constexpr int NBUF = line_buffers<T, N>();
  cx<T>* z0 = reinterpret_cast<cx<T>*>(smem_raw) + line * NBUF * line_len(N);
  cx<T>* z1 = z0 + (NBUF - 1) * line_len(N);
  T* stage = reinterpret_cast<T*>(smem_raw + rows_fft_bytes<T, N, EPT>());   // lpc lines
  const int step = gridDim.x * lpc;
  auto issue = [&](int r0) {
    const int cnt = min(lpc, nlines - r0);
    stage_issue(stage, in + (size_t)r0 * N, (uint32_t)(cnt * N * sizeof(T)), &bar);
  };
  int row0 = blockIdx.x * lpc;
  if constexpr (STG) {
    if (threadIdx.x == 0) stage_init(&bar);
    __syncthreads();
    if (threadIdx.x == 0 && row0 < nlines) issue(row0);
  }
  for (int it = 0; row0 < nlines; row0 += step, ++it) {
    const int row = row0 + line;
    const bool active = row < nlines;
    T* dst = out + (size_t)row * N;
    if constexpr (STG) {
      stage_wait(&bar, (uint32_t)(it & 1), err, polls);
      const T* src = stage + (size_t)line * N;
      dst_line<T, N, EPT>(
          [&](int m, bool upper) {
            return active ? packed<T, N>(src, m, upper) : cx<T>{T(0), T(0)};
          },
          z0, z1, t, stw, tw,
          [&](int, int k, T x) {
            if (active) dst[k] = x * scale;
          },
          [&] {                               // staging consumed: fetch the next block
            if (threadIdx.x == 0 && row0 + step < nlines) issue(row0 + step);
          });
    } else {
      const T* src = in + (size_t)(active ? row : 0) * N;
      dst_line<T, N, EPT>([&](int m, bool upper) {
                            return active ? packed<T, N>(src, m, upper) : cx<T>{T(0), T(0)};
                          },
                          z0, z1, t, stw, tw, [&](int, int k, T x) {
                            if (active) dst[k] = x * scale;
                          });
    }
    __syncthreads();
  }
}

template <int B> struct RawVec;
template <> struct RawVec<4> { typedef unsigned int type; };
template <> struct RawVec<8> { typedef uint2 type; };
template <> struct RawVec<16> { typedef uint4 type; };

// FP32: the hardware approximate reciprocal (relative error within 2^-22, a few ulp of the
// FP32 transform's own rounding), one instruction instead of a correctly rounded sequence
__device__ __forceinline__ float recip(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}
__device__ __forceinline__ double recip(double d) {
  // Newton-Raphson from the approximate FP32 reciprocal: two steps reach FP64 accuracy
  double r = (double)recip((float)d);
  r = r * (2.0 - d * r);
  r = r * (2.0 - d * r);
  return r;
}

// shared memory of one column line: raw values (N + 2 reals) and two FFT buffers
template <typename T, int N>
__host__ __device__ constexpr size_t col_line_bytes() {
  return ((size_t)(N + 2) * sizeof(T) + 15) / 16 * 16 +
         line_buffers<T, N>() * (size_t)line_len(N) * 2 * sizeof(T);
}

// the column tile is staged through shared memory unless one line alone fills it
template <typename T, int N>
__host__ __device__ constexpr bool cols_staged() {
  return col_line_bytes<T, N>() + (size_t)N * sizeof(T) <= 220 * 1024;
}

// column tile width: largest power of two <= 32 dividing N with L * tpl threads within
// the bound and L line buffers plus the staging tile within 220 KB of shared memory
template <typename T, int N, int EPT, int MAXT>
__host__ __device__ constexpr int cols_L() {
  constexpr CPlan P = cplan(N, EPT);
  int L = 1;
  while (L < 32 && N % (2 * L) == 0 && 2 * L * P.tpl <= MAXT &&
         (size_t)(2 * L) * (col_line_bytes<T, N>() + N * sizeof(T)) <= 220 * 1024)
    L *= 2;
  return L;
}

// ---------------------------------------------------------------------------- pass 2
// L consecutive columns (x-modes k) per CTA: DST-I along y, multiply by
// scale / (lam[k] + lam[l] - kappa^2), DST-I along y again.  The next column tile is
// copied into a shared-memory staging area with cp.async while the current one is
// transformed.
template <typename T, int N, int EPT, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT <= 256 ? 2 : 1)) cols_kernel(T* V, const cx<T>* __restrict__ stw,
                                                    const cx<T>* __restrict__ tw,
                                                    const T* __restrict__ lam, T kappa2, T scale) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int L = cols_L<T, N, EPT, MAXT>();
  constexpr int CH = (L * (int)sizeof(T) >= 16) ? L * (int)sizeof(T) / 16 : 1;
  constexpr int W = L / CH;
  constexpr int VB = W * (int)sizeof(T);
  constexpr int NCH = N * CH;                   // chunks per tile
  constexpr size_t LB = col_line_bytes<T, N>();
  typedef typename RawVec<VB>::type Raw;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Raw* stage_buf = reinterpret_cast<Raw*>(smem_raw + L * LB);   // N rows x L values
  const int line = threadIdx.x / P.tpl, t = threadIdx.x - line * P.tpl;
  unsigned char* lb = smem_raw + line * LB;
  T* raw = reinterpret_cast<T*>(lb);
  cx<T>* z0 = reinterpret_cast<cx<T>*>(lb + ((size_t)(N + 2) * sizeof(T) + 15) / 16 * 16);
  cx<T>* z1 = z0 + (line_buffers<T, N>() - 1) * line_len(N);
  constexpr bool STAGED = cols_staged<T, N>();
  static_assert(STAGED || L == 1, "an unstaged column tile holds one column");
  const int nthr = blockDim.x;
  auto raw_of = [&](int c) { return reinterpret_cast<T*>(smem_raw + c * LB); };

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
  if constexpr (STAGED) {
    if (c0 < N) prefetch(c0);
  }
  for (; c0 < N; c0 += gridDim.x * L) {
    if constexpr (STAGED) {
      asm volatile("cp.async.wait_group 0;\n" ::);
      __syncthreads();
      // staging tile -> raw lines
      for (int g = threadIdx.x; g < NCH; g += nthr) {
        const int r = g / CH, cc = g - r * CH;
        const Raw pk = stage_buf[g];
        const T* vals = reinterpret_cast<const T*>(&pk);
#pragma unroll
        for (int w = 0; w < W; ++w) raw_of(cc * W + w)[r] = vals[w];
      }
      __syncthreads();
      if (c0 + gridDim.x * L < N) prefetch(c0 + gridDim.x * L);
    } else {
      __syncthreads();                        // previous column written back
      for (int r = threadIdx.x; r < N; r += nthr) raw[r] = V[(size_t)r * N + c0];
      __syncthreads();
    }
    const int k = c0 + line;
    const T lk = lam[k] - kappa2;
    T X[P.ept];
    // forward transform with the spectral division; results replace the raw line (the
    // raw values were consumed by stage 0 before its barrier)
    dst_line<T, N, EPT>([&](int m, bool upper) { return packed<T, N>(raw, m, upper); }, z0, z1,
                        t, stw, tw, [&](int e, int l, T x) {
                          X[e] = (k == 0 || l == 0) ? T(0) : x * scale * recip(lk + lam[l]);
                        });
#pragma unroll
    for (int e = 0; e < P.ept; ++e) raw[out_index<T, N, EPT>(t, e)] = X[e];
    __syncthreads();
    dst_line<T, N, EPT>([&](int m, bool upper) { return packed<T, N>(raw, m, upper); }, z0, z1,
                        t, stw, tw, [&](int e, int, T x) { X[e] = x; });
    // stage 0 of the second transform consumed raw before a barrier: safe to overwrite
#pragma unroll
    for (int e = 0; e < P.ept; ++e) raw[out_index<T, N, EPT>(t, e)] = X[e];
    __syncthreads();
    if constexpr (STAGED) {
      for (int g = threadIdx.x; g < NCH; g += nthr) {
        const int r = g / CH, cc = g - r * CH;
        Raw pk;
        T* vals = reinterpret_cast<T*>(&pk);
#pragma unroll
        for (int w = 0; w < W; ++w) vals[w] = raw_of(cc * W + w)[r];
        *reinterpret_cast<Raw*>(V + (size_t)r * N + c0 + cc * W) = pk;
      }
    } else {
      for (int r = threadIdx.x; r < N; r += nthr) V[(size_t)r * N + c0] = raw[r];
    }
  }
  if constexpr (STAGED) asm volatile("cp.async.wait_group 0;\n" ::);
}

// ---------------------------------------------------------------------------- pass 2, transposed
// The column pass on contiguous lines: the work grid is transposed so that x-mode k is
// row k, every row gets DST-I along y, the spectral division and DST-I again (the
// product of the inverse scales (2/N)^2 included), and the grid is transposed back.
// Reads and writes are whole rows (and 32 x 32 tiles in the transposes) instead of the
// narrow column tiles of cols_kernel.
// out = in^T for an R x C matrix (out is C x R); blockIdx.z walks a batch of such
// matrices stored back to back.  32 x 32 tiles through shared memory, any R and C.
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ in, T* __restrict__ out, int R, int C) {
  __shared__ T tile[32][33];
  const size_t base = (size_t)blockIdx.z * R * C;
  in += base;
  out += base;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;   // column, row of the input tile
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int y = by + r, x = bx + threadIdx.x;
    if (x < C && y < R) tile[r][threadIdx.x] = in[(size_t)y * C + x];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int y = bx + r, x = by + threadIdx.x;           // row y of out = column y of in
    if (x < R && y < C) out[(size_t)y * R + x] = tile[threadIdx.x][r];
  }
}

// 16-byte vectors: 64 x 64 FP32 or 32 x 32 FP64 tiles, 16 x 16 threads, each row of a tile
// moved by 16 threads as one contiguous 256-byte segment (R and C multiples of the tile)
template <typename T>
__global__ void __launch_bounds__(256) transpose_vec_kernel(const T* __restrict__ in,
                                                            T* __restrict__ out, int R, int C) {
  constexpr int VEC = 16 / sizeof(T), TILE = 16 * VEC;
  typedef typename RawVec<16>::type V16;
  __shared__ T tile[TILE][TILE + 1];
  const size_t base = (size_t)blockIdx.z * R * C;
  in += base;
  out += base;
  const int bx = blockIdx.x * TILE, by = blockIdx.y * TILE;
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int r = 0; r < TILE / 16; ++r) {
    const int y = by + ty + 16 * r;
    const V16 pk = *reinterpret_cast<const V16*>(in + (size_t)y * C + bx + tx * VEC);
    const T* vals = reinterpret_cast<const T*>(&pk);
#pragma unroll
    for (int e = 0; e < VEC; ++e) tile[ty + 16 * r][tx * VEC + e] = vals[e];
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < TILE / 16; ++r) {
    const int y = bx + ty + 16 * r;                 // row y of out = column y of in
    V16 pk;
    T* vals = reinterpret_cast<T*>(&pk);
#pragma unroll
    for (int e = 0; e < VEC; ++e) vals[e] = tile[tx * VEC + e][ty + 16 * r];
    *reinterpret_cast<V16*>(out + (size_t)y * R + by + tx * VEC) = pk;
  }
}

// batch x (R x C) -> batch x (C x R)
template <typename T>
kfbi_status launch_transpose(Ctx& c, const T* in, T* out, int R, int C, int batch) {
  constexpr int TILE = 16 * (16 / sizeof(T));
  const int pr = prof_begin(c, ST_TRANS);
  if (R % TILE == 0 && C % TILE == 0) {
    transpose_vec_kernel<T><<<dim3(C / TILE, R / TILE, batch), dim3(16, 16), 0, c.stream>>>(in, out, R, C);
  } else {
    transpose_kernel<T><<<dim3((C + 31) / 32, (R + 31) / 32, batch), dim3(32, 8), 0, c.stream>>>(in, out, R, C);
  }
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

// lines per CTA of the transposed column pass: as many as make 256 threads, within the
// shared memory of a raw line plus its FFT buffers per line
template <typename T, int N, int EPT>
__host__ __device__ constexpr int yline_lpc() {
  constexpr CPlan P = cplan(N, EPT);
  int l = P.tpl >= 256 ? 1 : 256 / P.tpl;
  while (l > 1 && (size_t)l * col_line_bytes<T, N>() > 220 * 1024) l /= 2;
  return l;
}

// DIM = 2: line k of U is x-mode k (divisor lam[k] + lam[l] - kappa^2);
// DIM = 3: line L = i N + j holds x-mode i, y-mode j (divisor lam[i] + lam[j] + lam[l] -
// kappa^2); nlines = N^(DIM-1); scale = (2/N)^DIM
template <typename T, int N, int EPT>
__host__ __device__ constexpr bool yline_staged() {
  return (size_t)yline_lpc<T, N, EPT>() * (col_line_bytes<T, N>() + N * sizeof(T)) <= 220 * 1024;
}
template <typename T, int N, int EPT>
__host__ __device__ constexpr size_t yline_smem() {
  return (size_t)yline_lpc<T, N, EPT>() *
         (col_line_bytes<T, N>() + (yline_staged<T, N, EPT>() ? N * sizeof(T) : 0));
}

template <typename T, int N, int EPT, int DIM>
__global__ void __launch_bounds__((cplan(N, EPT).tpl > 256 ? cplan(N, EPT).tpl : 256),
                                  ((cplan(N, EPT).tpl > 256 && EPT >= 16) ? 1 : 2))
    yline_kernel(T* U, const cx<T>* __restrict__ stw, const cx<T>* __restrict__ tw,
                 const T* __restrict__ lam, T kappa2, T scale, int nlines, int* err, int polls) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr size_t LB = col_line_bytes<T, N>();
  constexpr bool STG = yline_staged<T, N, EPT>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  const int lpc = blockDim.x / P.tpl;
  const int line = threadIdx.x / P.tpl, t = threadIdx.x - line * P.tpl;
  unsigned char* lb = smem_raw + line * LB;
  T* raw = reinterpret_cast<T*>(lb);
  cx<T>* z0 = reinterpret_cast<cx<T>*>(lb + ((size_t)(N + 2) * sizeof(T) + 15) / 16 * 16);
  cx<T>* z1 = z0 + (line_buffers<T, N>() - 1) * line_len(N);
  T* stage = reinterpret_cast<T*>(smem_raw + (size_t)lpc * LB);        // lpc lines
  const int step = gridDim.x * lpc;
  auto issue = [&](int r0) {
    const int cnt = min(lpc, nlines - r0);
    stage_issue(stage, U + (size_t)r0 * N, (uint32_t)(cnt * N * sizeof(T)), &bar);
  };
  if constexpr (STG) {
    if (threadIdx.x == 0) stage_init(&bar);
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x * lpc < nlines) issue(blockIdx.x * lpc);
  }
  int it = 0;
  for (int k0 = blockIdx.x * lpc; k0 < nlines; k0 += step, ++it) {
    const int k = k0 + line;
    bool active = k < nlines;
    T* row = U + (size_t)(active ? k : 0) * N;
    T lk = T(0);
    if (active) {
      if constexpr (DIM == 2) {
        lk = lam[k] - kappa2;
      } else {
        const int i = k / N, j = k - (k / N) * N;
        lk = lam[i] + lam[j] - kappa2;
        active = active && i > 0 && j > 0;          // boundary modes stay zero
      }
    }
    const bool zero_line = !active || (DIM == 2 && k == 0);
    // forward transform and spectral division into the raw line
    auto divide = [&](int, int l, T x) {
      raw[l] = (zero_line || l == 0) ? T(0) : x * scale * recip(lk + lam[l]);
    };
    if constexpr (STG) {
      stage_wait(&bar, (uint32_t)(it & 1), err, polls);
      const T* src = stage + (size_t)line * N;
      dst_line<T, N, EPT>(
          [&](int m, bool upper) {
            return active ? packed<T, N>(src, m, upper) : cx<T>{T(0), T(0)};
          },
          z0, z1, t, stw, tw, divide, [&] {
            if (threadIdx.x == 0 && k0 + step < nlines) issue(k0 + step);
          });
    } else {
      dst_line<T, N, EPT>([&](int m, bool upper) {
                            return active ? packed<T, N>(row, m, upper) : cx<T>{T(0), T(0)};
                          },
                          z0, z1, t, stw, tw, divide);
    }
    __syncthreads();
    dst_line<T, N, EPT>([&](int m, bool upper) { return packed<T, N>(raw, m, upper); }, z0, z1,
                        t, stw, tw, [&](int, int j, T x) {
                          if (k < nlines) row[j] = x;
                        });
    __syncthreads();
  }
}

// The low x-modes of the row-layout y-pass (2-D): column k < ncols of the row-layout grid
// V (x-mode k along y, stride N) takes DST-I along y, the spectral division and DST-I again
// and is written to column k of Y.  Stage 0 gathers the column straight from global memory
// (each strided value one 32-byte sector, served by L2, where the preceding pass left the
// grid) and the outputs are scattered back, so no transposed copy of the low modes is
// made.  Shared memory holds the raw line and the FFT buffers of each of the lpc lines.
template <typename T, int N, int EPT>
__global__ void __launch_bounds__((cplan(N, EPT).tpl > 256 ? cplan(N, EPT).tpl : 256),
                                  ((cplan(N, EPT).tpl > 256 && EPT >= 16) ? 1 : 2))
    ycol_lines_kernel(const T* __restrict__ V, T* __restrict__ Y, const cx<T>* __restrict__ stw,
                      const cx<T>* __restrict__ tw, const T* __restrict__ lam, T kappa2,
                      T scale, int ncols) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr size_t LB = col_line_bytes<T, N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lpc = blockDim.x / P.tpl;
  const int line = threadIdx.x / P.tpl, t = threadIdx.x - line * P.tpl;
  unsigned char* lb = smem_raw + line * LB;
  T* raw = reinterpret_cast<T*>(lb);
  cx<T>* z0 = reinterpret_cast<cx<T>*>(lb + ((size_t)(N + 2) * sizeof(T) + 15) / 16 * 16);
  cx<T>* z1 = z0 + (line_buffers<T, N>() - 1) * line_len(N);
  for (int kk = blockIdx.x * lpc; kk < ncols; kk += gridDim.x * lpc) {
    const int k = kk + line;
    const bool active = k < ncols;
    const T* col = V + (active ? k : 0);
    const T lk = active ? lam[k] - kappa2 : T(0);
    const bool zero_line = !active || k == 0;
    auto at = [&](int j) -> T { return col[(size_t)j * N]; };       // 0 <= j < N
    // forward transform of the packed odd extension of the column, spectral division
    dst_line<T, N, EPT>(
        [&](int m, bool upper) -> cx<T> {
          if (!active) return cx<T>{T(0), T(0)};
          if (!upper) return cx<T>{at(2 * m), at(2 * m + 1)};
          const int mp = N - m;                                     // 0 < mp <= N/2
          const T hi = (mp < N / 2) ? at(2 * mp) : T(0);
          return cx<T>{-hi, -at(2 * mp - 1)};
        },
        z0, z1, t, stw, tw, [&](int, int l, T x) {
          raw[l] = (zero_line || l == 0) ? T(0) : x * scale * recip(lk + lam[l]);
        });
    __syncthreads();
    dst_line<T, N, EPT>([&](int m, bool upper) { return packed<T, N>(raw, m, upper); }, z0, z1,
                        t, stw, tw, [&](int, int j, T x) {
                          if (active) Y[(size_t)j * N + k] = x;
                        });
    __syncthreads();
  }
}

// dynamic shared memory of the two kernels
template <typename T, int N, int EPT>
__host__ __device__ constexpr size_t rows_smem(int lpc) {
  return rows_fft_bytes<T, N, EPT>() +
         (rows_staged<T, N, EPT>() ? (size_t)lpc * N * sizeof(T) : 0);
}
template <typename T, int N, int EPT, int MAXT>
__host__ __device__ constexpr size_t cols_smem() {
  constexpr int L = cols_L<T, N, EPT, MAXT>();
  return (size_t)L * col_line_bytes<T, N>() + (cols_staged<T, N>() ? (size_t)N * L * sizeof(T) : 0);
}

// ---------------------------------------------------------------------------- tables
// stage twiddles of the plan (N, EPT): entry twoff[s] + (r - 1) Ns + jm holds
// W_N^{jm r N/(Ns R)}, written from the base table tw[i] = e^{-i pi i/N}
template <typename T, int N, int EPT>
__global__ void stage_twiddles_kernel(const cx<T>* __restrict__ tw, cx<T>* __restrict__ stw) {
  constexpr CPlan P = cplan(N, EPT);
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= P.twtotal) return;
  int s = 1;
  while (s + 1 < P.nst && e >= P.twoff[s + 1]) ++s;
  const int loc = e - P.twoff[s], Ns = P.ns[s], R = P.radix[s];
  const int r = loc / Ns + 1, jm = loc - (r - 1) * Ns;
  stw[e] = tw[2 * ((jm * r * (N / (Ns * R))) % N)];
}

// ---------------------------------------------------------------------------- launch
inline int sm_count() {
  static const int n = [] {            // initialised once, thread-safe
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }();
  return n;
}

// per-plan stage-twiddle tables, built on first use for this context and precision
template <typename T, int N, int EPT>
kfbi_status stage_table(Ctx& c, const cx<T>* tw, const cx<T>** out) {
  constexpr CPlan P = cplan(N, EPT);
  const int slot = (sizeof(T) == 8 ? 2 : 0) + (EPT == default_ept(N) ? 0 : 1);
  if (!c.stw[slot]) {
    KFBI_TRY(alloc_bytes(c, &c.stw[slot], sizeof(cx<T>) * (P.twtotal > 0 ? P.twtotal : 1)));
    if (P.twtotal > 0) {
      prof_count(c, ST_SETUP);
      stage_twiddles_kernel<T, N, EPT><<<(P.twtotal + 255) / 256, 256, 0, c.stream>>>(
          tw, reinterpret_cast<cx<T>*>(c.stw[slot]));
      KFBI_CUDA_TRY(cudaGetLastError());
    }
  }
  *out = reinterpret_cast<const cx<T>*>(c.stw[slot]);
  return KFBI_OK;
}

template <typename T, int N, int EPT>
kfbi_status launch_rows(Ctx& c, const T* in, T* out, const cx<T>* tw, T scale, int nlines = N) {
  constexpr CPlan P = cplan(N, EPT);
  const cx<T>* stw = nullptr;
  KFBI_TRY((stage_table<T, N, EPT>(c, tw, &stw)));
  constexpr int lpc = P.tpl >= 256 ? 1 : 256 / P.tpl;
  static_assert(rows_smem<T, N, EPT>(lpc) <= 227 * 1024, "row pass exceeds shared memory");
  const int threads = lpc * P.tpl;
  const size_t smem = rows_smem<T, N, EPT>(lpc);
  KFBI_TRY(set_smem_limit((const void*)rows_kernel<T, N, EPT>, smem));
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_kernel<T, N, EPT>,
                                                              threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = (nlines + lpc - 1) / lpc;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_ROWS32 : ST_ROWS64);
  rows_kernel<T, N, EPT><<<blocks, threads, smem, c.stream>>>(in, out, stw, tw, scale, nlines,
                                                              c.err_flag + 2, c.poll_limit);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T, int N, int EPT, int MAXT>
kfbi_status launch_cols(Ctx& c, T* V, const cx<T>* tw, const T* lam) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int L = cols_L<T, N, EPT, MAXT>();
  const cx<T>* stw = nullptr;
  KFBI_TRY((stage_table<T, N, EPT>(c, tw, &stw)));
  static_assert(cols_smem<T, N, EPT, MAXT>() <= 227 * 1024, "column pass exceeds shared memory");
  const int threads = L * P.tpl;
  const size_t smem = cols_smem<T, N, EPT, MAXT>();
  KFBI_TRY(set_smem_limit((const void*)cols_kernel<T, N, EPT, MAXT>, smem));
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, cols_kernel<T, N, EPT, MAXT>, threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = N / L;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const T scale = T((2.0 / N) * (2.0 / N));
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_COLS32 : ST_COLS64);
  cols_kernel<T, N, EPT, MAXT><<<blocks, threads, smem, c.stream>>>(V, stw, tw, lam, T(c.kappa2),
                                                                    scale);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T, int N, int EPT>
kfbi_status launch_ylines(Ctx& c, T* V, const cx<T>* tw, const T* lam) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int lpc = yline_lpc<T, N, EPT>();
  static_assert(yline_smem<T, N, EPT>() <= 227 * 1024, "transposed column pass exceeds shared memory");
  const cx<T>* stw = nullptr;
  KFBI_TRY((stage_table<T, N, EPT>(c, tw, &stw)));
  T* X = reinterpret_cast<T*>(c.XT);
  const int threads = lpc * P.tpl;
  const size_t smem = yline_smem<T, N, EPT>();
  KFBI_TRY(set_smem_limit((const void*)yline_kernel<T, N, EPT, 2>, smem));
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, yline_kernel<T, N, EPT, 2>,
                                                              threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = (N + lpc - 1) / lpc;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const T scale = T((2.0 / N) * (2.0 / N));
  KFBI_TRY(launch_transpose<T>(c, V, X, N, N, 1));
  // FP32: the well-conditioned x-modes k >= tri_k0 are solved along y by elimination
  const int nfft = (std::is_same<T, float>::value && c.tri_k0 > 0 && c.tri_k0 < N) ? c.tri_k0 : N;
  const int fblocks = blocks < (nfft + lpc - 1) / lpc ? blocks : (nfft + lpc - 1) / lpc;
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_COLS32 : ST_COLS64);
  yline_kernel<T, N, EPT, 2><<<fblocks, threads, smem, c.stream>>>(X, stw, tw, lam, T(c.kappa2),
                                                                   scale, nfft, c.err_flag + 2,
                                                                   c.poll_limit);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  if constexpr (std::is_same<T, float>::value)
    if (nfft < N) KFBI_TRY(ytri_f32(c, X, nfft));
  KFBI_TRY(launch_transpose<T>(c, X, V, N, N, 1));
  return KFBI_OK;
}

// the y-transform pair alone on an already transposed grid (2-D): lines [0, nlines) of X,
// or, when nlines < 0, the lines below tri_k0 (FP32) followed by the tridiagonal pass on
// the others
template <typename T, int N, int EPT>
kfbi_status launch_ylines_only(Ctx& c, T* X, const cx<T>* tw, const T* lam, int nlines) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int lpc = yline_lpc<T, N, EPT>();
  const cx<T>* stw = nullptr;
  KFBI_TRY((stage_table<T, N, EPT>(c, tw, &stw)));
  const int threads = lpc * P.tpl;
  const size_t smem = yline_smem<T, N, EPT>();
  KFBI_TRY(set_smem_limit((const void*)yline_kernel<T, N, EPT, 2>, smem));
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, yline_kernel<T, N, EPT, 2>,
                                                              threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = (N + lpc - 1) / lpc;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const T scale = T((2.0 / N) * (2.0 / N));
  const bool split = nlines < 0;
  const int nfft = !split ? nlines
                          : ((std::is_same<T, float>::value && c.tri_k0 > 0 && c.tri_k0 < N) ? c.tri_k0 : N);
  const int fblocks = blocks < (nfft + lpc - 1) / lpc ? blocks : (nfft + lpc - 1) / lpc;
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_COLS32 : ST_COLS64);
  yline_kernel<T, N, EPT, 2><<<fblocks, threads, smem, c.stream>>>(X, stw, tw, lam, T(c.kappa2),
                                                                   scale, nfft, c.err_flag + 2,
                                                                   c.poll_limit);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  if constexpr (std::is_same<T, float>::value)
    if (split && nfft < N) KFBI_TRY(ytri_f32(c, X, nfft));
  return KFBI_OK;
}

template <typename T, int N, int EPT>
kfbi_status launch_ycol_lines(Ctx& c, const T* V, T* Y, const cx<T>* tw, const T* lam, int ncols) {
  constexpr CPlan P = cplan(N, EPT);
  constexpr int lpc = yline_lpc<T, N, EPT>();
  static_assert((size_t)lpc * col_line_bytes<T, N>() <= 227 * 1024,
                "low-mode column pass exceeds shared memory");
  const cx<T>* stw = nullptr;
  KFBI_TRY((stage_table<T, N, EPT>(c, tw, &stw)));
  const int threads = lpc * P.tpl;
  const size_t smem = (size_t)lpc * col_line_bytes<T, N>();
  KFBI_TRY(set_smem_limit((const void*)ycol_lines_kernel<T, N, EPT>, smem));
  int per_sm = 0;
  KFBI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ycol_lines_kernel<T, N, EPT>,
                                                              threads, smem));
  if (per_sm < 1) per_sm = 1;
  int blocks = (ncols + lpc - 1) / lpc;
  blocks = blocks < per_sm * sm_count() ? blocks : per_sm * sm_count();
  const T scale = T((2.0 / N) * (2.0 / N));
  const int pr = prof_begin(c, sizeof(T) == 4 ? ST_COLS32 : ST_COLS64);
  ycol_lines_kernel<T, N, EPT><<<blocks, threads, smem, c.stream>>>(V, Y, stw, tw, lam,
                                                                    T(c.kappa2), scale, ncols);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

// the transform pair along y of columns [0, ncols) of the row-layout grid V into Y
template <typename T>
kfbi_status ycol_lines_dispatch(Ctx& c, const T* V, T* Y, const cx<T>* tw, const T* lam, int ncols) {
  switch (c.N) {
#define KFBI_CASE(n) \
  case n: return launch_ycol_lines<T, n, default_ept(n)>(c, V, Y, tw, lam, ncols);
    KFBI_CASE(32) KFBI_CASE(48) KFBI_CASE(64) KFBI_CASE(96) KFBI_CASE(128) KFBI_CASE(192)
    KFBI_CASE(256) KFBI_CASE(384) KFBI_CASE(512) KFBI_CASE(768) KFBI_CASE(1024)
    KFBI_CASE(1536) KFBI_CASE(2048) KFBI_CASE(3072) KFBI_CASE(4096) KFBI_CASE(6144)
    KFBI_CASE(8192)
#undef KFBI_CASE
  }
  set_error("y-transform pass: no compiled plan for N = %d", c.N);
  return KFBI_ERR_UNSUPPORTED;
}

template <typename T>
kfbi_status ylines_dispatch(Ctx& c, T* X, const cx<T>* tw, const T* lam, int nlines = -1) {
  const bool half = (c.cols_variant[sizeof(T) == 8] & 2) != 0;
  switch (c.N) {
#define KFBI_CASE(n)                                                                          \
  case n:                                                                                     \
    if (half && n / (default_ept(n) / 2) <= 512)                                              \
      return launch_ylines_only<T, n, default_ept(n) / 2>(c, X, tw, lam, nlines);             \
    return launch_ylines_only<T, n, default_ept(n)>(c, X, tw, lam, nlines);
    KFBI_CASE(32) KFBI_CASE(48) KFBI_CASE(64) KFBI_CASE(96) KFBI_CASE(128) KFBI_CASE(192)
    KFBI_CASE(256) KFBI_CASE(384) KFBI_CASE(512) KFBI_CASE(768) KFBI_CASE(1024)
    KFBI_CASE(1536) KFBI_CASE(2048) KFBI_CASE(3072) KFBI_CASE(4096) KFBI_CASE(6144)
    KFBI_CASE(8192)
#undef KFBI_CASE
  }
  set_error("y-transform pass: no compiled plan for N = %d", c.N);
  return KFBI_ERR_UNSUPPORTED;
}

// transpose X (x-modes as rows) back into V and DST-I its rows (the last pass of a box
// solve whose column pass ran on X)
template <typename T>
kfbi_status x_pass_dispatch(Ctx& c, const T* X, T* V, const cx<T>* tw);

// Kernel variants chosen by the setup-time autotuner.  Row pass: 0 = default EPT (16 or
// 24 values per thread), 1 = half (8 or 12).  Column pass: bit 0 = CTAs of at most 256
// threads (one column tile per 256 threads, two CTAs per SM) instead of 512, bit 1 =
// half EPT, bit 2 = transposed pass (transpose, yline_kernel, transpose; bit 0 unused).
template <typename T, int N>
kfbi_status launch_rows_v(Ctx& c, const T* in, T* out, const cx<T>* tw, T scale, int variant) {
  constexpr int E = default_ept(N);
  if (variant == 1 && N / (E / 2) <= 512) return launch_rows<T, N, E / 2>(c, in, out, tw, scale);
  return launch_rows<T, N, E>(c, in, out, tw, scale);
}

template <typename T, int N>
kfbi_status launch_cols_v(Ctx& c, T* V, const cx<T>* tw, const T* lam, int variant) {
  constexpr int E = default_ept(N);
  constexpr int EH = E / 2;
  const bool small = variant & 1, half = (variant & 2) != 0;
  if (variant & 4) {
    if (half && N / EH <= 512) return launch_ylines<T, N, EH>(c, V, tw, lam);
    return launch_ylines<T, N, E>(c, V, tw, lam);
  }
  if (half && N / EH <= 512) {
    if (small && N / EH <= 256) return launch_cols<T, N, EH, 256>(c, V, tw, lam);
    return launch_cols<T, N, EH, 512>(c, V, tw, lam);
  }
  if (small && N / E <= 256) return launch_cols<T, N, E, 256>(c, V, tw, lam);
  return launch_cols<T, N, E, 512>(c, V, tw, lam);
}

template <typename T, int N>
kfbi_status box_after_rows_n(Ctx& c, T* work, const cx<T>* tw, const T* lam);

// Time every variant of both passes on the context's scratch work grid and keep the
// fastest for this precision (a column variant is timed with the row pass that follows
// it, since the row-layout y-pass hands that pass its own grid).
template <typename T, int N>
kfbi_status autotune(Ctx& c, T* V, const cx<T>* tw, const T* lam, int* rows_choice,
                     int* cols_choice) {
  cudaEvent_t e0, e1;
  KFBI_CUDA_TRY(cudaEventCreate(&e0));
  KFBI_CUDA_TRY(cudaEventCreate(&e1));
  auto time_it = [&](auto&& launch, float* ms) -> kfbi_status {
    KFBI_TRY(launch());                                     // warm-up (also builds tables)
    KFBI_CUDA_TRY(cudaEventRecord(e0, c.stream));
    for (int rep = 0; rep < 3; ++rep) KFBI_TRY(launch());
    KFBI_CUDA_TRY(cudaEventRecord(e1, c.stream));
    KFBI_CUDA_TRY(cudaEventSynchronize(e1));
    KFBI_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    return KFBI_OK;
  };
  float best = 1e30f;
  for (int v = 0; v < 2; ++v) {
    float ms = 0.f;
    KFBI_TRY(time_it([&] { return launch_rows_v<T, N>(c, V, V, tw, T(1), v); }, &ms));
    if (ms < best) { best = ms; *rows_choice = v; }
  }
  best = 1e30f;
  int best_v = 0;
  // FP32 2-D with well-conditioned modes: also the y-pass on the row layout (variant 8)
  const bool rowpass = std::is_same<T, float>::value && c.dim == 2 && c.ypass_k0 > 0 && c.ypass_k0 < N;
  for (int v : {0, 1, 2, 3, 4, 6, 8}) {
    if (v == 8 && !rowpass) continue;
    float ms = 0.f;
    KFBI_TRY(time_it([&] {
      *cols_choice = v;
      return box_after_rows_n<T, N>(c, V, tw, lam);
    }, &ms));
    if (ms < best) { best = ms; best_v = v; }
  }
  *cols_choice = best_v;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return KFBI_OK;
}

// the box solve after its first row pass: the column pass and the last row pass on work
// (the row-layout y-pass writes its own grid, which the last row pass reads)
template <typename T, int N>
kfbi_status box_after_rows_n(Ctx& c, T* work, const cx<T>* tw, const T* lam) {
  const int rv = c.rows_variant[sizeof(T) == 8], cv = c.cols_variant[sizeof(T) == 8];
  if constexpr (std::is_same<T, float>::value)
    if (cv & 8) {
      KFBI_TRY(ypass_rows_f32(c, work, ypass_out(c)));
      return launch_rows_v<T, N>(c, ypass_out(c), work, tw, T(1), rv);
    }
  KFBI_TRY((launch_cols_v<T, N>(c, work, tw, lam, cv)));
  KFBI_TRY((launch_rows_v<T, N>(c, work, work, tw, T(1), rv)));
  return KFBI_OK;
}

template <typename T, int N>
kfbi_status box_solve_n(Ctx& c, const T* rhs, T* work, const cx<T>* tw, const T* lam) {
  const int rv = c.rows_variant[sizeof(T) == 8];
  KFBI_TRY((launch_rows_v<T, N>(c, rhs, work, tw, T(1), rv)));
  return box_after_rows_n<T, N>(c, work, tw, lam);
}

template <typename T>
kfbi_status box_after_rows_dispatch(Ctx& c, T* work, const cx<T>* tw, const T* lam) {
  switch (c.N) {
#define KFBI_CASE(n) \
  case n: return box_after_rows_n<T, n>(c, work, tw, lam);
    KFBI_CASE(32) KFBI_CASE(48) KFBI_CASE(64) KFBI_CASE(96) KFBI_CASE(128) KFBI_CASE(192)
    KFBI_CASE(256) KFBI_CASE(384) KFBI_CASE(512) KFBI_CASE(768) KFBI_CASE(1024)
    KFBI_CASE(1536) KFBI_CASE(2048) KFBI_CASE(3072) KFBI_CASE(4096) KFBI_CASE(6144)
    KFBI_CASE(8192)
#undef KFBI_CASE
  }
  set_error("box solve: no compiled plan for N = %d", c.N);
  return KFBI_ERR_UNSUPPORTED;
}

// the x-transform of every row of the work grid alone (the first pass of a box solve)
template <typename T>
kfbi_status rows_dispatch(Ctx& c, const T* in, T* out, const cx<T>* tw) {
  const int rv = c.rows_variant[sizeof(T) == 8];
  switch (c.N) {
#define KFBI_CASE(n) \
  case n: return launch_rows_v<T, n>(c, in, out, tw, T(1), rv);
    KFBI_CASE(32) KFBI_CASE(48) KFBI_CASE(64) KFBI_CASE(96) KFBI_CASE(128) KFBI_CASE(192)
    KFBI_CASE(256) KFBI_CASE(384) KFBI_CASE(512) KFBI_CASE(768) KFBI_CASE(1024)
    KFBI_CASE(1536) KFBI_CASE(2048) KFBI_CASE(3072) KFBI_CASE(4096) KFBI_CASE(6144)
    KFBI_CASE(8192)
#undef KFBI_CASE
  }
  set_error("row pass: no compiled plan for N = %d", c.N);
  return KFBI_ERR_UNSUPPORTED;
}

template <typename T>
kfbi_status x_pass_dispatch(Ctx& c, const T* X, T* V, const cx<T>* tw) {
  KFBI_TRY(launch_transpose<T>(c, X, V, c.N, c.N, 1));
  const int rv = c.rows_variant[sizeof(T) == 8];
  switch (c.N) {
#define KFBI_CASE(n) \
  case n: return launch_rows_v<T, n>(c, V, V, tw, T(1), rv);
    KFBI_CASE(32) KFBI_CASE(48) KFBI_CASE(64) KFBI_CASE(96) KFBI_CASE(128) KFBI_CASE(192)
    KFBI_CASE(256) KFBI_CASE(384) KFBI_CASE(512) KFBI_CASE(768) KFBI_CASE(1024)
    KFBI_CASE(1536) KFBI_CASE(2048) KFBI_CASE(3072) KFBI_CASE(4096) KFBI_CASE(6144)
    KFBI_CASE(8192)
#undef KFBI_CASE
  }
  set_error("row pass: no compiled plan for N = %d", c.N);
  return KFBI_ERR_UNSUPPORTED;
}

template <typename T>
kfbi_status autotune_dispatch(Ctx& c, T* scratch, const cx<T>* tw, const T* lam) {
  int* rc = &c.rows_variant[sizeof(T) == 8];
  int* cc = &c.cols_variant[sizeof(T) == 8];
  switch (c.N) {
#define KFBI_CASE(n) \
  case n: return autotune<T, n>(c, scratch, tw, lam, rc, cc);
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
