// One application of the layer potential (Alg. 1 steps 4-6) and the interface solves
// built from the same stages:
//   correction     b_p = F~_p + sum over crossed arms of sigma/h^2 (Taylor jump) (Alg. 2)
//   box solve      (Lap_h - kappa^2) v = b, v = 0 on the box boundary            (Alg. 4)
//   interpolation  v^+(z_k) = sum_p w_p v_p + jump Taylor terms                  (Alg. 3)
// The correction is a gather over the compacted irregular-node list with precomputed
// FP64 weights (one thread per irregular node, consecutive nodes per warp).  For the
// double-layer apply the right-hand side is nonzero only at irregular nodes, so only
// those entries of a persistent zero grid are written.
//
// Precisions of the box solve:
//   FP64                 FP64 sine transforms.
//   FP32                 FP32 sine transforms.
//   FP32 refined (1/2)   c1 = FP32 solve of b, then one or two corrections
//                        c_{k+1} = FP32 solve of r_k = b - (Lap_h - kappa^2)(c1 + ... + c_k);
//                        v = c1 + c2 (+ c3) summed in FP64 where it is read.  The residual
//                        is formed in double-single arithmetic: the iterate is the exact
//                        sum of FP32 values, the 5-point sum uses error-free TwoSum steps
//                        and an FMA-exact product with 1/h^2, and b is held as an exact
//                        FP32 pair (hi, lo) - FP32 instructions only, because FP64
//                        throughput on GB300 is 1/64 of FP32.  Where b is sparse (double
//                        layer) the irregular nodes are recomputed in FP64.
#include "fpbits.cuh"
#include "kfbi_internal.cuh"

namespace kfbi {

__device__ __forceinline__ int wrap(int k, int M) { return k < 0 ? k + M : (k >= M ? k - M : k); }

// ------------------------------------------------------------------ correction
// b[irr_node[k]] = (add ? b : 0) + sum_arms sum_r (wD dens + wS psi + wF f); with Blo the
// right-hand side is the FP32 pair (B, Blo): the sum is formed in FP64 from the pair and
// split into a pair again
template <typename T>
__global__ void correction_kernel(int nirr, int M, const int* __restrict__ irr_node,
                                  const int* __restrict__ arm_ptr, const int* __restrict__ arm_seg,
                                  const double* __restrict__ wD, const double* __restrict__ wS,
                                  const double* __restrict__ wF, const double* __restrict__ dens,
                                  const double* __restrict__ psi, const double* __restrict__ fctl,
                                  T* __restrict__ B, int add, double* __restrict__ B64,
                                  float* __restrict__ Blo) {
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
  if (Blo) {
    const double v = (add ? (double)B[node] + (double)Blo[node] : 0.0) + acc;
    const T h = (T)v;
    B[node] = h;
    Blo[node] = (float)(v - (double)h);
  } else {
    B[node] = add ? (T)((double)B[node] + acc) : (T)acc;
  }
  if (B64) B64[node] = acc;        // FP64 copy for the refinement residual
}

// dense right-hand side as an FP32 pair (hi, lo = FP32 of the FP64 remainder): F at inside
// interior nodes, 0 elsewhere
__global__ void rhs_pair_kernel(int N, const double* __restrict__ F,
                                const uint8_t* __restrict__ inside, float* __restrict__ hi,
                                float* __restrict__ lo) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const long idx = (long)j * N + i;
    double v = 0.0;
    if (F && i > 0 && j > 0) {
      const long g = (long)j * (N + 1) + i;
      if (inside[g]) v = F[g];
    }
    float h, l;
    f64_to_f32_pair(v, h, l);                    // integer operations, not the FP64 pipe
    hi[idx] = h;
    lo[idx] = l;
  }
}

// ------------------------------------------------------------------ double-single residual
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// value of the iterate at work-grid index q: c1 (+ c2) as an unevaluated pair
struct DSPair {
  float hi, lo;
};
__device__ __forceinline__ DSPair iterate_at(const float* c1, const float* c2, long q) {
  if (!c2) return {c1[q], 0.f};
  DSPair p;
  two_sum(c1[q], c2[q], p.hi, p.lo);
  return p;
}

// r = b - (Lap_h - kappa^2) v, v = c1 (+ c2), b = bhi + blo (dense) or 0 (bhi == nullptr);
// kappa^2 = k2hi + k2lo exactly.  Every product and sum that can cancel is carried as an
// exact FP32 pair; only the final residual is rounded to FP32.
// Four consecutive points of a row per thread (N a multiple of 4): the row and the rows
// above and below as 16-byte loads, the two outer neighbours as scalars.
__device__ __forceinline__ float ds_point(float inv_h2, float k2hi, float k2lo, DSPair vc,
                                          DSPair ve, DSPair vw, DSPair vn, DSPair vs,
                                          const float* bhi, const float* blo, int idx) {
  float s1, t1, s2, t2, s3, t3, s4, t4;
  two_sum(ve.hi, vw.hi, s1, t1);
  two_sum(vn.hi, vs.hi, s2, t2);
  two_sum(s1, s2, s3, t3);
  two_sum(s3, -4.f * vc.hi, s4, t4);
  const float lo = ((t1 + t2) + (t3 + t4)) + ((ve.lo + vw.lo) + (vn.lo + vs.lo) - 4.f * vc.lo);
  const float p1 = s4 * inv_h2;
  const float e1 = fmaf(s4, inv_h2, -p1) + lo * inv_h2;
  const float p2 = k2hi * vc.hi;
  const float e2 = fmaf(k2hi, vc.hi, -p2) + (k2hi * vc.lo + k2lo * vc.hi);
  float d, de;
  two_sum(p2, -p1, d, de);
  float tail = de - e1 + e2;
  if (bhi) {
    float d2, de2;
    two_sum(bhi[idx], d, d2, de2);
    d = d2;
    tail += de2 + blo[idx];
  }
  return d + tail;
}

__device__ __forceinline__ void ds_row4(const float* c1, const float* c2, int q, DSPair (&v)[4]) {
  const float4 a = *reinterpret_cast<const float4*>(c1 + q);
  if (!c2) {
    v[0] = {a.x, 0.f};
    v[1] = {a.y, 0.f};
    v[2] = {a.z, 0.f};
    v[3] = {a.w, 0.f};
    return;
  }
  const float4 b = *reinterpret_cast<const float4*>(c2 + q);
  two_sum(a.x, b.x, v[0].hi, v[0].lo);
  two_sum(a.y, b.y, v[1].hi, v[1].lo);
  two_sum(a.z, b.z, v[2].hi, v[2].lo);
  two_sum(a.w, b.w, v[3].hi, v[3].lo);
}

__global__ void ds_residual4_kernel(int N, float inv_h2, float k2hi, float k2lo,
                                    const float* __restrict__ bhi, const float* __restrict__ blo,
                                    const float* __restrict__ c1, const float* __restrict__ c2,
                                    float* __restrict__ r) {
  const int j = blockIdx.y;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= N) return;
  const int base = j * N + i0;
  float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
  if (j > 0) {
    DSPair c[4], n[4], so[4];
    ds_row4(c1, c2, base, c);
    ds_row4(c1, c2, base - N, so);
    if (j + 1 < N) {
      ds_row4(c1, c2, base + N, n);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u) n[u] = {0.f, 0.f};
    }
    const DSPair w0 = i0 > 0 ? iterate_at(c1, c2, base - 1) : DSPair{0.f, 0.f};
    const DSPair e3 = i0 + 4 < N ? iterate_at(c1, c2, base + 4) : DSPair{0.f, 0.f};
    float o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const DSPair vw = u == 0 ? w0 : c[u > 0 ? u - 1 : 0];
      const DSPair ve = u == 3 ? e3 : c[u < 3 ? u + 1 : 3];
      o[u] = (i0 + u == 0) ? 0.f
                           : ds_point(inv_h2, k2hi, k2lo, c[u], ve, vw, n[u], so[u], bhi, blo, base + u);
    }
    res = make_float4(o[0], o[1], o[2], o[3]);
  }
  *reinterpret_cast<float4*>(r + base) = res;
}

// r = b - (Lap_h - kappa^2)(c1 + c2) at the irregular nodes, in FP64 (sparse b)
__global__ void residual_fix_kernel(int nirr, int N, double inv_h2, double kappa2,
                                    const int* __restrict__ irr_node, const double* __restrict__ b,
                                    const float* __restrict__ c1, const float* __restrict__ c2,
                                    float* __restrict__ r) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nirr) return;
  const int idx = irr_node[k];
  const int i = idx % N, j = idx / N;
  auto v = [&](int q) { return (double)c1[q] + (c2 ? (double)c2[q] : 0.0); };
  const double s = (i + 1 < N ? v(idx + 1) : 0.0) + v(idx - 1) +
                   (j + 1 < N ? v(idx + N) : 0.0) + v(idx - N);
  const double vc = v(idx);
  r[idx] = (float)(b[idx] - ((s - 4.0 * vc) * inv_h2 - kappa2 * vc));
}

// dense FP64 right-hand side -> exact FP32 pair (hi, lo)
__global__ void split_kernel(long n, const double* __restrict__ b, float* __restrict__ hi,
                             float* __restrict__ lo) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
       k += (long)gridDim.x * blockDim.x) {
    float h, l;
    f64_to_f32_pair(b[k], h, l);                 // integer operations, not the FP64 pipe
    hi[k] = h;
    lo[k] = l;
  }
}

// ------------------------------------------------------------------ sparse plain apply
// The double- (single-) layer right-hand side is nonzero only at irregular nodes, so the
// plain FP32 apply fuses the correction gather (Alg. 2) with the first sine transform
// (along x, Alg. 4) and writes the transformed rows straight into the work grid:
//   X[j][k] = sum over irregular (i, j) of b_ij sin(pi i k / N).
// One CTA per work item: a grid row j, or a part of the nodes of a row with many (T threads
// in W = T/32 warps).  Warp w prepares the item's nodes q = w, w + W, ...: lanes over
// (crossed arm, weight) pairs form b_ij from the density (up to 4 x 6 FP64 products
// gathered at once, summed by shuffles; the FP64 value also goes to B64 at the node when
// a refined apply needs it for its residuals), and the node's phase
// tables go to shared memory: e^{i pi i l / N} for the lanes l < 32, e^{i pi i 32 v / N}
// for the warps v < W, and the rotation e^{i pi i T / N}.  Then thread t = 32 v + l
// accumulates the modes k = t + s T (s < S, k < N/4), starting from the product of its
// lane and warp factors and advancing by the rotation, and by the symmetries of the sine
// with theta = pi i k / N,
//   sin(pi i (N - k) / N)    = (-1)^(i+1) sin theta,
//   sin(pi i (N/2 +- k) / N) = sin(pi i / 2 +- theta) = +-sin theta or cos theta by i mod 4,
// the modes N - k, N/2 + k and N/2 - k as well.  Modes N/4 and 3N/4 come from table
// values kept with the node.  Rows without irregular nodes are zero.  The parts of a split
// row write partial rows to scratch slots; the last part to arrive (a counter, reset by
// it) adds them in part order into the row, so the result does not depend on scheduling.
constexpr int SPX_THREADS_MAX = 256;
constexpr int SPX_NODES = 32;          // irregular nodes of a row held in shared memory at once

// x mod 2N for 0 <= x < 2^31 with x / 2N < 2^20 (the float quotient is then off by at most
// one, corrected by one step either way)
__device__ __forceinline__ int mod_2n(int x, int n2, float inv_n2) {
  int r = x - n2 * (int)((float)x * inv_n2);
  r += r < 0 ? n2 : 0;
  r -= r >= n2 ? n2 : 0;
  return r;
}

template <int S>
__global__ void __launch_bounds__(SPX_THREADS_MAX)
    sparse_rows_kernel(int N, int M, const int4* __restrict__ items,
                       const int* __restrict__ irr_node, const int* __restrict__ arm_ptr,
                       const int* __restrict__ arm_seg, const double* __restrict__ wgt,
                       const double* __restrict__ dens, const float2* __restrict__ tw,
                       float* __restrict__ X, float* part, unsigned* counter,
                       double* __restrict__ B64) {
  constexpr int WMAX = SPX_THREADS_MAX / 32;
  __shared__ float2 s_lane[SPX_NODES][32];
  __shared__ float2 s_warp[SPX_NODES][WMAX];
  __shared__ float4 s_node[SPX_NODES];   // (b, rotation cos, rotation sin, i as bits)
  __shared__ float2 s_q[SPX_NODES];      // sin(pi i / 4), sin(3 pi i / 4)
  __shared__ bool s_last;
  const int t = threadIdx.x, T = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarps = T >> 5;
  const int Q = N / 4, H = N / 2, N2 = 2 * N;
  const float inv_n2 = 1.f / (float)N2;
  // item: (row, first node, end node, part), (parts, first scratch slot, counter, 0)
  const int4 ia = items[2 * blockIdx.x], ib = items[2 * blockIdx.x + 1];
  const int j = ia.x, n0 = ia.y, n1 = ia.z, nparts = ib.x;
  float* row = nparts == 1 ? X + (size_t)j * N : part + (size_t)(ib.y + ia.w) * N;
  if (n1 == n0) {                                     // no irregular node: the row is zero
    for (int k = 4 * t; k < N; k += 4 * T) *reinterpret_cast<float4*>(row + k) = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  float a1[S], a2[S], a3[S], a4[S];
#pragma unroll
  for (int s = 0; s < S; ++s) a1[s] = a2[s] = a3[s] = a4[s] = 0.f;
  float aq = 0.f, a3q = 0.f;                          // modes N/4, 3N/4 (thread 0)
  for (int base = n0; base < n1; base += SPX_NODES) {
    const int cnt = min(SPX_NODES, n1 - base);
    __syncthreads();                                  // previous batch consumed
    for (int q = warp; q < cnt; q += nwarps) {
      const int n = base + q;
      const int a0 = arm_ptr[n], na = arm_ptr[n + 1] - a0;
      const int i = irr_node[n] - j * N;
      const int a = lane / 6, r = lane - 6 * (lane / 6);
      double v = 0.0;
      if (lane < 24 && a < na)
        v = wgt[6 * (a0 + a) + r] * dens[wrap(arm_seg[a0 + a] - 2 + r, M)];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const float2 pl = tw[mod_2n(i * lane, N2, inv_n2)];
      s_lane[q][lane] = make_float2(pl.x, -pl.y);
      if (lane < nwarps) {
        const float2 pw = tw[mod_2n(i * 32 * lane, N2, inv_n2)];
        s_warp[q][lane] = make_float2(pw.x, -pw.y);
      }
      if (lane == 0) {
        if (B64) B64[j * N + i] = v;
        const float2 rt = tw[mod_2n(i * T, N2, inv_n2)];
        s_node[q] = make_float4((float)v, rt.x, -rt.y, __int_as_float(i));
        s_q[q] = make_float2(-tw[mod_2n(i * Q, N2, inv_n2)].y, -tw[mod_2n(i * 3 * Q, N2, inv_n2)].y);
      }
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const float4 nd = s_node[q];
      const int i = __float_as_int(nd.w);
      const float b = nd.x;
      const float2 pl = s_lane[q][lane], pw = s_warp[q][warp];
      float cs = pl.x * pw.x - pl.y * pw.y;           // e^{i pi i t / N}, t = 32 warp + lane
      float sn = fmaf(pl.x, pw.y, pl.y * pw.x);
      const bool odd = i & 1;
      const float p2 = odd ? b : -b;                              // mode N - k
      const float p3 = ((i & 3) == 0 || (i & 3) == 1) ? b : -b;   // mode N/2 + k
      const float p4 = odd ? p3 : -p3;                            // mode N/2 - k
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const float tt = odd ? cs : sn;
        a1[s] = fmaf(b, sn, a1[s]);
        a2[s] = fmaf(p2, sn, a2[s]);
        a3[s] = fmaf(p3, tt, a3[s]);
        a4[s] = fmaf(p4, tt, a4[s]);
        if (s + 1 < S) {
          const float cn = cs * nd.y - sn * nd.z;
          sn = fmaf(sn, nd.y, cs * nd.z);
          cs = cn;
        }
      }
      if (t == 0) {
        aq = fmaf(b, s_q[q].x, aq);
        a3q = fmaf(b, s_q[q].y, a3q);
      }
    }
  }
  // every mode written exactly once: k in [0, N/4) with N/2 + k, and N - k, N/2 - k for
  // 0 < k < N/4; then N/4 and 3N/4 (X[0] = 0)
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int k = t + s * T;
    if (k >= Q) break;
    row[k] = (k == 0) ? 0.f : a1[s];
    row[H + k] = a3[s];
    if (k > 0) {
      row[N - k] = a2[s];
      row[H - k] = a4[s];
    }
  }
  if (t == 0) {
    row[Q] = aq;
    row[3 * Q] = a3q;
  }
  if (nparts == 1) return;                            // uniform over the CTA
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(counter + ib.z, 1u) == (unsigned)(nparts - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const float4* src = reinterpret_cast<const float4*>(part + (size_t)ib.y * N);
  float4* dst = reinterpret_cast<float4*>(X + (size_t)j * N);
  for (int e = t; e < Q; e += T) {                    // N / 4 float4 per row
    float4 v = __ldcg(src + e);
    for (int p = 1; p < nparts; ++p) {
      const float4 u = __ldcg(src + (size_t)p * Q + e);
      v.x += u.x;
      v.y += u.y;
      v.z += u.z;
      v.w += u.w;
    }
    dst[e] = v;
  }
  if (t == 0) counter[ib.z] = 0u;
}

// ------------------------------------------------------------------ sparse-output x-transform
// The plain apply's interpolation reads the grid only at the control points' stencil nodes
// (a few per grid row near Gamma), so its last sine transform along x is evaluated there
// only:  v[j][i] = sum_k Y[j][k] sin(pi i k / N)  for the listed nodes (i, j).  One CTA per
// work item (a row's nodes, or a part of them: a few each, longest items first); thread
// t = 32 w + l of T takes the modes k = 1 + t + T s (s < S, k < N/4) and, by the symmetries
// used in sparse_rows_kernel, the modes N - k, N/2 + k and N/2 - k with the same (cos, sin)
// of theta = pi i k / N:
//   v = sum_k sin(theta) A_k + cos(theta) B_k,
//   i = 0 mod 4: A = (Y_k - Y_{N-k}) + (Y_{N/2+k} - Y_{N/2-k}),  B = 0
//   i = 1 mod 4: A = Y_k + Y_{N-k},  B = Y_{N/2+k} + Y_{N/2-k}
//   i = 2 mod 4: A = (Y_k - Y_{N-k}) - (Y_{N/2+k} - Y_{N/2-k}),  B = 0
//   i = 3 mod 4: A = Y_k + Y_{N-k},  B = -(Y_{N/2+k} + Y_{N/2-k})
// plus the modes N/2 (sin(pi i / 2)), N/4 and 3N/4 (sin(pi i / 4), sin(3 pi i / 4)).  The
// phase of thread t starts at the product of per-node lane and warp factors
// e^{i pi i (1 + l) / N} e^{i pi i 32 w / N} kept in shared memory, advances by the rotation
// e^{i pi i T / N} and is re-seeded every 4 steps from e^{i pi i 4 T r / N} (no long rotation
// chains); the warp sums of each node go through shared memory to one total.
constexpr int SPO_T = 128;
constexpr int SPO_NODES = 32;              // nodes of an item per batch

template <int S>
__global__ void __launch_bounds__(SPO_T)
    sparse_out_kernel(int N, const float* __restrict__ Y, const int4* __restrict__ items,
                      const int* __restrict__ col, const float2* __restrict__ tw,
                      float* __restrict__ out) {
  constexpr int WMAX = SPO_T / 32, RS = (S + 3) / 4;
  __shared__ float2 s_lane[SPO_NODES][32];
  __shared__ float2 s_warp[SPO_NODES][WMAX];
  __shared__ float2 s_seed[SPO_NODES][RS];
  __shared__ float2 s_rot[SPO_NODES];
  __shared__ float s_part[SPO_NODES][WMAX];
  __shared__ int s_col[SPO_NODES];
  const int t = threadIdx.x, T = blockDim.x;
  const int lane = t & 31, warp = t >> 5, nwarps = T >> 5;
  const int Q = N / 4, H = N / 2, N2 = 2 * N;
  const float inv_n2 = 1.f / (float)N2;
  const int4 item = items[blockIdx.x];                 // (row, first node, end node, 0)
  const int j = item.x, n0 = item.y, n1 = item.z;
  const float* row = Y + (size_t)j * N;
  // the thread's mode combinations: sums and differences of the four symmetric modes
  float a12[S], d12[S], a34[S], d34[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int k = 1 + t + s * T;
    float y1 = 0.f, y2 = 0.f, y3 = 0.f, y4 = 0.f;
    if (k < Q) {
      y1 = row[k];
      y2 = row[N - k];
      y3 = row[H + k];
      y4 = row[H - k];
    }
    a12[s] = y1 + y2;
    d12[s] = y1 - y2;
    a34[s] = y3 + y4;
    d34[s] = y3 - y4;
  }
  const float yh = row[H], yq = row[Q], y3q = row[3 * Q];
  for (int base = n0; base < n1; base += SPO_NODES) {
    const int cnt = min(SPO_NODES, n1 - base);
    __syncthreads();                                   // previous batch's tables consumed
    for (int q = warp; q < cnt; q += nwarps) {         // per-node phase tables
      const int i = col[base + q];
      const float2 pl = tw[mod_2n(i * (1 + lane), N2, inv_n2)];
      s_lane[q][lane] = make_float2(pl.x, -pl.y);
      if (lane < nwarps) {
        const float2 pw = tw[mod_2n(i * 32 * lane, N2, inv_n2)];
        s_warp[q][lane] = make_float2(pw.x, -pw.y);
      }
      if (lane < RS) {
        const float2 ps = tw[mod_2n(i * 4 * T * lane, N2, inv_n2)];
        s_seed[q][lane] = make_float2(ps.x, -ps.y);
      }
      if (lane == 0) {
        const float2 pr = tw[mod_2n(i * T, N2, inv_n2)];
        s_rot[q] = make_float2(pr.x, -pr.y);
        s_col[q] = i;
      }
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const int i = s_col[q];
      const int cls = i & 3;
      const float2 pl = s_lane[q][lane], pw = s_warp[q][warp], rot = s_rot[q];
      const float c0 = pl.x * pw.x - pl.y * pw.y;      // e^{i pi i (1 + t) / N}
      const float s0 = fmaf(pl.x, pw.y, pl.y * pw.x);
      float cs = c0, sn = s0, acc = 0.f;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        if (s > 0 && (s & 3) == 0) {                   // re-seed from the table
          const float2 sd = s_seed[q][s >> 2];
          cs = c0 * sd.x - s0 * sd.y;
          sn = fmaf(c0, sd.y, s0 * sd.x);
        }
        const float A = (cls & 1) ? a12[s] : (cls == 0 ? d12[s] + d34[s] : d12[s] - d34[s]);
        const float B = (cls & 1) ? (cls == 1 ? a34[s] : -a34[s]) : 0.f;
        acc = fmaf(sn, A, fmaf(cs, B, acc));
        const float cn = cs * rot.x - sn * rot.y;
        sn = fmaf(sn, rot.x, cs * rot.y);
        cs = cn;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) s_part[q][warp] = acc;
    }
    __syncthreads();
    for (int q = t; q < cnt; q += T) {                 // totals and the special modes
      const int i = s_col[q];
      float v = 0.f;
      for (int w = 0; w < nwarps; ++w) v += s_part[q][w];
      const float sh = (i & 1) ? ((i & 3) == 1 ? 1.f : -1.f) : 0.f;     // sin(pi i / 2)
      v = fmaf(yh, sh, v);
      v = fmaf(yq, -tw[mod_2n(i * Q, N2, inv_n2)].y, v);
      v = fmaf(y3q, -tw[mod_2n(i * 3 * Q, N2, inv_n2)].y, v);
      out[base + q] = v;
    }
  }
}

template <int S>
static void launch_sparse_out(Ctx& c, int T, const float* Y) {
  sparse_out_kernel<S><<<c.sn_nitems, T, 0, c.stream>>>(
      c.N, Y, reinterpret_cast<const int4*>(c.sn_items), c.sn_col,
      reinterpret_cast<const float2*>(c.t32.tw), c.sn_val);
}

// threads per item: the N/4 - 1 modes rounded up to a warp, at most 128; S steps each
static kfbi_status sparse_out(Ctx& c, const float* Y) {
  if (c.sn_nitems == 0) return KFBI_OK;
  const int Q = c.N / 4;
  const int T = Q - 1 >= SPO_T ? SPO_T : ((Q - 1 + 31) / 32) * 32;
  const int S = (Q - 1 + T - 1) / T;
  const int pr = prof_begin(c, ST_ROWS32);
  switch (S) {
    case 1: launch_sparse_out<1>(c, T, Y); break;
    case 2: launch_sparse_out<2>(c, T, Y); break;
    case 3: launch_sparse_out<3>(c, T, Y); break;
    case 4: launch_sparse_out<4>(c, T, Y); break;
    case 6: launch_sparse_out<6>(c, T, Y); break;
    case 8: launch_sparse_out<8>(c, T, Y); break;
    case 12: launch_sparse_out<12>(c, T, Y); break;
    case 16: launch_sparse_out<16>(c, T, Y); break;
    default:
      prof_end(c, pr);
      set_error("sparse-output x-transform: N = %d not supported", c.N);
      return KFBI_ERR_UNSUPPORTED;
  }
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <int S>
static void launch_sparse_rows(Ctx& c, int T, const double* wgt, const double* dens, float* X,
                               double* B64) {
  sparse_rows_kernel<S><<<c.spx_nitems, T, 0, c.stream>>>(
      c.N, c.M, reinterpret_cast<const int4*>(c.spx_items), c.irr_node, c.arm_ptr, c.arm_seg,
      wgt, dens, reinterpret_cast<const float2*>(c.t32.tw), X, c.spx_part, c.spx_cnt, B64);
}

// threads per item: N/4 rounded up to a warp, at most 256; S = ceil(N/4 / T) steps
// (B64: also the FP64 right-hand side at the irregular nodes, for refinement residuals)
static kfbi_status sparse_rows(Ctx& c, const double* wgt, const double* dens, float* X,
                               double* B64 = nullptr) {
  const int Q = c.N / 4;
  const int T = Q >= SPX_THREADS_MAX ? SPX_THREADS_MAX : ((Q + 31) / 32) * 32;
  const int S = (Q + T - 1) / T;
  const int pr = prof_begin(c, ST_SPARSE);
  switch (S) {
    case 1: launch_sparse_rows<1>(c, T, wgt, dens, X, B64); break;
    case 2: launch_sparse_rows<2>(c, T, wgt, dens, X, B64); break;
    case 3: launch_sparse_rows<3>(c, T, wgt, dens, X, B64); break;
    case 4: launch_sparse_rows<4>(c, T, wgt, dens, X, B64); break;
    case 6: launch_sparse_rows<6>(c, T, wgt, dens, X, B64); break;
    case 8: launch_sparse_rows<8>(c, T, wgt, dens, X, B64); break;
    default:
      prof_end(c, pr);
      set_error("sparse x-transform: N = %d not supported", c.N);
      return KFBI_ERR_UNSUPPORTED;
  }
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

// ------------------------------------------------------------------ grid kernels
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

__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }   // exact, integer ops

// work grid(s) -> (N+1)^2 FP64 grid: value w1 (+ w2 + w3); mask keeps inside nodes only.
// Each thread takes W2G_U nodes of its row, W2G_U apart (independent loads in flight).
constexpr int W2G_U = 4;
template <typename T>
__global__ void work_to_grid_kernel(int N, const T* __restrict__ w1, const float* __restrict__ w2,
                                    const float* __restrict__ w3, const uint8_t* __restrict__ mask,
                                    double* __restrict__ G) {
  const int j = blockIdx.y;
  const int stride = gridDim.x * blockDim.x;
  for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 <= N; i0 += W2G_U * stride) {
    double v[W2G_U];
#pragma unroll
    for (int u = 0; u < W2G_U; ++u) {
      const int i = i0 + u * stride;
      v[u] = 0.0;
      if (i < N && j < N) {
        const long q = (long)j * N + i;
        v[u] = to_f64(w1[q]);
        if (w2) v[u] += to_f64(w2[q]);
        if (w3) v[u] += to_f64(w3[q]);
      }
    }
#pragma unroll
    for (int u = 0; u < W2G_U; ++u) {
      const int i = i0 + u * stride;
      if (i > N) break;
      const long g = (long)j * (N + 1) + i;
      G[g] = (mask && !mask[g]) ? 0.0 : v[u];
    }
  }
}

// ------------------------------------------------------------------ interpolation
// out_k = sum_p w_p v(node_p) + sum_r (cD dens + cS psi) + eF f_k, v = v1 (+ v2 + v3) at the
// work-grid node (each grid optional) plus vs at the node's slot in the compact list of
// stencil-node values (when given)
template <typename T>
__global__ void interp_kernel(int M, const int* __restrict__ node, const int* __restrict__ slot,
                              const double* __restrict__ w,
                              const double* __restrict__ cD, const double* __restrict__ cS,
                              const double* __restrict__ eF, const T* __restrict__ v1,
                              const float* __restrict__ v2, const float* __restrict__ v3,
                              const float* __restrict__ vs,
                              const double* __restrict__ dens, const double* __restrict__ psi,
                              const double* __restrict__ fctl, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  double acc = 0.0;
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int nd = node[6 * k + p];
    if (nd >= 0) {
      double v = v1 ? (double)v1[nd] : 0.0;
      if (v2) v += (double)v2[nd];
      if (v3) v += (double)v3[nd];
      if (vs) v += (double)vs[slot[6 * k + p]];
      acc += w[6 * k + p] * v;
    }
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

// ------------------------------------------------------------------ host helpers
static inline dim3 rows_grid(int cols, int rows) {
  const int bx = (cols + 255) / 256;
  return dim3((unsigned)(bx < 8 ? bx : 8), (unsigned)rows);
}

static inline int gs_blocks(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

template <typename T>
static kfbi_status correct(Ctx& c, const double* dens, const double* psi, const double* fctl,
                           T* B, int add, double* B64 = nullptr, float* Blo = nullptr) {
  if (c.nirr == 0) return KFBI_OK;
  const int pr = prof_begin(c, ST_CORR);
  correction_kernel<T><<<(c.nirr + 127) / 128, 128, 0, c.stream>>>(
      c.nirr, c.M, c.irr_node, c.arm_ptr, c.arm_seg, c.arm_wD, c.arm_wS, c.arm_wF, dens, psi,
      fctl, B, add, B64, Blo);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

// v^+ at the control points, or with dn the normal derivative d_n v^+ (the same gather with
// the weights of n . grad of the fitted quadratic); v = v1 (+ v2 + v3) on the work grid plus
// vs, the compact values at the stencil nodes left by the sparse-output transform
template <typename T>
static kfbi_status interp(Ctx& c, const T* v1, const float* v2, const float* v3,
                          const double* dens, const double* psi, const double* fctl,
                          double* out, bool dn = false, const float* vs = nullptr) {
  const int pr = prof_begin(c, ST_INTERP);
  interp_kernel<T><<<(c.M + 127) / 128, 128, 0, c.stream>>>(
      c.M, c.ctrl_node, c.ctrl_slot, dn ? c.ctrl_wn : c.ctrl_w, dn ? c.ctrl_cDn : c.ctrl_cD,
      dn ? c.ctrl_cSn : c.ctrl_cS, dn ? c.ctrl_eFn : c.ctrl_eF, v1, v2, v3, vs, dens, psi, fctl,
      out);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T>
static kfbi_status to_grid(Ctx& c, const T* w1, const float* w2, const float* w3,
                           const uint8_t* mask, double* G) {
  prof_count(c, ST_GRID);
  work_to_grid_kernel<T><<<rows_grid(c.N + 1, c.N + 1), 256, 0, c.stream>>>(c.N, w1, w2, w3,
                                                                              mask, G);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

static int refine_steps_of(int precision) {
  return precision == KFBI_FP32_REFINED ? 2 : (precision == KFBI_FP32_REFINED_ONCE ? 1 : 0);
}

// Refinement steps of an FP32 box solve whose first solution is in V32: the residuals use
// the dense exact pair (bhi, blo) or, when bhi is null, the sparse FP64 right-hand side in
// B64 at the irregular nodes (zero elsewhere).  Result: v = V32 + U32 (+ T32 if steps = 2);
// with stencil_last the last correction is evaluated at the control points' stencil nodes
// only (its last x-transform by the sparse-output kernel, into sn_val) instead.
static kfbi_status refine_steps(Ctx& c, const float* bhi, const float* blo, int steps,
                                bool stencil_last) {
  const float inv_h2 = (float)(1.0 / (c.h * c.h));
  const float k2hi = (float)c.kappa2, k2lo = (float)(c.kappa2 - (double)k2hi);
  for (int s = 0; s < steps; ++s) {
    const float* c2 = s == 0 ? nullptr : c.U32;      // current iterate = V32 (+ U32)
    const int pr = prof_begin(c, ST_REFINE);
    ds_residual4_kernel<<<dim3((c.N / 4 + 255) / 256, c.N), 256, 0, c.stream>>>(
        c.N, inv_h2, k2hi, k2lo, bhi, blo, c.V32, c2, c.W32);
    if (!bhi && c.nirr > 0)
      residual_fix_kernel<<<(c.nirr + 127) / 128, 128, 0, c.stream>>>(
          c.nirr, c.N, 1.0 / (c.h * c.h), c.kappa2, c.irr_node, c.B64, c.V32, c2, c.W32);
    prof_end(c, pr);
    if (!bhi && c.nirr > 0) prof_count(c, ST_REFINE);
    KFBI_CUDA_TRY(cudaGetLastError());
    float* corr = s == 0 ? c.U32 : c.T32;
    if (stencil_last && s == steps - 1) {
      KFBI_TRY(rows_pass_f32(c, c.W32, corr));
      KFBI_TRY(ypass_rows_f32(c, corr, ypass_out(c)));
      KFBI_TRY(sparse_out(c, ypass_out(c)));
    } else {
      KFBI_TRY(box_solve_f32(c, c.W32, corr));
    }
  }
  return KFBI_OK;
}

// Refined FP32 box solve of the FP32 right-hand side b32 (first solve into V32, then the
// refinement steps above with full-grid corrections)
static kfbi_status refined_solve(Ctx& c, const float* b32, const float* bhi, const float* blo,
                                 int steps) {
  KFBI_TRY(box_solve_f32(c, b32, c.V32));
  return refine_steps(c, bhi, blo, steps, false);
}

// ------------------------------------------------------------------ apply
kfbi_status apply_potential(Ctx& c, Layer layer, int precision, const double* dens, double* out,
                            bool dn) {
  if (c.dim == 3) {
    if (dn) {
      set_error("normal derivative of a layer potential: 2-D only");
      return KFBI_ERR_UNSUPPORTED;
    }
    return apply_potential3(c, layer, precision, dens, out);
  }
  const double* d = layer == Layer::Double ? dens : nullptr;
  const double* s = layer == Layer::Single ? dens : nullptr;
  if (precision == KFBI_FP64) {
    KFBI_TRY(correct<double>(c, d, s, nullptr, c.B64, 0));
    KFBI_TRY(box_solve_f64(c, c.B64, c.V64));
    return interp<double>(c, c.V64, nullptr, nullptr, d, s, nullptr, out, dn);
  }
  const int steps = refine_steps_of(precision);
  if (steps == 0 && precision != KFBI_TF32X3 && c.irr_rowptr && c.dim == 2) {
    // correction fused with the first x-transform (sparse right-hand side), then the rest
    // of the box solve on the transformed rows: with the row-layout y-pass the last
    // x-transform is evaluated at the stencil nodes only
    KFBI_TRY(sparse_rows(c, d ? c.arm_wD : c.arm_wS, d ? d : s, c.V32));
    if (c.cols_variant[0] & 8) {
      KFBI_TRY(ypass_rows_f32(c, c.V32, ypass_out(c)));
      KFBI_TRY(sparse_out(c, ypass_out(c)));
      return interp<float>(c, nullptr, nullptr, nullptr, d, s, nullptr, out, dn, c.sn_val);
    }
    KFBI_TRY(box_solve_after_rows_f32(c, c.V32));
    return interp<float>(c, c.V32, nullptr, nullptr, d, s, nullptr, out, dn);
  }
  if (steps > 0 && precision != KFBI_TF32X3 && c.irr_rowptr) {
    // refined: the first solve from the sparse right-hand side (correction fused with the
    // first x-transform, which also leaves the FP64 values for the residuals in B64); with
    // the row-layout y-pass the last correction is evaluated at the stencil nodes only
    KFBI_TRY(sparse_rows(c, d ? c.arm_wD : c.arm_wS, d ? d : s, c.V32, c.B64));
    KFBI_TRY(box_solve_after_rows_f32(c, c.V32));
    const bool stencil = (c.cols_variant[0] & 8) != 0;
    KFBI_TRY(refine_steps(c, nullptr, nullptr, steps, stencil));
    if (stencil)
      return interp<float>(c, c.V32, steps > 1 ? c.U32 : nullptr, nullptr, d, s, nullptr, out, dn,
                           c.sn_val);
    return interp<float>(c, c.V32, c.U32, steps > 1 ? c.T32 : nullptr, d, s, nullptr, out, dn);
  }
  KFBI_TRY(correct<float>(c, d, s, nullptr, c.B32, 0, steps ? c.B64 : nullptr));
  if (precision == KFBI_TF32X3) {                   // dense sine transforms on tensor cores
    KFBI_TRY(box_solve_tc(c, c.B32, c.V32));
    return interp<float>(c, c.V32, nullptr, nullptr, d, s, nullptr, out, dn);
  }
  if (steps == 0) {
    KFBI_TRY(box_solve_f32(c, c.B32, c.V32));
    return interp<float>(c, c.V32, nullptr, nullptr, d, s, nullptr, out, dn);
  }
  KFBI_TRY(refined_solve(c, c.B32, nullptr, nullptr, steps));
  return interp<float>(c, c.V32, c.U32, steps > 1 ? c.T32 : nullptr, d, s, nullptr, out, dn);
}

// ------------------------------------------------------------------ dense interface solves
// F~ + corrections in FP64 in V64 (work layout)
static kfbi_status dense_rhs64(Ctx& c, const double* dens, const double* f_grid,
                               const double* f_ctrl, const double* psi = nullptr) {
  prof_count(c, ST_GRID);
  rhs_dense_kernel<double><<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, f_grid, c.inside,
                                                                      c.V64);
  KFBI_CUDA_TRY(cudaGetLastError());
  return correct<double>(c, dens, psi, f_ctrl, c.V64, 1);
}

// F~ + corrections as an FP32 pair in (H32, D32), without the FP64 grid (the refined
// solves' right-hand side when no caller asks for the grid itself)
static kfbi_status dense_rhs_pair(Ctx& c, const double* dens, const double* f_grid,
                                  const double* f_ctrl, const double* psi = nullptr) {
  prof_count(c, ST_GRID);
  rhs_pair_kernel<<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, f_grid, c.inside, c.H32,
                                                             c.D32);
  KFBI_CUDA_TRY(cudaGetLastError());
  return correct<float>(c, dens, psi, f_ctrl, c.H32, 1, nullptr, c.D32);
}

// refined FP32 solve of the FP64 right-hand side in V64, split into an exact pair
static kfbi_status refined_dense(Ctx& c, int steps) {
  const long n = (long)c.N * c.N;
  prof_count(c, ST_GRID);
  split_kernel<<<gs_blocks(n), 256, 0, c.stream>>>(n, c.V64, c.H32, c.D32);
  KFBI_CUDA_TRY(cudaGetLastError());
  return refined_solve(c, c.H32, c.H32, c.D32, steps);
}

kfbi_status interface_solve(Ctx& c, int precision, const double* dens, const double* f_grid,
                            const double* f_ctrl, double* rhs_grid, double* v_grid,
                            double* out, const double* psi, bool dn) {
  if (c.dim == 3) {
    if (psi || dn) {
      set_error("interface solve with a single-layer density or a normal derivative: 2-D only");
      return KFBI_ERR_UNSUPPORTED;
    }
    return interface_solve3(c, precision, dens, f_grid, f_ctrl, rhs_grid, v_grid, out);
  }
  const int steps = refine_steps_of(precision);
  if (steps > 0 && !rhs_grid) {                     // refined, the right-hand side as a pair
    KFBI_TRY(dense_rhs_pair(c, dens, f_grid, f_ctrl, psi));
    KFBI_TRY(refined_solve(c, c.H32, c.H32, c.D32, steps));
    const float* v3 = steps > 1 ? c.T32 : nullptr;
    if (v_grid) KFBI_TRY(to_grid<float>(c, c.V32, c.U32, v3, nullptr, v_grid));
    if (out) KFBI_TRY(interp<float>(c, c.V32, c.U32, v3, dens, psi, f_ctrl, out, dn));
    return KFBI_OK;
  }
  if (precision == KFBI_FP64 || steps > 0) {
    KFBI_TRY(dense_rhs64(c, dens, f_grid, f_ctrl, psi));
    if (rhs_grid) KFBI_TRY(to_grid<double>(c, c.V64, nullptr, nullptr, nullptr, rhs_grid));
    if (precision == KFBI_FP64) {
      KFBI_TRY(box_solve_f64(c, c.V64, c.V64));
      if (v_grid) KFBI_TRY(to_grid<double>(c, c.V64, nullptr, nullptr, nullptr, v_grid));
      if (out) KFBI_TRY(interp<double>(c, c.V64, nullptr, nullptr, dens, psi, f_ctrl, out, dn));
      return KFBI_OK;
    }
    KFBI_TRY(refined_dense(c, steps));
    const float* v3 = steps > 1 ? c.T32 : nullptr;
    if (v_grid) KFBI_TRY(to_grid<float>(c, c.V32, c.U32, v3, nullptr, v_grid));
    if (out) KFBI_TRY(interp<float>(c, c.V32, c.U32, v3, dens, psi, f_ctrl, out, dn));
    return KFBI_OK;
  }
  // plain FP32
  float* W = c.V32;
  prof_count(c, ST_GRID);
  rhs_dense_kernel<float><<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, f_grid, c.inside, W);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_TRY(correct<float>(c, dens, psi, f_ctrl, W, 1));
  if (rhs_grid) KFBI_TRY(to_grid<float>(c, W, nullptr, nullptr, nullptr, rhs_grid));
  if (precision == KFBI_TF32X3) KFBI_TRY(box_solve_tc(c, W, W));
  else KFBI_TRY(box_solve_f32(c, W, W));
  if (v_grid) KFBI_TRY(to_grid<float>(c, W, nullptr, nullptr, nullptr, v_grid));
  if (out) KFBI_TRY(interp<float>(c, W, nullptr, nullptr, dens, psi, f_ctrl, out, dn));
  return KFBI_OK;
}

// u on the grid: inside nodes of the combined solve (Phi = phi, F = f~), zero elsewhere
kfbi_status combined_u(Ctx& c, int precision, const double* dens, const double* f_grid,
                       const double* f_ctrl, double* u_grid, const double* psi) {
  if (c.dim == 3) {
    if (psi) {
      set_error("grid solution with a single-layer density: 2-D only");
      return KFBI_ERR_UNSUPPORTED;
    }
    return combined_u3(c, precision, dens, f_grid, f_ctrl, u_grid);
  }
  if (precision == KFBI_FP64) {
    KFBI_TRY(dense_rhs64(c, dens, f_grid, f_ctrl, psi));
    KFBI_TRY(box_solve_f64(c, c.V64, c.V64));
    return to_grid<double>(c, c.V64, nullptr, nullptr, c.inside, u_grid);
  }
  const int steps = refine_steps_of(precision) > 0 ? refine_steps_of(precision) : 1;
  KFBI_TRY(dense_rhs_pair(c, dens, f_grid, f_ctrl, psi));
  KFBI_TRY(refined_solve(c, c.H32, c.H32, c.D32, steps));
  return to_grid<float>(c, c.V32, c.U32, steps > 1 ? c.T32 : nullptr, c.inside, u_grid);
}

kfbi_status box_solve_grid(Ctx& c, int precision, const double* b_grid, double* v_grid) {
  if (c.dim == 3) return box_solve_grid3(c, precision, b_grid, v_grid);
  const int steps = refine_steps_of(precision);
  if (precision == KFBI_FP64 || steps > 0) {
    prof_count(c, ST_GRID);
    grid_to_work_kernel<double><<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, b_grid, c.V64);
    KFBI_CUDA_TRY(cudaGetLastError());
    if (precision == KFBI_FP64) {
      KFBI_TRY(box_solve_f64(c, c.V64, c.V64));
      return to_grid<double>(c, c.V64, nullptr, nullptr, nullptr, v_grid);
    }
    KFBI_TRY(refined_dense(c, steps));
    return to_grid<float>(c, c.V32, c.U32, steps > 1 ? c.T32 : nullptr, nullptr, v_grid);
  }
  prof_count(c, ST_GRID);
  grid_to_work_kernel<float><<<rows_grid(c.N, c.N), 256, 0, c.stream>>>(c.N, b_grid, c.V32);
  KFBI_CUDA_TRY(cudaGetLastError());
  if (precision == KFBI_TF32X3) KFBI_TRY(box_solve_tc(c, c.V32, c.V32));
  else KFBI_TRY(box_solve_f32(c, c.V32, c.V32));
  return to_grid<float>(c, c.V32, nullptr, nullptr, nullptr, v_grid);
}

__global__ void copy_mask_kernel(long n, const uint8_t* in, uint8_t* out) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n;
       k += (long)gridDim.x * blockDim.x)
    out[k] = in[k];
}

kfbi_status inside_mask(Ctx& c, uint8_t* mask) {
  if (c.dim == 3) return inside_mask3(c, mask);
  const long n = (long)(c.N + 1) * (c.N + 1);
  prof_count(c, ST_GRID);
  copy_mask_kernel<<<gs_blocks(n), 256, 0, c.stream>>>(n, c.inside, mask);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace kfbi
