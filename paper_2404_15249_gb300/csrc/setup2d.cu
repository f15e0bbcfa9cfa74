// Setup of the discrete interface problem on the GPU, all in FP64 (Sec. 2.2, Alg. 1
// steps 1-3, Procedure 1 of Sec. 4.4).
//
// Geometry rules (the paper defers them to its CPU predecessor; these are the readings
// this library implements):
//  * Gamma is the periodic degree-5 Lagrange interpolant of the control points in the
//    uniform parameter t_k = 2 pi k / M; on [t_k, t_{k+1}) it interpolates X_{k-2..k+3}.
//  * Crossings with the grid lines: each segment is sampled at tau = s/8; a sub-interval
//    with end values A, B holds a crossing with the line c iff (A >= c) != (B >= c); the
//    crossing is located by bisection to below FP64 resolution and its coordinate along
//    the line is moved onto a grid node when it lies within 1e-10 h of it.
//  * Node (i, j) is inside iff an odd number of crossings on row j lie at x <= x_i.
//  * On every grid line the k-th crossing (in increasing order) belongs to the k-th arm
//    whose end labels differ and must lie on it (1e-8 h slack); otherwise the interface
//    is under-resolved (KFBI_ERR_GEOMETRY).  No node within two cells of the box
//    boundary may be inside.
//  * Irregular node: an interior node with a 5-point neighbour of the other label.
// The density -> corrected-RHS map (Alg. 2) and the grid -> v^+ map (Alg. 3) are linear;
// their FP64 weights are precomputed here so that an apply is a sparse gather.
#include <cstdarg>
#include <cstring>

#include <algorithm>
#include <array>
#include <vector>

#include "kfbi_internal.cuh"

namespace kfbi {

enum : int { ERR_GEOM_EDGE = 1, ERR_GEOM_MATCH = 2, ERR_GEOM_TOL = 4, ERR_GEOM_ARM = 8 };
constexpr double GRAZE_CURV = 0.5;   // |curvature| h of an accepted grazing pair
constexpr double MAX_CURV_H = 4.0;   // |curvature| h above this at a control point: rejected

constexpr int SUB = 8;
constexpr int BISECT = 64;
constexpr double SNAP = 1e-10;
constexpr double ARM_TOL = 1e-8;

__device__ __forceinline__ double grid_coord(double lo, int i, double h) {
  return __dadd_rn(lo, __dmul_rn((double)i, h));
}

// Lagrange basis of the nodes -2..3 at tau, with first and second derivatives.
__device__ __forceinline__ void lagrange6(double tau, double L0[6], double L1[6], double L2[6]) {
  const double den[6] = {-120.0, 24.0, -12.0, 12.0, -24.0, 120.0};
  double d[6];
#pragma unroll
  for (int s = 0; s < 6; ++s) d[s] = tau - (double)(s - 2);
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    double p0 = 1.0, p1 = 0.0, p2 = 0.0;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      if (s == r) continue;
      p2 = p2 * d[s] + 2.0 * p1;
      p1 = p1 * d[s] + p0;
      p0 = p0 * d[s];
    }
    L0[r] = p0 / den[r];
    L1[r] = p1 / den[r];
    L2[r] = p2 / den[r];
  }
}

__device__ __forceinline__ double lagrange_coord(const double* pts, int M, int seg, double tau,
                                                 int axis) {
  double L0[6], L1[6], L2[6];
  lagrange6(tau, L0, L1, L2);
  double acc = 0.0;
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    int k = seg - 2 + r;
    k = (k % M + M) % M;
    acc += L0[r] * pts[2 * k + axis];
  }
  return acc;
}

// ------------------------------------------------------------------ crossings
__global__ void samples_kernel(const double* pts, int M, double* samp) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;   // seg * (SUB+1) + s
  if (idx >= M * (SUB + 1)) return;
  const int seg = idx / (SUB + 1), s = idx - seg * (SUB + 1);
  double x, y;
  if (s == 0) {
    x = pts[2 * seg]; y = pts[2 * seg + 1];
  } else if (s == SUB) {
    const int k = (seg + 1) % M;
    x = pts[2 * k]; y = pts[2 * k + 1];
  } else {
    const double tau = (double)s / SUB;
    x = lagrange_coord(pts, M, seg, tau, 0);
    y = lagrange_coord(pts, M, seg, tau, 1);
  }
  samp[2 * idx] = x;
  samp[2 * idx + 1] = y;
}

// Lines crossed inside one sub-interval: i in [ilo, ihi] with (A >= x_i) != (B >= x_i).
__device__ __forceinline__ void subinterval_range(double A, double B, double lo, double h, int N,
                                                  int* ilo, int* ihi) {
  const double mn = fmin(A, B), mx = fmax(A, B);
  int a = (int)floor((mn - lo) / h) - 1, b = (int)ceil((mx - lo) / h) + 1;
  *ilo = a < 0 ? 0 : a;
  *ihi = b > N ? N : b;
}

// thread = (axis, seg, s); count (pass 0) or write (pass 1) the crossings it holds
__global__ void crossings_kernel(const double* pts, const double* samp, int M, int N, double lo,
                                 double h, int pass, int* counts, const int* offsets,
                                 int* out_line, int* out_seg, double* out_tau,
                                 double* out_along) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int per_axis = M * SUB;
  if (idx >= 2 * per_axis) return;
  const int axis = idx / per_axis, rem = idx - axis * per_axis;
  const int seg = rem / SUB, s = rem - seg * SUB;
  const double A = samp[2 * (seg * (SUB + 1) + s) + axis];
  const double B = samp[2 * (seg * (SUB + 1) + s + 1) + axis];
  int ilo, ihi;
  subinterval_range(A, B, lo, h, N, &ilo, &ihi);
  int cnt = 0, slot = pass ? offsets[idx] : 0;
  for (int i = ilo; i <= ihi; ++i) {
    const double c = grid_coord(lo, i, h);
    const bool pa = A >= c, pb = B >= c;
    if (pa == pb) continue;
    ++cnt;
    if (!pass) continue;
    double ta = (double)s / SUB, tb = (double)(s + 1) / SUB;
    for (int it = 0; it < BISECT; ++it) {
      const double tm = 0.5 * (ta + tb);
      const bool pm = lagrange_coord(pts, M, seg, tm, axis) >= c;
      if (pm == pa) ta = tm; else tb = tm;
    }
    const double tq = 0.5 * (ta + tb);
    double along = lagrange_coord(pts, M, seg, tq, 1 - axis);
    const int kn = (int)floor((along - lo) / h + 0.5);
    if (kn >= 0 && kn <= N) {
      const double xn = grid_coord(lo, kn, h);
      if (fabs(along - xn) <= SNAP * h) along = xn;
    }
    out_line[slot] = i;
    out_seg[slot] = seg;
    out_tau[slot] = tq;
    out_along[slot] = along;
    ++slot;
  }
  if (!pass) counts[idx] = cnt;
}

// Exclusive scan of n ints by one block (setup sizes only); total written to out[n].
__global__ void scan_kernel(const int* in, int* out, int n) {
  __shared__ int part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int chunk = (n + T - 1) / T;
  const int b = t * chunk, e = min(n, b + chunk);
  int s = 0;
  for (int i = b; i < e; ++i) s += in[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int i = 0; i < T; ++i) { const int v = part[i]; part[i] = run; run += v; }
    out[n] = run;
  }
  __syncthreads();
  int run = part[t];
  for (int i = b; i < e; ++i) { const int v = in[i]; out[i] = run; run += v; }
}

__global__ void line_count_kernel(const int* line, int n, int* cnt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) atomicAdd(&cnt[line[k]], 1);
}

__global__ void line_scatter_kernel(const int* line, int n, const int* ptr, int* fill, int* perm) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    const int L = line[k];
    perm[ptr[L] + atomicAdd(&fill[L], 1)] = k;
  }
}

// sort each line's crossings by (along, seg, tau): insertion sort, one thread per line
__global__ void line_sort_kernel(int nlines, const int* ptr, int* perm, const double* along,
                                 const int* seg, const double* tau) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlines) return;
  const int b = ptr[L], e = ptr[L + 1];
  for (int a = b + 1; a < e; ++a) {
    const int key = perm[a];
    int c = a - 1;
    while (c >= b) {
      const int o = perm[c];
      const bool gt = along[o] > along[key] ||
                      (along[o] == along[key] && (seg[o] > seg[key] ||
                                                  (seg[o] == seg[key] && tau[o] > tau[key])));
      if (!gt) break;
      perm[c + 1] = o;
      --c;
    }
    perm[c + 1] = key;
  }
}

__global__ void gather_cross_kernel(int n, const int* perm, const int* line, const int* seg,
                                    const double* tau, const double* along, int* line2,
                                    int* seg2, double* tau2, double* along2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int o = perm[k];
  line2[k] = line[o];
  seg2[k] = seg[o];
  tau2[k] = tau[o];
  along2[k] = along[o];
}

// ------------------------------------------------------------------ labels
__global__ void labels_kernel(int N, double lo, double h, const int* row_ptr,
                              const double* row_along, uint8_t* inside, int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i > N) return;
  const double x = grid_coord(lo, i, h);
  int cnt = 0;
  for (int q = row_ptr[j]; q < row_ptr[j + 1]; ++q) cnt += row_along[q] <= x;
  const uint8_t in = (uint8_t)(cnt & 1);
  inside[j * (N + 1) + i] = in;
  if (in && (i <= 1 || j <= 1 || i >= N - 1 || j >= N - 1)) atomicOr(err, ERR_GEOM_EDGE);
}

// one thread per grid line: the k-th crossing <-> the k-th arm with a label change
// |curvature| of the interpolant at (seg, tau): |X' x X''| / |X'|^3 (the t-scaling cancels)
__device__ double abs_curvature(const double* pts, int M, int seg, double tau) {
  double L0[6], L1[6], L2[6];
  lagrange6(tau, L0, L1, L2);
  double x1 = 0, y1 = 0, x2 = 0, y2 = 0;
  for (int r = 0; r < 6; ++r) {
    int k = seg - 2 + r;
    k = (k % M + M) % M;
    x1 += L1[r] * pts[2 * k];
    y1 += L1[r] * pts[2 * k + 1];
    x2 += L2[r] * pts[2 * k];
    y2 += L2[r] * pts[2 * k + 1];
  }
  const double s = sqrt(x1 * x1 + y1 * y1);
  return fabs(x1 * y2 - y1 * x2) / (s * s * s);
}

__global__ void match_kernel(int N, double lo, double h, int axis, const int* ptr,
                             const double* along, const int* seg, const double* tau,
                             const double* pts, int M, const uint8_t* inside, int* flip, int* err) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L > N) return;
  const int b = ptr[L], e = ptr[L + 1];
  const double tol = ARM_TOL * h;
  // axis 1 crossings lie on row L (walk i); axis 0 crossings on column L (walk j)
  auto label = [&](int t) -> uint8_t {
    return axis ? inside[L * (N + 1) + t] : inside[t * (N + 1) + L];
  };
  // grazing pairs: two consecutive crossings strictly inside one arm whose end labels
  // agree, on a part of the curve resolved by the grid (radius of curvature above 2 h),
  // carry no correction; marked -2 - arm until the end
  for (int q = b; q < e;) {
    if (q + 1 < e) {
      const double a0 = along[q], a1 = along[q + 1];
      const int t = (int)floor((a0 - lo) / h);
      if (t >= 0 && t < N && a0 > grid_coord(lo, t, h) + tol && a1 < grid_coord(lo, t + 1, h) - tol &&
          label(t) == label(t + 1) && abs_curvature(pts, M, seg[q], tau[q]) * h <= GRAZE_CURV &&
          abs_curvature(pts, M, seg[q + 1], tau[q + 1]) * h <= GRAZE_CURV) {
        flip[q] = flip[q + 1] = -2 - t;
        q += 2;
        continue;
      }
    }
    flip[q] = -1;
    ++q;
  }
  // every other crossing, in order, belongs to the next arm whose end labels differ
  int r = b;
  uint8_t prev = label(0);
  for (int t = 0; t < N; ++t) {
    const uint8_t next = label(t + 1);
    if (next != prev) {
      while (r < e && flip[r] <= -2) ++r;
      if (r >= e) { atomicOr(err, ERR_GEOM_MATCH); return; }
      const double a = along[r];
      if (a < grid_coord(lo, t, h) - tol || a > grid_coord(lo, t + 1, h) + tol) {
        atomicOr(err, ERR_GEOM_TOL);
        return;
      }
      flip[r] = t;
      ++r;
    }
    prev = next;
  }
  while (r < e && flip[r] <= -2) ++r;
  if (r != e) { atomicOr(err, ERR_GEOM_MATCH); return; }
  for (int q = b; q < e; ++q)
    if (flip[q] <= -2) flip[q] = -2 - flip[q];     // arm of the grazing pair (never looked up)
}

__global__ void count_inside_kernel(int n, const uint8_t* inside, int* out) {
  int s = 0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    s += inside[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// ------------------------------------------------------------------ irregular nodes
__device__ __forceinline__ int arm_mask(int N, const uint8_t* inside, int i, int j) {
  const uint8_t c = inside[j * (N + 1) + i];
  int m = 0;
  m |= (inside[j * (N + 1) + i + 1] != c) << 0;
  m |= (inside[j * (N + 1) + i - 1] != c) << 1;
  m |= (inside[(j + 1) * (N + 1) + i] != c) << 2;
  m |= (inside[(j - 1) * (N + 1) + i] != c) << 3;
  return m;
}

// per interior row: number of irregular nodes and of crossed arms
__global__ void irr_row_count_kernel(int N, const uint8_t* inside, int* row_nodes,
                                     int* row_arms) {
  const int j = blockIdx.x + 1;
  int nn = 0, na = 0;
  for (int i = 1 + threadIdx.x; i < N; i += blockDim.x) {
    const int m = arm_mask(N, inside, i, j);
    nn += m != 0;
    na += __popc(m);
  }
  __shared__ int sn[32], sa[32];
  for (int o = 16; o > 0; o >>= 1) {
    nn += __shfl_down_sync(0xffffffffu, nn, o);
    na += __shfl_down_sync(0xffffffffu, na, o);
  }
  if ((threadIdx.x & 31) == 0) { sn[threadIdx.x >> 5] = nn; sa[threadIdx.x >> 5] = na; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) { a += sn[w]; b += sa[w]; }
    row_nodes[j - 1] = a;
    row_arms[j - 1] = b;
  }
}

// per interior row, in increasing i: node list, arm pointers, arm (node, direction)
__global__ void irr_row_fill_kernel(int N, const uint8_t* inside, const int* node_off,
                                    const int* arm_off, int* irr_node, int* arm_ptr,
                                    int* arm_dir, int* arm_owner) {
  const int j = blockIdx.x + 1;
  __shared__ int wn[32], wa[32];
  __shared__ int base_n, base_a;
  if (threadIdx.x == 0) { base_n = node_off[j - 1]; base_a = arm_off[j - 1]; }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 1; i0 < N; i0 += blockDim.x) {
    const int i = i0 + threadIdx.x;
    const int m = (i < N) ? arm_mask(N, inside, i, j) : 0;
    const int isn = m != 0, na = __popc(m);
    int pn = isn, pa = na;
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(0xffffffffu, pn, o), b = __shfl_up_sync(0xffffffffu, pa, o);
      if (lane >= o) { pn += a; pa += b; }
    }
    if (lane == 31) { wn[warp] = pn; wa[warp] = pa; }
    __syncthreads();
    int on = 0, oa = 0, tn = 0, ta = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) { on += wn[w]; oa += wa[w]; }
      tn += wn[w];
      ta += wa[w];
    }
    if (isn) {
      const int k = base_n + on + pn - 1;
      int a = base_a + oa + pa - na;
      irr_node[k] = j * N + i;
      arm_ptr[k] = a;
      for (int d = 0; d < 4; ++d)
        if (m & (1 << d)) { arm_dir[a] = d; arm_owner[a] = k; ++a; }
    }
    __syncthreads();
    if (threadIdx.x == 0) { base_n += tn; base_a += ta; }
    __syncthreads();
  }
}

struct CurvePoint {
  double tx, ty, nx, ny, chi, sp, spp;   // unit tangent, outward normal, curvature, s', s''
};

__device__ __forceinline__ CurvePoint curve_point(const double* pts, int M, int seg,
                                                  const double L1[6], const double L2[6],
                                                  double dt) {
  double x1 = 0, y1 = 0, x2 = 0, y2 = 0;
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    int k = seg - 2 + r;
    k = (k % M + M) % M;
    x1 += L1[r] * pts[2 * k];
    y1 += L1[r] * pts[2 * k + 1];
    x2 += L2[r] * pts[2 * k];
    y2 += L2[r] * pts[2 * k + 1];
  }
  x1 /= dt; y1 /= dt; x2 /= dt * dt; y2 /= dt * dt;
  CurvePoint c;
  c.sp = sqrt(x1 * x1 + y1 * y1);
  c.spp = (x1 * x2 + y1 * y2) / c.sp;
  c.tx = x1 / c.sp;
  c.ty = y1 / c.sp;
  c.nx = c.ty;
  c.ny = -c.tx;
  c.chi = (x1 * y2 - y1 * x2) / (c.sp * c.sp * c.sp);
  return c;
}

// first / second arc-length derivative weights of a control-point function
__device__ __forceinline__ void surface_weights(const double L1[6], const double L2[6], double dt,
                                                double sp, double spp, double D1[6],
                                                double D2[6]) {
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    D1[r] = L1[r] / (dt * sp);
    D2[r] = (L2[r] / (dt * dt) - D1[r] * spp) / (sp * sp);
  }
}

// crossing id on a line whose sorted crossings carry flip[] = lower arm index
__device__ __forceinline__ int find_crossing(const int* ptr, const int* flip, int line, int arm) {
  int a = ptr[line], b = ptr[line + 1] - 1;
  while (a <= b) {
    const int m = (a + b) >> 1;
    if (flip[m] == arm) return m;
    if (flip[m] < arm) a = m + 1; else b = m - 1;
  }
  return -1;
}

// Taylor correction weights per crossed arm (Alg. 2):
//   b_p += sigma/h^2 ([v] + d [v_a] + d^2/2 [v_aa])(q),  d = nb_a - q_a,
// with the jumps of the double layer ([v] = phi, [d_n v] = 0), single layer
// ([v] = 0, [d_n v] = psi) and volume term ([F] = f) written through the interpolant.
__global__ void arm_weights_kernel(int N, int M, double lo, double h, double kappa2,
                                   const double* pts, const uint8_t* inside, const int* irr_node,
                                   int narms, const int* arm_dir, const int* arm_owner,
                                   const int* ptr0, const int* flip0, const int* seg0,
                                   const double* tau0, const double* along0, const int* ptr1,
                                   const int* flip1, const int* seg1, const double* tau1,
                                   const double* along1, int* arm_seg, double* wD, double* wS,
                                   double* wF, int* err) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= narms) return;
  const int node = irr_node[arm_owner[a]];
  const int i = node % N, j = node / N;
  const int d = arm_dir[a];
  const int di = d == 0 ? 1 : (d == 1 ? -1 : 0), dj = d == 2 ? 1 : (d == 3 ? -1 : 0);
  const bool horiz = dj == 0;
  int q, seg;
  double tau, qa, nba;
  if (horiz) {   // arm on row j between min(i, i+di) and max; crossing of a horizontal line
    q = find_crossing(ptr1, flip1, j, min(i, i + di));
    if (q < 0) { atomicOr(err, ERR_GEOM_ARM); return; }
    seg = seg1[q]; tau = tau1[q]; qa = along1[q]; nba = grid_coord(lo, i + di, h);
  } else {
    q = find_crossing(ptr0, flip0, i, min(j, j + dj));
    if (q < 0) { atomicOr(err, ERR_GEOM_ARM); return; }
    seg = seg0[q]; tau = tau0[q]; qa = along0[q]; nba = grid_coord(lo, j + dj, h);
  }
  const double dt = 2.0 * M_PI / M;
  double L0[6], L1[6], L2[6], D1[6], D2[6];
  lagrange6(tau, L0, L1, L2);
  const CurvePoint cp = curve_point(pts, M, seg, L1, L2, dt);
  surface_weights(L1, L2, dt, cp.sp, cp.spp, D1, D2);
  const double na = horiz ? cp.nx : cp.ny, ta = horiz ? cp.tx : cp.ty;
  const double dl = nba - qa;
  const double sigma = inside[j * (N + 1) + i] ? -1.0 : 1.0;
  const double f = sigma / (h * h), hd2 = 0.5 * dl * dl;
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    wD[6 * a + r] = f * (L0[r] + dl * ta * D1[r] +
                         hd2 * (kappa2 * na * na * L0[r] + (ta * ta - na * na) * D2[r] -
                                2.0 * cp.chi * na * ta * D1[r]));
    wS[6 * a + r] = f * (dl * na * L0[r] +
                         hd2 * (cp.chi * (ta * ta - na * na) * L0[r] + 2.0 * na * ta * D1[r]));
    wF[6 * a + r] = f * hd2 * na * na * L0[r];
  }
  arm_seg[a] = seg;
}

// Interpolation stencil and weights at each control point (Alg. 3): nearest node c,
// nodes c, c+-e_x, c+-e_y, c + s_x e_x + s_y e_y; closed-form quadratic interpolation
// weights at z; the second-order Taylor expansion of the jump about z is added at
// outside nodes, folded into density / f weights.
// With cwn/cDn/cSn/eFn: the same for n . grad of the quadratic at z (the Neumann data d_n v^+):
// the cardinal weights differentiated in the local coordinates (A, B) and divided by h.
__global__ void ctrl_weights_kernel(int N, int M, double lo, double h, double kappa2,
                                    const double* pts, const double* nrm, const double* curv,
                                    const uint8_t* inside, int* cnode, double* cw, double* cD,
                                    double* cS, double* eF, double* cwn, double* cDn,
                                    double* cSn, double* eFn, int* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  const double zx = pts[2 * k], zy = pts[2 * k + 1];
  const int ci = (int)floor((zx - lo) / h + 0.5), cj = (int)floor((zy - lo) / h + 0.5);
  if (ci < 1 || cj < 1 || ci > N - 1 || cj > N - 1) { atomicOr(err, ERR_GEOM_EDGE); return; }
  const double xc = grid_coord(lo, ci, h), yc = grid_coord(lo, cj, h);
  const int sx = zx >= xc ? 1 : -1, sy = zy >= yc ? 1 : -1;
  const int oi[6] = {0, 1, -1, 0, 0, sx}, oj[6] = {0, 0, 0, 1, -1, sy};
  const double A = (zx - xc) / h, B = (zy - yc) / h, S = (double)(sx * sy), SAB = S * A * B;
  double w[6];
  w[0] = 1.0 - A * A - B * B + SAB;
  w[1] = 0.5 * A + 0.5 * A * A - 0.5 * SAB * (sx + 1);
  w[2] = -0.5 * A + 0.5 * A * A + 0.5 * SAB * (sx - 1);
  w[3] = 0.5 * B + 0.5 * B * B - 0.5 * SAB * (sy + 1);
  w[4] = -0.5 * B + 0.5 * B * B + 0.5 * SAB * (sy - 1);
  w[5] = SAB;
  // d w / d A and d w / d B (A = (z_x - x_c)/h, B = (z_y - y_c)/h)
  const double SA = S * A, SB = S * B;
  const double wA[6] = {-2.0 * A + SB, 0.5 + A - 0.5 * SB * (sx + 1), -0.5 + A + 0.5 * SB * (sx - 1),
                        -0.5 * SB * (sy + 1), 0.5 * SB * (sy - 1), SB};
  const double wB[6] = {-2.0 * B + SA, -0.5 * SA * (sx + 1), 0.5 * SA * (sx - 1),
                        0.5 + B - 0.5 * SA * (sy + 1), -0.5 + B + 0.5 * SA * (sy - 1), SA};
  const double dt = 2.0 * M_PI / M;
  double L0[6], L1[6], L2[6], D1[6], D2[6];
  lagrange6(0.0, L0, L1, L2);
  const CurvePoint cp = curve_point(pts, M, k, L1, L2, dt);
  surface_weights(L1, L2, dt, cp.sp, cp.spp, D1, D2);
  const double nx = nrm[2 * k], ny = nrm[2 * k + 1], tx = -ny, ty = nx, chi = curv[k];
  double wn[6];
#pragma unroll
  for (int p = 0; p < 6; ++p) wn[p] = (nx * wA[p] + ny * wB[p]) / h;
  double accD[6] = {0, 0, 0, 0, 0, 0}, accS[6] = {0, 0, 0, 0, 0, 0}, accF = 0.0;
  double accDn[6] = {0, 0, 0, 0, 0, 0}, accSn[6] = {0, 0, 0, 0, 0, 0}, accFn = 0.0;
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const int ii = ci + oi[p], jj = cj + oj[p];
    const bool interior = ii >= 1 && jj >= 1 && ii <= N - 1 && jj <= N - 1;
    cnode[6 * k + p] = interior ? jj * N + ii : -1;
    cw[6 * k + p] = w[p];
    cwn[6 * k + p] = wn[p];
    if (inside[jj * (N + 1) + ii]) continue;
    const double px = grid_coord(lo, ii, h) - zx, py = grid_coord(lo, jj, h) - zy;
    const double dn = px * nx + py * ny, dtau = px * tx + py * ty;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      // the jump's Taylor term at node p as weights of the density (D) and psi (S)
      const double tD = L0[r] + dtau * D1[r] +
                        0.5 * (kappa2 * dn * dn * L0[r] + (dtau * dtau - dn * dn) * D2[r] -
                               2.0 * chi * dn * dtau * D1[r]);
      const double tS = dn * L0[r] + 0.5 * (chi * (dtau * dtau - dn * dn) * L0[r] +
                                            2.0 * dn * dtau * D1[r]);
      accD[r] += w[p] * tD;
      accS[r] += w[p] * tS;
      accDn[r] += wn[p] * tD;
      accSn[r] += wn[p] * tS;
    }
    accF += w[p] * 0.5 * dn * dn;
    accFn += wn[p] * 0.5 * dn * dn;
  }
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    cD[6 * k + r] = accD[r];
    cS[6 * k + r] = accS[r];
    cDn[6 * k + r] = accDn[r];
    cSn[6 * k + r] = accSn[r];
  }
  eF[k] = accF;
  eFn[k] = accFn;
}

// ------------------------------------------------------------------ host driver
static inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

// Work items of the sparse first x-transform (one CTA each).  A row with at most
// kSpxNodes irregular nodes is one item; a longer one (where Gamma runs nearly along the
// row) is split into parts of near-equal node counts, whose partial rows go to scratch
// slots and are added, in part order, by the last part to finish.  Items are ordered by
// decreasing node count, so the longest start first and the empty rows fill the tail.
// (Item sizes from a sweep of the N = 4096 mixed solve: at most 64 irregular nodes and 24
// stencil nodes per item, 11.35 ms; 16 / 12: 11.49 ms, 32 / 24: 11.37, 64 / 48: 11.43,
// rows never split: 12.24.)
constexpr int kSpxNodes = 64;
// stencil nodes per work item of the sparse-output x-transform
constexpr int kSnNodes = 24;

static kfbi_status build_spx_items(Ctx& c, const int* node_off) {
  const int N = c.N;
  cudaStream_t st = c.stream;
  std::vector<int> off(N);
  KFBI_CUDA_TRY(cudaMemcpyAsync(off.data(), node_off, sizeof(int) * N, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<std::array<int, 8>> items;
  items.reserve(N + c.nirr / kSpxNodes + 1);
  int slots = 0, split = 0;
  for (int j = 0; j < N; ++j) {
    const int n0 = j > 0 ? off[j - 1] : 0, n1 = j > 0 ? off[j] : 0, cnt = n1 - n0;
    if (cnt <= kSpxNodes) {
      items.push_back({j, n0, n1, 0, 1, 0, 0, 0});
      continue;
    }
    const int P = (cnt + kSpxNodes - 1) / kSpxNodes;
    for (int p = 0; p < P; ++p)
      items.push_back({j, n0 + (int)((long)cnt * p / P), n0 + (int)((long)cnt * (p + 1) / P), p, P,
                       slots, split, 0});
    slots += P;
    ++split;
  }
  std::stable_sort(items.begin(), items.end(), [](const std::array<int, 8>& a,
                                                  const std::array<int, 8>& b) {
    return a[2] - a[1] > b[2] - b[1];
  });
  c.spx_nitems = (int)items.size();
  KFBI_TRY(alloc_bytes(c, (void**)&c.spx_items, sizeof(int) * 8 * items.size()));
  KFBI_TRY(alloc_bytes(c, (void**)&c.spx_part, sizeof(float) * (size_t)std::max(slots, 1) * N));
  KFBI_TRY(alloc_bytes(c, (void**)&c.spx_cnt, sizeof(unsigned) * (split + 1)));
  KFBI_CUDA_TRY(cudaMemsetAsync(c.spx_cnt, 0, sizeof(unsigned) * (split + 1), st));
  KFBI_CUDA_TRY(cudaMemcpyAsync(c.spx_items, items.data(), sizeof(int) * 8 * items.size(),
                                cudaMemcpyHostToDevice, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));   // the host vector goes out of scope
  return KFBI_OK;
}

// The distinct interior stencil nodes of the control points, sorted by grid row then
// column (the plain FP32 apply evaluates its last x-transform only there), each stencil
// entry's slot in that list (-1 on the box boundary), and the work items: each row's
// nodes in parts of at most kSnNodes, longest first.
static kfbi_status build_stencil_nodes(Ctx& c) {
  const int N = c.N, M = c.M;
  cudaStream_t st = c.stream;
  std::vector<int> cn((size_t)6 * M);
  KFBI_CUDA_TRY(cudaMemcpyAsync(cn.data(), c.ctrl_node, sizeof(int) * 6 * M,
                                cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int> nodes;
  nodes.reserve(cn.size());
  for (int q : cn)
    if (q >= 0) nodes.push_back(q);
  std::sort(nodes.begin(), nodes.end());
  nodes.erase(std::unique(nodes.begin(), nodes.end()), nodes.end());
  std::vector<int> slot(cn.size()), col(nodes.size());
  for (size_t e = 0; e < cn.size(); ++e)
    slot[e] = cn[e] < 0 ? -1
                        : (int)(std::lower_bound(nodes.begin(), nodes.end(), cn[e]) - nodes.begin());
  std::vector<std::array<int, 4>> items;
  for (size_t q0 = 0; q0 < nodes.size();) {        // one row's nodes [q0, q1), in parts
    const int j = nodes[q0] / N;
    size_t q1 = q0;
    for (; q1 < nodes.size() && nodes[q1] / N == j; ++q1) col[q1] = nodes[q1] - j * N;
    const int cnt = (int)(q1 - q0), P = (cnt + kSnNodes - 1) / kSnNodes;
    for (int p = 0; p < P; ++p)
      items.push_back({j, (int)q0 + cnt * p / P, (int)q0 + cnt * (p + 1) / P, 0});
    q0 = q1;
  }
  std::stable_sort(items.begin(), items.end(), [](const std::array<int, 4>& a,
                                                  const std::array<int, 4>& b) {
    return a[2] - a[1] > b[2] - b[1];
  });
  c.sn_count = (int)nodes.size();
  c.sn_nitems = (int)items.size();
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_slot, sizeof(int) * 6 * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.sn_col, sizeof(int) * (nodes.size() + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.sn_items, sizeof(int) * 4 * (items.size() + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.sn_val, sizeof(float) * (nodes.size() + 1)));
  KFBI_CUDA_TRY(cudaMemcpyAsync(c.ctrl_slot, slot.data(), sizeof(int) * slot.size(),
                                cudaMemcpyHostToDevice, st));
  if (!nodes.empty()) {
    KFBI_CUDA_TRY(cudaMemcpyAsync(c.sn_col, col.data(), sizeof(int) * col.size(),
                                  cudaMemcpyHostToDevice, st));
    KFBI_CUDA_TRY(cudaMemcpyAsync(c.sn_items, items.data(), sizeof(int) * 4 * items.size(),
                                  cudaMemcpyHostToDevice, st));
  }
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));   // the host vectors go out of scope
  return KFBI_OK;
}

kfbi_status setup_geometry(Ctx& c) {
  const int N = c.N, M = c.M;
  cudaStream_t st = c.stream;
  int* tmp_i = nullptr;
  KFBI_CUDA_TRY(cudaMemsetAsync(c.err_flag, 0, sizeof(int), st));
  {
    // the grid must resolve the curve: radius of curvature of at least a quarter cell
    std::vector<double> curv(M);
    KFBI_CUDA_TRY(cudaMemcpyAsync(curv.data(), c.curv, sizeof(double) * M, cudaMemcpyDeviceToHost, st));
    KFBI_CUDA_TRY(cudaStreamSynchronize(st));
    double kmax = 0.0;
    for (double k : curv) kmax = fmax(kmax, fabs(k));
    if (!(kmax * c.h <= MAX_CURV_H)) {
      set_error("kfbi_setup: interface geometry rejected: radius of curvature below a quarter cell "
                "(max |curvature| h = %.3g, under-resolved interface)", kmax * c.h);
      return KFBI_ERR_GEOMETRY;
    }
  }

  // samples and crossings
  double* samp = nullptr;
  const int nsub = 2 * M * SUB;
  KFBI_TRY(alloc_bytes(c, (void**)&samp, sizeof(double) * 2 * M * (SUB + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&tmp_i, sizeof(int) * (2 * nsub + 2)));
  int* counts = tmp_i;
  int* offs = tmp_i + nsub;
  prof_count(c, ST_SETUP);
  samples_kernel<<<nblk(M * (SUB + 1), 256), 256, 0, st>>>(c.pts, M, samp);
  prof_count(c, ST_SETUP);
  crossings_kernel<<<nblk(nsub, 256), 256, 0, st>>>(c.pts, samp, M, N, c.lo, c.h, 0, counts,
                                                     nullptr, nullptr, nullptr, nullptr, nullptr);
  prof_count(c, ST_SETUP);
  scan_kernel<<<1, 1024, 0, st>>>(counts, offs, nsub);
  KFBI_CUDA_TRY(cudaGetLastError());
  // per-axis totals: the axis-0 sub-intervals come first
  int h_tot[2];
  KFBI_CUDA_TRY(cudaMemcpyAsync(&h_tot[0], offs + M * SUB, sizeof(int), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaMemcpyAsync(&h_tot[1], offs + nsub, sizeof(int), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  const int total = h_tot[1];
  c.ncross[0] = h_tot[0];
  c.ncross[1] = total - h_tot[0];
  int *line = nullptr, *seg = nullptr;
  double *tau = nullptr, *along = nullptr;
  KFBI_TRY(alloc_bytes(c, (void**)&line, sizeof(int) * (total + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&seg, sizeof(int) * (total + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&tau, sizeof(double) * (total + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&along, sizeof(double) * (total + 1)));
  prof_count(c, ST_SETUP);
  crossings_kernel<<<nblk(nsub, 256), 256, 0, st>>>(c.pts, samp, M, N, c.lo, c.h, 1, nullptr,
                                                     offs, line, seg, tau, along);
  KFBI_CUDA_TRY(cudaGetLastError());

  // per axis: bin by line, sort along the line, gather into sorted arrays
  int* lcnt = nullptr;
  int* fill = nullptr;
  int* perm = nullptr;
  KFBI_TRY(alloc_bytes(c, (void**)&lcnt, sizeof(int) * (N + 2)));
  KFBI_TRY(alloc_bytes(c, (void**)&fill, sizeof(int) * (N + 2)));
  KFBI_TRY(alloc_bytes(c, (void**)&perm, sizeof(int) * (total + 1)));
  for (int ax = 0; ax < 2; ++ax) {
    const int n = c.ncross[ax], base = ax ? c.ncross[0] : 0;
    KFBI_TRY(alloc_bytes(c, (void**)&c.line_ptr[ax], sizeof(int) * (N + 3)));
    KFBI_TRY(alloc_bytes(c, (void**)&c.cr_line[ax], sizeof(int) * (n + 1)));
    KFBI_TRY(alloc_bytes(c, (void**)&c.cr_seg[ax], sizeof(int) * (n + 1)));
    KFBI_TRY(alloc_bytes(c, (void**)&c.cr_tau[ax], sizeof(double) * (n + 1)));
    KFBI_TRY(alloc_bytes(c, (void**)&c.cr_along[ax], sizeof(double) * (n + 1)));
    KFBI_TRY(alloc_bytes(c, (void**)&c.cr_flip[ax], sizeof(int) * (n + 1)));
    KFBI_CUDA_TRY(cudaMemsetAsync(lcnt, 0, sizeof(int) * (N + 2), st));
    KFBI_CUDA_TRY(cudaMemsetAsync(fill, 0, sizeof(int) * (N + 2), st));
    if (n > 0) line_count_kernel<<<nblk(n, 256), 256, 0, st>>>(line + base, n, lcnt);
    prof_count(c, ST_SETUP);
    scan_kernel<<<1, 1024, 0, st>>>(lcnt, c.line_ptr[ax], N + 1);
    if (n > 0) {
      prof_count(c, ST_SETUP);
      line_scatter_kernel<<<nblk(n, 256), 256, 0, st>>>(line + base, n, c.line_ptr[ax], fill,
                                                        perm);
      prof_count(c, ST_SETUP);
      line_sort_kernel<<<nblk(N + 1, 128), 128, 0, st>>>(N + 1, c.line_ptr[ax], perm,
                                                         along + base, seg + base, tau + base);
      prof_count(c, ST_SETUP);
      gather_cross_kernel<<<nblk(n, 256), 256, 0, st>>>(n, perm, line + base, seg + base,
                                                         tau + base, along + base, c.cr_line[ax],
                                                         c.cr_seg[ax], c.cr_tau[ax],
                                                         c.cr_along[ax]);
    }
    KFBI_CUDA_TRY(cudaGetLastError());
  }

  // labels from row parity; matching of crossings to label changes on every line
  KFBI_TRY(alloc_bytes(c, (void**)&c.inside, (size_t)(N + 1) * (N + 1)));
  prof_count(c, ST_SETUP);
  labels_kernel<<<dim3(nblk(N + 1, 256), N + 1), 256, 0, st>>>(N, c.lo, c.h, c.line_ptr[1],
                                                               c.cr_along[1], c.inside,
                                                               c.err_flag);
  for (int ax = 0; ax < 2; ++ax) {
    prof_count(c, ST_SETUP);
    match_kernel<<<nblk(N + 1, 64), 64, 0, st>>>(N, c.lo, c.h, ax, c.line_ptr[ax],
                                                 c.cr_along[ax], c.cr_seg[ax], c.cr_tau[ax],
                                                 c.pts, M, c.inside, c.cr_flip[ax], c.err_flag);
  }
  KFBI_CUDA_TRY(cudaGetLastError());
  int* d_inside_cnt = counts;   // reuse scratch
  KFBI_CUDA_TRY(cudaMemsetAsync(d_inside_cnt, 0, sizeof(int), st));
  prof_count(c, ST_SETUP);
  count_inside_kernel<<<256, 256, 0, st>>>((N + 1) * (N + 1), c.inside, d_inside_cnt);
  int h_err = 0;
  KFBI_CUDA_TRY(cudaMemcpyAsync(&h_err, c.err_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaMemcpyAsync(&c.n_inside, d_inside_cnt, sizeof(int), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_err) {
    set_error("interface geometry rejected (code %d): %s", h_err,
              (h_err & ERR_GEOM_EDGE) ? "interface within two cells of the box boundary"
                                      : "a grid line meets the interface where the node labels "
                                        "do not change (tangency or under-resolved interface)");
    return KFBI_ERR_GEOMETRY;
  }

  // irregular nodes and crossed arms, compacted row by row
  int* row_nodes = nullptr;
  int* row_arms = nullptr;
  KFBI_TRY(alloc_bytes(c, (void**)&row_nodes, sizeof(int) * (N + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&row_arms, sizeof(int) * (N + 1)));
  int* node_off = nullptr;
  int* arm_off = nullptr;
  KFBI_TRY(alloc_bytes(c, (void**)&node_off, sizeof(int) * (N + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&arm_off, sizeof(int) * (N + 1)));
  prof_count(c, ST_SETUP);
  irr_row_count_kernel<<<N - 1, 256, 0, st>>>(N, c.inside, row_nodes, row_arms);
  prof_count(c, ST_SETUP);
  scan_kernel<<<1, 1024, 0, st>>>(row_nodes, node_off, N - 1);
  prof_count(c, ST_SETUP);
  scan_kernel<<<1, 1024, 0, st>>>(row_arms, arm_off, N - 1);
  KFBI_CUDA_TRY(cudaGetLastError());
  int h_n[2];
  KFBI_CUDA_TRY(cudaMemcpyAsync(&h_n[0], node_off + (N - 1), sizeof(int), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaMemcpyAsync(&h_n[1], arm_off + (N - 1), sizeof(int), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  c.nirr = h_n[0];
  c.narms = h_n[1];
  int* arm_dir = nullptr;
  int* arm_owner = nullptr;
  KFBI_TRY(alloc_bytes(c, (void**)&c.irr_node, sizeof(int) * (c.nirr + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm_ptr, sizeof(int) * (c.nirr + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&arm_dir, sizeof(int) * (c.narms + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&arm_owner, sizeof(int) * (c.narms + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm_seg, sizeof(int) * (c.narms + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm_wD, sizeof(double) * 6 * (c.narms + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm_wS, sizeof(double) * 6 * (c.narms + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm_wF, sizeof(double) * 6 * (c.narms + 1)));
  prof_count(c, ST_SETUP);
  irr_row_fill_kernel<<<N - 1, 256, 0, st>>>(N, c.inside, node_off, arm_off, c.irr_node,
                                             c.arm_ptr, arm_dir, arm_owner);
  KFBI_CUDA_TRY(cudaMemcpyAsync(c.arm_ptr + c.nirr, &c.narms, sizeof(int), cudaMemcpyHostToDevice, st));
  if (c.narms > 0)
    arm_weights_kernel<<<nblk(c.narms, 128), 128, 0, st>>>(
        N, M, c.lo, c.h, c.kappa2, c.pts, c.inside, c.irr_node, c.narms, arm_dir, arm_owner,
        c.line_ptr[0], c.cr_flip[0], c.cr_seg[0], c.cr_tau[0], c.cr_along[0], c.line_ptr[1],
        c.cr_flip[1], c.cr_seg[1], c.cr_tau[1], c.cr_along[1], c.arm_seg, c.arm_wD, c.arm_wS,
        c.arm_wF, c.err_flag);
  KFBI_CUDA_TRY(cudaGetLastError());

  // control-point stencils
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_node, sizeof(int) * 6 * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_w, sizeof(double) * 6 * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_cD, sizeof(double) * 6 * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_cS, sizeof(double) * 6 * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_eF, sizeof(double) * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_wn, sizeof(double) * 6 * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_cDn, sizeof(double) * 6 * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_cSn, sizeof(double) * 6 * M));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ctrl_eFn, sizeof(double) * M));
  prof_count(c, ST_SETUP);
  ctrl_weights_kernel<<<nblk(M, 128), 128, 0, st>>>(N, M, c.lo, c.h, c.kappa2, c.pts, c.nrm,
                                                    c.curv, c.inside, c.ctrl_node, c.ctrl_w,
                                                    c.ctrl_cD, c.ctrl_cS, c.ctrl_eF, c.ctrl_wn,
                                                    c.ctrl_cDn, c.ctrl_cSn, c.ctrl_eFn, c.err_flag);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_CUDA_TRY(cudaMemcpyAsync(&h_err, c.err_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  if (h_err) {
    set_error("interface geometry rejected while building stencils (code %d)", h_err);
    return KFBI_ERR_GEOMETRY;
  }
  c.irr_rowptr = node_off;       // row j (1 <= j < N) holds irregular nodes [j-1], [j]
  KFBI_TRY(build_spx_items(c, node_off));
  KFBI_TRY(build_stencil_nodes(c));

  return KFBI_OK;
}

}  // namespace kfbi
