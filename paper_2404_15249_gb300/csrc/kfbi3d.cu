// 3-D KFBI (box [lo, hi]^3, 7-point Laplacian): setup of the interface given by its
// grid-line intersection points, the jumps of a density at the points, the right-hand
// side correction at irregular nodes, the 10-point corrected interpolation, and the
// interface solves built from them.  Readings of the unstated 3-D details:
//   * the control points are the caller's grid-line intersections (outward normals,
//     symmetric shape operators S with dn = S dx, packed Sxx Syy Szz Sxy Sxz Syz); a point
//     lies on the line of axis a when its two other coordinates are grid values to
//     1e-9 h, on the edge x_e < x_q < x_{e+1} of that line;
//   * node labels by parity along x-lines (node i inside iff an odd number of the line's
//     points lie below it), checked against the y- and z-line parities; an edge whose end
//     labels differ holds exactly one point (two points on one edge: a grazing line, no
//     arm); no inside node within two cells of the box boundary;
//   * surface derivatives: least-squares quadratic in tangent-plane coordinates scaled by
//     h over the points within 2.5 h (3.5 h when fewer than 10), normal equations by
//     Cholesky in FP64; the fitted value replaces the point value in the jumps, and the
//     double-layer apply adds half the difference between the two (the identity part of
//     the second-kind equation acts on the point values, Sec. 2.1);
//   * jumps in the local frame (n, t1, t2): grad[v] = psi n + grad_G Phi, tangential block
//     Hess_G Phi + psi II, mixed d_a psi - t_a . S grad_G Phi, normal-normal
//     [F] + kappa^2 Phi - Lap_G Phi - tr(S) psi, rotated to Cartesian axes;
//   * correction along the 6 arms as in 2-D (Alg. 2), interpolation on the 10-node stencil
//     c, c +- e_a, c + s_a e_a + s_b e_b (Alg. 3) with Taylor terms at outside nodes.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "fpbits.cuh"
#include "kfbi_internal.cuh"

namespace kfbi {

namespace {

constexpr double TAG_TOL = 1e-9;
constexpr double LS_R = 2.5, LS_R_WIDE = 3.5;
constexpr int LS_MIN = 10;
constexpr int ERR3_LABELS = 1, ERR3_BAND = 2, ERR3_ARM = 4, ERR3_LS = 8, ERR3_STENCIL = 16;

inline int nblk(long n, int t) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ long gidx3(int N, int i, int j, int k) {   // (N+1)^3 grid
  return ((long)k * (N + 1) + j) * (N + 1) + i;
}
__device__ __forceinline__ long widx3(int N, int i, int j, int k) {   // N^3 work grid
  return ((long)k * N + j) * N + i;
}

// line of axis a through node (i, j, k): off-axis indices (o1 < o2 in axis order)
__device__ __forceinline__ int line_key(int N, int a, int i, int j, int k) {
  return a == 0 ? j + (N + 1) * k : (a == 1 ? i + (N + 1) * k : i + (N + 1) * j);
}

// ------------------------------------------------------------------- labels
// parity along every line of axis a; a == 0 writes the labels, a = 1, 2 compare
__global__ void labels3_kernel(int N, int a, const int* __restrict__ ptr, const int* __restrict__ pts,
                               const int* __restrict__ edge, uint8_t* inside, int* err) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= (N + 1) * (N + 1)) return;
  const int o1 = L % (N + 1), o2 = L / (N + 1);
  int q = ptr[L];
  const int qe = ptr[L + 1];
  int par = 0;
  for (int t = 0; t <= N; ++t) {
    while (q < qe && edge[pts[q]] < t) { par ^= 1; ++q; }
    int i, j, k;
    if (a == 0) { i = t; j = o1; k = o2; }
    else if (a == 1) { i = o1; j = t; k = o2; }
    else { i = o1; j = o2; k = t; }
    const long g = gidx3(N, i, j, k);
    if (a == 0) inside[g] = (uint8_t)par;
    else if (inside[g] != par) atomicOr(err, ERR3_LABELS);
  }
}

__global__ void band3_kernel(int N, const uint8_t* __restrict__ inside, int* err, int* n_in) {
  const long n = (long)(N + 1) * (N + 1) * (N + 1);
  int cnt = 0;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n; g += (long)gridDim.x * blockDim.x) {
    if (!inside[g]) continue;
    ++cnt;
    const int i = (int)(g % (N + 1)), j = (int)((g / (N + 1)) % (N + 1)), k = (int)(g / ((long)(N + 1) * (N + 1)));
    if (min(i, min(j, k)) <= 2 || max(i, max(j, k)) >= N - 2) atomicOr(err, ERR3_BAND);
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_in, cnt);
}

// ------------------------------------------------------------------- irregular nodes
// 6-neighbour label changes of interior node (i, j, k): bit d for +x, -x, +y, -y, +z, -z
__device__ __forceinline__ int arm_mask3(int N, const uint8_t* in, int i, int j, int k) {
  const uint8_t c = in[gidx3(N, i, j, k)];
  int m = 0;
  m |= (in[gidx3(N, i + 1, j, k)] != c) << 0;
  m |= (in[gidx3(N, i - 1, j, k)] != c) << 1;
  m |= (in[gidx3(N, i, j + 1, k)] != c) << 2;
  m |= (in[gidx3(N, i, j - 1, k)] != c) << 3;
  m |= (in[gidx3(N, i, j, k + 1)] != c) << 4;
  m |= (in[gidx3(N, i, j, k - 1)] != c) << 5;
  return m;
}

// one warp per interior x-line (j, k): counts of irregular nodes and arms
__global__ void irr3_count_kernel(int N, const uint8_t* __restrict__ inside, int* nodes, int* arms) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nl = (N - 1) * (N - 1);
  if (w >= nl) return;
  const int j = 1 + w % (N - 1), k = 1 + w / (N - 1);
  int nn = 0, na = 0;
  for (int i = 1 + lane; i < N; i += 32) {
    const int m = arm_mask3(N, inside, i, j, k);
    nn += m != 0;
    na += __popc(m);
  }
  for (int o = 16; o > 0; o >>= 1) {
    nn += __shfl_down_sync(0xffffffffu, nn, o);
    na += __shfl_down_sync(0xffffffffu, na, o);
  }
  if (lane == 0) { nodes[w] = nn; arms[w] = na; }
}

// the point on edge e of the line `key` of axis a (exactly one, else -1)
__device__ int edge_point(const int* ptr, const int* pts, const int* edge, int key, int e) {
  int lo = ptr[key], hi = ptr[key + 1];
  while (lo < hi) {                      // first point with edge >= e
    const int mid = (lo + hi) >> 1;
    if (edge[pts[mid]] < e) lo = mid + 1; else hi = mid;
  }
  if (lo >= ptr[key + 1] || edge[pts[lo]] != e) return -1;
  if (lo + 1 < ptr[key + 1] && edge[pts[lo + 1]] == e) return -1;
  return pts[lo];
}

struct Lines3 {
  const int* ptr[3];
  const int* pts[3];
};

__global__ void irr3_fill_kernel(int N, double lo, double h, const uint8_t* __restrict__ inside,
                                 const int* node_off, const int* arm_off, Lines3 L,
                                 const int* __restrict__ edge, const double* __restrict__ X,
                                 int* irr_node, double* irr_sigma, int* arm_ptr, int* arm_pt,
                                 int* arm_axis, double* arm_delta, int* err) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nl = (N - 1) * (N - 1);
  if (w >= nl) return;
  const int j = 1 + w % (N - 1), k = 1 + w / (N - 1);
  int bn = node_off[w], ba = arm_off[w];
  for (int i0 = 1; i0 < N; i0 += 32) {
    const int i = i0 + lane;
    const int m = i < N ? arm_mask3(N, inside, i, j, k) : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, m != 0);
    int na = __popc(m);
    int pa = na;                                  // inclusive prefix of arm counts
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, pa, o);
      if (lane >= o) pa += t;
    }
    const int tot_a = __shfl_sync(0xffffffffu, pa, 31);
    if (m) {
      const int n = bn + __popc(bal & ((1u << lane) - 1u));
      int a = ba + pa - na;
      const bool in = inside[gidx3(N, i, j, k)] != 0;
      irr_node[n] = (int)widx3(N, i, j, k);
      irr_sigma[n] = in ? -1.0 : 1.0;
      arm_ptr[n] = a;
      const int node[3] = {i, j, k};
      for (int d = 0; d < 6; ++d) {
        if (!(m & (1 << d))) continue;
        const int ax = d >> 1, sg = (d & 1) ? -1 : 1;
        const int e = sg > 0 ? node[ax] : node[ax] - 1;
        const int key = line_key(N, ax, i, j, k);
        const int q = edge_point(L.ptr[ax], L.pts[ax], edge, key, e);
        if (q < 0) { atomicOr(err, ERR3_ARM); arm_pt[a] = 0; }
        else arm_pt[a] = q;
        arm_axis[a] = ax;
        arm_delta[a] = (lo + (node[ax] + sg) * h) - (q < 0 ? 0.0 : X[3 * q + ax]);
        ++a;
      }
    }
    bn += __popc(bal);
    ba += tot_a;
  }
}

// ------------------------------------------------------------------- least squares
__device__ __forceinline__ void frame_of(const double* n, double* t1, double* t2) {
  const double ax = fabs(n[0]), ay = fabs(n[1]), az = fabs(n[2]);
  const int e = (ax <= ay && ax <= az) ? 0 : (ay <= az ? 1 : 2);   // least aligned, lowest first
  double u[3];
  if (e == 0) { u[0] = 0.0; u[1] = -n[2]; u[2] = n[1]; }           // e_x x n
  else if (e == 1) { u[0] = n[2]; u[1] = 0.0; u[2] = -n[0]; }      // e_y x n
  else { u[0] = -n[1]; u[1] = n[0]; u[2] = 0.0; }                  // e_z x n
  const double s = 1.0 / sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  t1[0] = u[0] * s; t1[1] = u[1] * s; t1[2] = u[2] * s;
  t2[0] = n[1] * t1[2] - n[2] * t1[1];
  t2[1] = n[2] * t1[0] - n[0] * t1[2];
  t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

// visit every point within radius r of X (all three line families); f(q) per hit
template <typename F>
__device__ void for_neighbours(int N, double lo, double h, const double* __restrict__ XP,
                               const Lines3& L, const double* Xp, double r, F&& f) {
  const double r2 = r * r * (1.0 + 2e-12);
  for (int a = 0; a < 3; ++a) {
    const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
    const int i1a = max(0, (int)ceil((Xp[o1] - r - lo) / h)), i1b = min(N, (int)floor((Xp[o1] + r - lo) / h));
    const int i2a = max(0, (int)ceil((Xp[o2] - r - lo) / h)), i2b = min(N, (int)floor((Xp[o2] + r - lo) / h));
    for (int i2 = i2a; i2 <= i2b; ++i2)
      for (int i1 = i1a; i1 <= i1b; ++i1) {
        const int key = i1 + (N + 1) * i2;
        int qa = L.ptr[a][key], qb = L.ptr[a][key + 1];
        while (qa < qb) {                 // first point with along >= X_a - r
          const int mid = (qa + qb) >> 1;
          if (XP[3 * L.pts[a][mid] + a] < Xp[a] - r) qa = mid + 1; else qb = mid;
        }
        for (int m = qa; m < L.ptr[a][key + 1]; ++m) {
          const int q = L.pts[a][m];
          const double dx = XP[3 * q] - Xp[0], dy = XP[3 * q + 1] - Xp[1], dz = XP[3 * q + 2] - Xp[2];
          if (XP[3 * q + a] > Xp[a] + r) break;
          if (dx * dx + dy * dy + dz * dz <= r2) f(q, dx, dy, dz);
        }
      }
  }
}

__global__ void ls_count_kernel(int P, int N, double lo, double h, const double* __restrict__ X,
                                Lines3 L, int* cnt, double* radius, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double Xp[3] = {X[3 * p], X[3 * p + 1], X[3 * p + 2]};
  int c = 0;
  double r = LS_R * h;
  for_neighbours(N, lo, h, X, L, Xp, r, [&](int, double, double, double) { ++c; });
  if (c < LS_MIN) {
    r = LS_R_WIDE * h;
    c = 0;
    for_neighbours(N, lo, h, X, L, Xp, r, [&](int, double, double, double) { ++c; });
  }
  if (c < LS_MIN) atomicOr(err, ERR3_LS);
  cnt[p] = c;
  radius[p] = r;
}

// Normal equations G = A^T A of the quadratic fit, Cholesky, and per neighbour the six
// weights G^{-1} a_q (a_q = [1, a, b, a^2, a b, b^2]); frames t1, t2 stored per point.
__global__ void ls_fill_kernel(int P, int N, double lo, double h, const double* __restrict__ X,
                               const double* __restrict__ nrm, Lines3 L, const int* ptr,
                               const double* radius, int* idx, double* wts, double* frame, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double Xp[3] = {X[3 * p], X[3 * p + 1], X[3 * p + 2]};
  const double n[3] = {nrm[3 * p], nrm[3 * p + 1], nrm[3 * p + 2]};
  double t1[3], t2[3];
  frame_of(n, t1, t2);
  for (int d = 0; d < 3; ++d) { frame[6 * p + d] = t1[d]; frame[6 * p + 3 + d] = t2[d]; }
  const double inv_h = 1.0 / h;
  double G[21] = {0.0};                     // packed lower triangle, row-major
  auto row = [&](double dx, double dy, double dz, double* v) {
    const double a = (dx * t1[0] + dy * t1[1] + dz * t1[2]) * inv_h;
    const double b = (dx * t2[0] + dy * t2[1] + dz * t2[2]) * inv_h;
    v[0] = 1.0; v[1] = a; v[2] = b; v[3] = a * a; v[4] = a * b; v[5] = b * b;
  };
  for_neighbours(N, lo, h, X, L, Xp, radius[p], [&](int, double dx, double dy, double dz) {
    double v[6];
    row(dx, dy, dz, v);
    int e = 0;
    for (int r = 0; r < 6; ++r)
      for (int s = 0; s <= r; ++s) G[e++] += v[r] * v[s];
  });
  // Cholesky G = C C^T (lower triangular, packed like G)
  double C[21];
  bool ok = true;
  for (int r = 0; r < 6; ++r) {
    for (int s = 0; s <= r; ++s) {
      double sum = G[r * (r + 1) / 2 + s];
      for (int t = 0; t < s; ++t) sum -= C[r * (r + 1) / 2 + t] * C[s * (s + 1) / 2 + t];
      if (r == s) {
        if (!(sum > 0.0)) { ok = false; sum = 1.0; }
        C[r * (r + 1) / 2 + r] = sqrt(sum);
      } else {
        C[r * (r + 1) / 2 + s] = sum / C[s * (s + 1) / 2 + s];
      }
    }
  }
  if (!ok) atomicOr(err, ERR3_LS);
  int m = ptr[p];
  for_neighbours(N, lo, h, X, L, Xp, radius[p], [&](int q, double dx, double dy, double dz) {
    double v[6], y[6];
    row(dx, dy, dz, v);
    for (int r = 0; r < 6; ++r) {           // C y = v
      double sum = v[r];
      for (int t = 0; t < r; ++t) sum -= C[r * (r + 1) / 2 + t] * y[t];
      y[r] = sum / C[r * (r + 1) / 2 + r];
    }
    for (int r = 5; r >= 0; --r) {          // C^T w = y
      double sum = y[r];
      for (int t = r + 1; t < 6; ++t) sum -= C[t * (t + 1) / 2 + r] * y[t];
      y[r] = sum / C[r * (r + 1) / 2 + r];
    }
    idx[m] = q;
    for (int r = 0; r < 6; ++r) wts[6 * (long)m + r] = y[r];
    ++m;
  });
}

// ------------------------------------------------------------------- interpolation stencils
// 10 nodes c, c +- e_a, c + s_a e_a + s_b e_b; closed-form weights of the quadratic through
// them at z; moments of the outside nodes (e0 = sum w, e1 = sum w d, e2 = sum w d d^T with
// d = node - z) for the Taylor terms of the jump.
__global__ void interp3_kernel_setup(int P, int N, double lo, double h, const double* __restrict__ X,
                                     const uint8_t* __restrict__ inside, int* nodes, double* w,
                                     double* mom, int* err) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int c[3], s[3];
  double d[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = (int)floor((X[3 * p + a] - lo) / h + 0.5);
    s[a] = (X[3 * p + a] >= lo + c[a] * h) ? 1 : -1;
    d[a] = (X[3 * p + a] - (lo + c[a] * h)) / h;
  }
  int off[10][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
                    {s[0], s[1], 0}, {s[0], 0, s[2]}, {0, s[1], s[2]}};
  const double pxy = d[0] * d[1] * s[0] * s[1], pxz = d[0] * d[2] * s[0] * s[2],
               pyz = d[1] * d[2] * s[1] * s[2];
  const double pa[3] = {pxy + pxz, pxy + pyz, pxz + pyz};   // sum over b != a of p_ab
  double wt[10];
  wt[0] = 1.0 - d[0] * d[0] - d[1] * d[1] - d[2] * d[2] + pxy + pxz + pyz;
  for (int a = 0; a < 3; ++a) {
    wt[1 + 2 * a] = 0.5 * d[a] + 0.5 * d[a] * d[a] - 0.5 * (s[a] + 1) * pa[a];
    wt[2 + 2 * a] = -0.5 * d[a] + 0.5 * d[a] * d[a] + 0.5 * (s[a] - 1) * pa[a];
  }
  wt[7] = pxy; wt[8] = pxz; wt[9] = pyz;
  double e0 = 0.0, e1[3] = {0.0, 0.0, 0.0}, e2[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int t = 0; t < 10; ++t) {
    const int i = c[0] + off[t][0], j = c[1] + off[t][1], k = c[2] + off[t][2];
    if (i < 1 || j < 1 || k < 1 || i > N - 1 || j > N - 1 || k > N - 1) {
      atomicOr(err, ERR3_STENCIL);
      nodes[10 * p + t] = 0;
      w[10 * p + t] = 0.0;
      continue;
    }
    nodes[10 * p + t] = (int)widx3(N, i, j, k);
    w[10 * p + t] = wt[t];
    if (!inside[gidx3(N, i, j, k)]) {
      const double dd[3] = {lo + i * h - X[3 * p], lo + j * h - X[3 * p + 1], lo + k * h - X[3 * p + 2]};
      e0 += wt[t];
      for (int a = 0; a < 3; ++a) e1[a] += wt[t] * dd[a];
      e2[0] += wt[t] * dd[0] * dd[0]; e2[1] += wt[t] * dd[1] * dd[1]; e2[2] += wt[t] * dd[2] * dd[2];
      e2[3] += wt[t] * dd[0] * dd[1]; e2[4] += wt[t] * dd[0] * dd[2]; e2[5] += wt[t] * dd[1] * dd[2];
    }
  }
  mom[10 * p] = e0;
  for (int a = 0; a < 3; ++a) mom[10 * p + 1 + a] = e1[a];
  for (int a = 0; a < 6; ++a) mom[10 * p + 4 + a] = e2[a];
}

// ------------------------------------------------------------------- per-apply kernels
// Jumps at every point: fitted value, surface gradient and Hessian of the density (and
// of psi, for the single layer) from the least-squares weights, [F] from f on Gamma, in
// Cartesian axes: jmp[10 p ..] = J, Gx, Gy, Gz, Hxx, Hyy, Hzz, Hxy, Hxz, Hyz.
__global__ void jumps3_kernel(int P, double h, double kappa2, const int* __restrict__ ptr,
                              const int* __restrict__ idx, const double* __restrict__ wts,
                              const double* __restrict__ nrm, const double* __restrict__ shape,
                              const double* __restrict__ frame, const double* __restrict__ dens,
                              const double* __restrict__ psi, const double* __restrict__ fctl,
                              double* jmp, double* fit) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double c[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  double cp[3] = {0.0, 0.0, 0.0};     // fitted psi: value and the two tangential slopes
  if (dens)
    for (int m = ptr[p]; m < ptr[p + 1]; ++m) {
      const double v = dens[idx[m]];
      for (int r = 0; r < 6; ++r) c[r] += wts[6 * (long)m + r] * v;
    }
  if (psi)
    for (int m = ptr[p]; m < ptr[p + 1]; ++m) {
      const double v = psi[idx[m]];
      for (int r = 0; r < 3; ++r) cp[r] += wts[6 * (long)m + r] * v;
    }
  const double Fj = fctl ? fctl[p] : 0.0;
  const double n[3] = {nrm[3 * p], nrm[3 * p + 1], nrm[3 * p + 2]};
  const double t[2][3] = {{frame[6 * p], frame[6 * p + 1], frame[6 * p + 2]},
                          {frame[6 * p + 3], frame[6 * p + 4], frame[6 * p + 5]}};
  const double* sp = shape + 6 * p;
  const double S[3][3] = {{sp[0], sp[3], sp[4]}, {sp[3], sp[1], sp[5]}, {sp[4], sp[5], sp[2]}};
  const double inv_h = 1.0 / h;
  const double g1 = c[1] * inv_h, g2 = c[2] * inv_h;
  const double H11 = 2.0 * c[3] * inv_h * inv_h, H12 = c[4] * inv_h * inv_h,
               H22 = 2.0 * c[5] * inv_h * inv_h;
  double gG[3];
  for (int a = 0; a < 3; ++a) gG[a] = g1 * t[0][a] + g2 * t[1][a];
  double SgG[3];
  for (int a = 0; a < 3; ++a) SgG[a] = S[a][0] * gG[0] + S[a][1] * gG[1] + S[a][2] * gG[2];
  // single layer: [v_n] = psi~, the tangential block gains psi~ II (II_su = t_s . S t_u), the
  // mixed terms the tangential gradient of psi, the normal-normal term -tr(S) psi~
  const double ps = cp[0];
  double II[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double v = 0.0;
      for (int q = 0; q < 3; ++q)
        for (int r = 0; r < 3; ++r) v += t[a][q] * S[q][r] * t[b][r];
      II[a][b] = v;
    }
  const double mixed[2] = {cp[1] * inv_h - (t[0][0] * SgG[0] + t[0][1] * SgG[1] + t[0][2] * SgG[2]),
                           cp[2] * inv_h - (t[1][0] * SgG[0] + t[1][1] * SgG[1] + t[1][2] * SgG[2])};
  const double tan_[2][2] = {{H11 + ps * II[0][0], H12 + ps * II[0][1]},
                             {H12 + ps * II[1][0], H22 + ps * II[1][1]}};
  const double nn = Fj + kappa2 * c[0] - (H11 + H22) - (S[0][0] + S[1][1] + S[2][2]) * ps;
  for (int a = 0; a < 3; ++a) gG[a] += ps * n[a];
  double H[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = nn * n[a] * n[b];
      for (int s = 0; s < 2; ++s) v += mixed[s] * (n[a] * t[s][b] + t[s][a] * n[b]);
      for (int s = 0; s < 2; ++s)
        for (int u = 0; u < 2; ++u) v += tan_[s][u] * t[s][a] * t[u][b];
      H[a][b] = v;
    }
  double* o = jmp + 10 * (long)p;
  o[0] = c[0];
  o[1] = gG[0]; o[2] = gG[1]; o[3] = gG[2];
  o[4] = H[0][0]; o[5] = H[1][1]; o[6] = H[2][2]; o[7] = H[0][1]; o[8] = H[0][2]; o[9] = H[1][2];
  if (fit) fit[p] = c[0];
}

// b[node] (+)= sigma sum_arms (J + d [v_a] + d^2/2 [v_aa])(q) / h^2 (Alg. 2)
template <typename T>
__global__ void correction3_kernel(int nirr, double inv_h2, const int* __restrict__ irr_node,
                                   const double* __restrict__ sigma, const int* __restrict__ arm_ptr,
                                   const int* __restrict__ arm_pt, const int* __restrict__ arm_axis,
                                   const double* __restrict__ arm_delta, const double* __restrict__ jmp,
                                   T* B, int add, double* B64) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nirr) return;
  double s = 0.0;
  for (int a = arm_ptr[n]; a < arm_ptr[n + 1]; ++a) {
    const double* J = jmp + 10 * (long)arm_pt[a];
    const int ax = arm_axis[a];
    const double d = arm_delta[a];
    s += J[0] + d * J[1 + ax] + 0.5 * d * d * J[4 + ax];
  }
  const double b = sigma[n] * s * inv_h2;
  const int node = irr_node[n];
  if (add) B[node] = (T)((double)B[node] + b);
  else B[node] = (T)b;
  if (B64) B64[node] = b;
}

// v^+ at every point from the 10 node values and the outside-node Taylor moments; for
// the double-layer apply out = v^+ + (phi - fitted phi) / 2
template <typename T>
__global__ void interp3_kernel(int P, const int* __restrict__ nodes, const double* __restrict__ w,
                               const double* __restrict__ mom, const double* __restrict__ jmp,
                               const T* __restrict__ V, const float* __restrict__ V2,
                               const float* __restrict__ V3, const double* __restrict__ dens,
                               const double* __restrict__ fit, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double acc = 0.0;
  for (int t = 0; t < 10; ++t) {
    const int q = nodes[10 * (long)p + t];
    double v = (double)V[q];
    if (V2) v += (double)V2[q];
    if (V3) v += (double)V3[q];
    acc += w[10 * (long)p + t] * v;
  }
  const double* e = mom + 10 * (long)p;
  const double* J = jmp + 10 * (long)p;
  acc += e[0] * J[0] + e[1] * J[1] + e[2] * J[2] + e[3] * J[3] +
         0.5 * (e[4] * J[4] + e[5] * J[5] + e[6] * J[6]) + e[7] * J[7] + e[8] * J[8] + e[9] * J[9];
  if (dens) acc += 0.5 * (dens[p] - fit[p]);
  out[p] = acc;
}

// ------------------------------------------------------------------- refinement
__device__ __forceinline__ void two_sum3(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct Pair3 {
  float hi, lo;
};
__device__ __forceinline__ Pair3 at3(const float* c1, const float* c2, long q) {
  if (!c2) return {c1[q], 0.f};
  Pair3 p;
  two_sum3(c1[q], c2[q], p.hi, p.lo);
  return p;
}

// r = b - (Lap_h - kappa^2) v on the N^3 work grid, v = c1 (+ c2), b = bhi + blo (dense)
// or 0 (bhi == nullptr), kappa^2 = k2hi + k2lo exactly: the 7-point sum and every product
// that can cancel are carried as exact FP32 pairs (6 v_c = 4 v_c + 2 v_c, both exact);
// only the final residual is rounded.
__global__ void ds_residual3_kernel(int N, float inv_h2, float k2hi, float k2lo,
                                    const float* __restrict__ bhi, const float* __restrict__ blo,
                                    const float* __restrict__ c1, const float* __restrict__ c2,
                                    float* __restrict__ r) {
  const long n = (long)N * N * N, NN = (long)N * N;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int i = (int)(q % N), j = (int)((q / N) % N), k = (int)(q / NN);
    if (i == 0 || j == 0 || k == 0) {
      r[q] = 0.f;
      continue;
    }
    const Pair3 z = {0.f, 0.f};
    const Pair3 vc = at3(c1, c2, q);
    const Pair3 v0 = (i + 1 < N) ? at3(c1, c2, q + 1) : z, v1 = at3(c1, c2, q - 1);
    const Pair3 v2 = (j + 1 < N) ? at3(c1, c2, q + N) : z, v3 = at3(c1, c2, q - N);
    const Pair3 v4 = (k + 1 < N) ? at3(c1, c2, q + NN) : z, v5 = at3(c1, c2, q - NN);
    float s1, t1, s2, t2, s3, t3, s4, t4, s5, t5, s6, t6, s7, t7;
    two_sum3(v0.hi, v1.hi, s1, t1);
    two_sum3(v2.hi, v3.hi, s2, t2);
    two_sum3(v4.hi, v5.hi, s3, t3);
    two_sum3(s1, s2, s4, t4);
    two_sum3(s4, s3, s5, t5);
    two_sum3(s5, -4.f * vc.hi, s6, t6);
    two_sum3(s6, -2.f * vc.hi, s7, t7);
    const float lo = (((t1 + t2) + (t3 + t4)) + ((t5 + t6) + t7)) +
                     (((v0.lo + v1.lo) + (v2.lo + v3.lo)) + (v4.lo + v5.lo) - 6.f * vc.lo);
    const float p1 = s7 * inv_h2;
    const float e1 = fmaf(s7, inv_h2, -p1) + lo * inv_h2;
    const float p2 = k2hi * vc.hi;
    const float e2 = fmaf(k2hi, vc.hi, -p2) + (k2hi * vc.lo + k2lo * vc.hi);
    float d, de;
    two_sum3(p2, -p1, d, de);
    float tail = de - e1 + e2;
    if (bhi) {
      float d2, de2;
      two_sum3(bhi[q], d, d2, de2);
      d = d2;
      tail += de2 + blo[q];
    }
    r[q] = d + tail;
  }
}

// the residual at the irregular nodes in FP64 against the sparse FP64 right-hand side
__global__ void residual_fix3_kernel(int nirr, int N, double inv_h2, double kappa2,
                                     const int* __restrict__ irr_node, const double* __restrict__ b,
                                     const float* __restrict__ c1, const float* __restrict__ c2,
                                     float* __restrict__ r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nirr) return;
  const long q = irr_node[t], NN = (long)N * N;
  const int i = (int)(q % N), j = (int)((q / N) % N), k = (int)(q / NN);
  auto v = [&](long p) { return (double)c1[p] + (c2 ? (double)c2[p] : 0.0); };
  const double s = (i + 1 < N ? v(q + 1) : 0.0) + v(q - 1) + (j + 1 < N ? v(q + N) : 0.0) +
                   v(q - N) + (k + 1 < N ? v(q + NN) : 0.0) + v(q - NN);
  const double vc = v(q);
  r[q] = (float)(b[q] - ((s - 6.0 * vc) * inv_h2 - kappa2 * vc));
}

__global__ void split3_kernel(long n, const double* __restrict__ b, float* __restrict__ hi,
                              float* __restrict__ lo) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    float h, l;
    f64_to_f32_pair(b[q], h, l);                 // integer operations, not the FP64 pipe
    hi[q] = h;
    lo[q] = l;
  }
}

// v = w1 (+ w2 + w3) summed in FP64
__global__ void sum3_kernel(long n, const float* __restrict__ w1, const float* __restrict__ w2,
                            const float* __restrict__ w3, double* __restrict__ out) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    out[q] = f32_to_f64(w1[q]) + (w2 ? f32_to_f64(w2[q]) : 0.0) + (w3 ? f32_to_f64(w3[q]) : 0.0);
}

// dense right-hand side: F~ (f inside Omega, 0 outside) on the N^3 work grid
template <typename T>
__global__ void rhs_dense3_kernel(int N, const double* __restrict__ f, const uint8_t* __restrict__ inside,
                                  T* W) {
  const long n = (long)N * N * N;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int i = (int)(q % N), j = (int)((q / N) % N), k = (int)(q / ((long)N * N));
    const long g = gidx3(N, i, j, k);
    W[q] = (i > 0 && j > 0 && k > 0 && inside[g]) ? (T)f[g] : T(0);
  }
}

template <typename T>
__global__ void grid_to_work3_kernel(int N, const double* __restrict__ G, T* W) {
  const long n = (long)N * N * N;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int i = (int)(q % N), j = (int)((q / N) % N), k = (int)(q / ((long)N * N));
    W[q] = (i > 0 && j > 0 && k > 0) ? (T)G[gidx3(N, i, j, k)] : T(0);
  }
}

__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f32_to_f64(x); }   // exact, integer ops

template <typename T>
__global__ void work_to_grid3_kernel(int N, const T* __restrict__ W, const uint8_t* __restrict__ mask,
                                     double* G) {
  const long n = (long)(N + 1) * (N + 1) * (N + 1);
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n; g += (long)gridDim.x * blockDim.x) {
    const int i = (int)(g % (N + 1)), j = (int)((g / (N + 1)) % (N + 1)), k = (int)(g / ((long)(N + 1) * (N + 1)));
    double v = (i < N && j < N && k < N) ? to_f64(W[widx3(N, i, j, k)]) : 0.0;
    if (mask && !mask[g]) v = 0.0;
    G[g] = v;
  }
}

__global__ void copy_bytes_kernel(long n, const uint8_t* in, uint8_t* out) {
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x)
    out[k] = in[k];
}

__global__ void convert_kernel3(long n, const double* __restrict__ in, float* out) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    out[q] = (float)in[q];
}

inline int grid_blocks(long n) {
  const long b = (n + 255) / 256;
  return (int)(b < 8192 ? (b < 1 ? 1 : b) : 8192);
}

template <typename T>
kfbi_status upload(Ctx& c, T** dst, const std::vector<T>& v) {
  KFBI_TRY(alloc_bytes(c, (void**)dst, sizeof(T) * (v.size() ? v.size() : 1)));
  if (!v.empty())
    KFBI_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, c.stream));
  return KFBI_OK;
}

kfbi_status exclusive_scan_host(Ctx& c, const int* d_in, int n, int** d_out, int* total) {
  std::vector<int> h(n + 1, 0);
  if (n > 0) KFBI_CUDA_TRY(cudaMemcpyAsync(h.data(), d_in, sizeof(int) * n, cudaMemcpyDeviceToHost, c.stream));
  KFBI_CUDA_TRY(cudaStreamSynchronize(c.stream));
  int run = 0;
  for (int i = 0; i < n; ++i) { const int v = h[i]; h[i] = run; run += v; }
  h[n] = run;
  *total = run;
  return upload(c, d_out, h);
}

}  // namespace

// ============================================================================ setup
kfbi_status setup_geometry3(Ctx& c) {
  const int N = c.N, P = c.M;
  const double lo = c.lo, h = c.h;
  cudaStream_t st = c.stream;
  // ---- tags (host): axis, off-axis node indices, edge
  std::vector<double> X(3 * (size_t)P);
  KFBI_CUDA_TRY(cudaMemcpyAsync(X.data(), c.pts, sizeof(double) * 3 * P, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int> axis(P), key(P), edge(P);
  for (int p = 0; p < P; ++p) {
    double g[3];
    bool on[3];
    for (int a = 0; a < 3; ++a) {
      g[a] = (X[3 * p + a] - lo) / h;
      on[a] = std::fabs(g[a] - std::nearbyint(g[a])) <= TAG_TOL;
    }
    int ax = -1, hits = 0;
    for (int a = 0; a < 3; ++a) {
      const int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
      if (on[o1] && on[o2] && !on[a]) { ax = a; ++hits; }
    }
    if (hits != 1) {
      set_error("kfbi_setup: point %d lies on no grid line or on a grid node", p);
      return KFBI_ERR_GEOMETRY;
    }
    const int o1 = ax == 0 ? 1 : 0, o2 = ax == 2 ? 1 : 2;
    const int i1 = (int)std::nearbyint(g[o1]), i2 = (int)std::nearbyint(g[o2]);
    const int e = (int)std::floor(g[ax]);
    if (e < 0 || e >= N || i1 < 0 || i1 > N || i2 < 0 || i2 > N) {
      set_error("kfbi_setup: point %d lies outside the box", p);
      return KFBI_ERR_GEOMETRY;
    }
    axis[p] = ax;
    key[p] = i1 + (N + 1) * i2;
    edge[p] = e;
  }
  // ---- per-axis line CSR, points sorted by (line, along)
  const int nlines = (N + 1) * (N + 1);
  Lines3 L{};
  for (int a = 0; a < 3; ++a) {
    std::vector<int> ids;
    for (int p = 0; p < P; ++p)
      if (axis[p] == a) ids.push_back(p);
    std::sort(ids.begin(), ids.end(), [&](int u, int v) {
      if (key[u] != key[v]) return key[u] < key[v];
      return X[3 * u + a] < X[3 * v + a];
    });
    std::vector<int> ptr(nlines + 1, 0);
    for (int p : ids) ptr[key[p] + 1]++;
    for (int l = 0; l < nlines; ++l) ptr[l + 1] += ptr[l];
    c.npts_axis[a] = (int)ids.size();
    KFBI_TRY(upload(c, &c.l3_ptr[a], ptr));
    KFBI_TRY(upload(c, &c.l3_pts[a], ids));
    L.ptr[a] = c.l3_ptr[a];
    L.pts[a] = c.l3_pts[a];
  }
  KFBI_TRY(upload(c, &c.pt_edge, edge));
  int* err = c.err_flag;
  KFBI_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int) * 4, st));
  // ---- labels
  const long ngrid = (long)(N + 1) * (N + 1) * (N + 1);
  KFBI_TRY(alloc_bytes(c, (void**)&c.inside, ngrid));
  for (int a = 0; a < 3; ++a) {
    prof_count(c, ST_SETUP);
    labels3_kernel<<<nblk(nlines, 128), 128, 0, st>>>(N, a, L.ptr[a], L.pts[a], c.pt_edge, c.inside, err);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  prof_count(c, ST_SETUP);
  band3_kernel<<<grid_blocks(ngrid), 256, 0, st>>>(N, c.inside, err, err + 1);
  KFBI_CUDA_TRY(cudaGetLastError());
  // ---- irregular nodes and arms
  const int nl = (N - 1) * (N - 1);
  int *cnt_n = nullptr, *cnt_a = nullptr, *off_n = nullptr, *off_a = nullptr;
  KFBI_TRY(alloc_bytes(c, (void**)&cnt_n, sizeof(int) * nl));
  KFBI_TRY(alloc_bytes(c, (void**)&cnt_a, sizeof(int) * nl));
  prof_count(c, ST_SETUP);
  irr3_count_kernel<<<nblk((long)nl * 32, 256), 256, 0, st>>>(N, c.inside, cnt_n, cnt_a);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_TRY(exclusive_scan_host(c, cnt_n, nl, &off_n, &c.nirr));
  KFBI_TRY(exclusive_scan_host(c, cnt_a, nl, &off_a, &c.narms));
  KFBI_TRY(alloc_bytes(c, (void**)&c.irr_node, sizeof(int) * (c.nirr + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.irr_sigma, sizeof(double) * (c.nirr + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm_ptr, sizeof(int) * (c.nirr + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm3_pt, sizeof(int) * (c.narms + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm3_axis, sizeof(int) * (c.narms + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.arm3_delta, sizeof(double) * (c.narms + 1)));
  prof_count(c, ST_SETUP);
  irr3_fill_kernel<<<nblk((long)nl * 32, 256), 256, 0, st>>>(
      N, lo, h, c.inside, off_n, off_a, L, c.pt_edge, c.pts, c.irr_node, c.irr_sigma, c.arm_ptr,
      c.arm3_pt, c.arm3_axis, c.arm3_delta, err);
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_CUDA_TRY(cudaMemcpyAsync(c.arm_ptr + c.nirr, &c.narms, sizeof(int), cudaMemcpyHostToDevice, st));
  // ---- least-squares stencils and frames
  int* ls_cnt = nullptr;
  double* radius = nullptr;
  KFBI_TRY(alloc_bytes(c, (void**)&ls_cnt, sizeof(int) * P));
  KFBI_TRY(alloc_bytes(c, (void**)&radius, sizeof(double) * P));
  prof_count(c, ST_SETUP);
  ls_count_kernel<<<nblk(P, 128), 128, 0, st>>>(P, N, lo, h, c.pts, L, ls_cnt, radius, err);
  KFBI_CUDA_TRY(cudaGetLastError());
  int nls = 0;
  KFBI_TRY(exclusive_scan_host(c, ls_cnt, P, &c.ls_ptr, &nls));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ls_idx, sizeof(int) * (nls + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ls_w, sizeof(double) * 6 * ((size_t)nls + 1)));
  KFBI_TRY(alloc_bytes(c, (void**)&c.frame, sizeof(double) * 6 * P));
  prof_count(c, ST_SETUP);
  ls_fill_kernel<<<nblk(P, 128), 128, 0, st>>>(P, N, lo, h, c.pts, c.nrm, L, c.ls_ptr, radius,
                                               c.ls_idx, c.ls_w, c.frame, err);
  KFBI_CUDA_TRY(cudaGetLastError());
  // ---- interpolation stencils
  KFBI_TRY(alloc_bytes(c, (void**)&c.ip_node, sizeof(int) * 10 * P));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ip_w, sizeof(double) * 10 * P));
  KFBI_TRY(alloc_bytes(c, (void**)&c.ip_mom, sizeof(double) * 10 * P));
  KFBI_TRY(alloc_bytes(c, (void**)&c.jmp3, sizeof(double) * 10 * P));
  KFBI_TRY(alloc_bytes(c, (void**)&c.fit3, sizeof(double) * P));
  prof_count(c, ST_SETUP);
  interp3_kernel_setup<<<nblk(P, 128), 128, 0, st>>>(P, N, lo, h, c.pts, c.inside, c.ip_node,
                                                     c.ip_w, c.ip_mom, err);
  KFBI_CUDA_TRY(cudaGetLastError());
  int h_err[2];
  KFBI_CUDA_TRY(cudaMemcpyAsync(h_err, err, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
  KFBI_CUDA_TRY(cudaStreamSynchronize(st));
  c.n_inside = h_err[1];
  const int e = h_err[0];
  if (e) {
    set_error("kfbi_setup: %s",
              (e & ERR3_LABELS) ? "node labels from x-, y- and z-lines disagree (a point missing?)"
              : (e & ERR3_BAND) ? "interface within two cells of the box boundary"
              : (e & ERR3_ARM) ? "an edge with a label change does not hold exactly one point"
              : (e & ERR3_LS) ? "fewer than 10 points near a point (surface under-resolved)"
                              : "interpolation stencil leaves the interior of the box");
    return KFBI_ERR_GEOMETRY;
  }
  return KFBI_OK;
}

// ============================================================================ apply
static kfbi_status jumps3(Ctx& c, const double* dens, const double* fctl, bool fit,
                          const double* psi = nullptr) {
  const int pr = prof_begin(c, ST_CORR);
  jumps3_kernel<<<nblk(c.M, 128), 128, 0, c.stream>>>(c.M, c.h, c.kappa2, c.ls_ptr, c.ls_idx,
                                                      c.ls_w, c.nrm, c.curv, c.frame, dens, psi,
                                                      fctl, c.jmp3, fit ? c.fit3 : nullptr);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T>
static kfbi_status correct3(Ctx& c, T* B, int add, double* B64 = nullptr) {
  if (c.nirr == 0) return KFBI_OK;
  const int pr = prof_begin(c, ST_CORR);
  correction3_kernel<T><<<nblk(c.nirr, 128), 128, 0, c.stream>>>(
      c.nirr, 1.0 / (c.h * c.h), c.irr_node, c.irr_sigma, c.arm_ptr, c.arm3_pt, c.arm3_axis,
      c.arm3_delta, c.jmp3, B, add, B64);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

template <typename T>
static kfbi_status interp3(Ctx& c, const T* V, const double* dens, double* out,
                           const float* V2 = nullptr, const float* V3 = nullptr) {
  const int pr = prof_begin(c, ST_INTERP);
  interp3_kernel<T><<<nblk(c.M, 128), 128, 0, c.stream>>>(c.M, c.ip_node, c.ip_w, c.ip_mom, c.jmp3,
                                                         V, V2, V3, dens, c.fit3, out);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

static int steps_of(int precision) {
  return precision == KFBI_FP32_REFINED ? 2 : (precision == KFBI_FP32_REFINED_ONCE ? 1 : 0);
}

// FP32 solve of b32, then `steps` corrections from the residual of the 7-point system in
// double-single arithmetic against the exact pair (bhi, blo), or (bhi null) against the
// sparse right-hand side, FP64 copy in B64, at the irregular nodes.  v = V32 + U32 (+ T32).
static kfbi_status refined_solve3(Ctx& c, const float* b32, const float* bhi, const float* blo,
                                  int steps) {
  KFBI_TRY(box_solve3_f32(c, b32, c.V32));
  const float inv_h2 = (float)(1.0 / (c.h * c.h));
  const float k2hi = (float)c.kappa2, k2lo = (float)(c.kappa2 - (double)k2hi);
  const long nw = (long)c.N * c.N * c.N;
  for (int s = 0; s < steps; ++s) {
    const float* c2 = s == 0 ? nullptr : c.U32;
    const int pr = prof_begin(c, ST_REFINE);
    ds_residual3_kernel<<<grid_blocks(nw), 256, 0, c.stream>>>(c.N, inv_h2, k2hi, k2lo, bhi, blo,
                                                               c.V32, c2, c.W32);
    if (!bhi && c.nirr > 0)
      residual_fix3_kernel<<<nblk(c.nirr, 128), 128, 0, c.stream>>>(
          c.nirr, c.N, 1.0 / (c.h * c.h), c.kappa2, c.irr_node, c.B64, c.V32, c2, c.W32);
    prof_end(c, pr);
    if (!bhi && c.nirr > 0) prof_count(c, ST_REFINE);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(box_solve3_f32(c, c.W32, s == 0 ? c.U32 : c.T32));
  }
  return KFBI_OK;
}

// FP64 transforms for FP64, FP32 transforms (refined or not) otherwise
static bool use_fp32(int precision) { return precision != KFBI_FP64; }

// plain FP32 box solve: FFT form, or the dense form on the tensor cores for KFBI_TF32X3
static kfbi_status plain_solve3(Ctx& c, int precision, const float* b, float* v) {
  return precision == KFBI_TF32X3 ? box_solve_tc(c, b, v) : box_solve3_f32(c, b, v);
}

// Double layer: jumps of the fitted density plus half the fit's residual at the points
// (reading S10); single layer ([v] = 0, [d_n v] = psi): jumps of the fitted psi, no
// identity part (dens below is then the density used only by that part: null).
kfbi_status apply_potential3(Ctx& c, Layer layer, int precision, const double* density,
                             double* out) {
  const bool single = layer == Layer::Single;
  const double* dens = single ? nullptr : density;
  KFBI_TRY(jumps3(c, dens, nullptr, !single, single ? density : nullptr));
  const int steps = steps_of(precision);
  if (use_fp32(precision)) {
    KFBI_TRY(correct3<float>(c, c.B32, 0, steps ? c.B64 : nullptr));
    if (steps == 0) {
      KFBI_TRY(plain_solve3(c, precision, c.B32, c.V32));
      return interp3<float>(c, c.V32, dens, out);
    }
    KFBI_TRY(refined_solve3(c, c.B32, nullptr, nullptr, steps));
    return interp3<float>(c, c.V32, dens, out, c.U32, steps > 1 ? c.T32 : nullptr);
  }
  KFBI_TRY(correct3<double>(c, c.B64, 0));
  KFBI_TRY(box_solve3_f64(c, c.B64, c.V64));
  return interp3<double>(c, c.V64, dens, out);
}

// Interface problem with Phi = fitted density, F = zero-extended f and [F] = f on Gamma:
// corrected right-hand side, grid solution and v^+ at the points (each output optional).
kfbi_status interface_solve3(Ctx& c, int precision, const double* dens, const double* f_grid,
                             const double* f_ctrl, double* rhs_grid, double* v_grid, double* out) {
  const int N = c.N;
  const long nw = (long)N * N * N, ng = (long)(N + 1) * (N + 1) * (N + 1);
  KFBI_TRY(jumps3(c, dens, f_ctrl, dens != nullptr));
  // dense right-hand side in FP64 (the sparse buffers keep zeros away from irregular nodes)
  double* B = c.V64;
  prof_count(c, ST_GRID);
  if (f_grid) rhs_dense3_kernel<double><<<grid_blocks(nw), 256, 0, c.stream>>>(N, f_grid, c.inside, B);
  else KFBI_CUDA_TRY(cudaMemsetAsync(B, 0, sizeof(double) * nw, c.stream));
  KFBI_CUDA_TRY(cudaGetLastError());
  KFBI_TRY(correct3<double>(c, B, 1));
  if (rhs_grid) {
    prof_count(c, ST_GRID);
    work_to_grid3_kernel<double><<<grid_blocks(ng), 256, 0, c.stream>>>(N, B, nullptr, rhs_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  const int steps = steps_of(precision);
  if (use_fp32(precision) && steps == 0) {
    prof_count(c, ST_GRID);
    convert_kernel3<<<grid_blocks(nw), 256, 0, c.stream>>>(nw, B, c.V32);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(plain_solve3(c, precision, c.V32, c.V32));
    if (v_grid) {
      prof_count(c, ST_GRID);
      work_to_grid3_kernel<float><<<grid_blocks(ng), 256, 0, c.stream>>>(N, c.V32, nullptr, v_grid);
      KFBI_CUDA_TRY(cudaGetLastError());
    }
    return out ? interp3<float>(c, c.V32, nullptr, out) : KFBI_OK;
  }
  if (use_fp32(precision)) {
    // exact FP32 pair of the dense FP64 right-hand side, refined FP32 solves, v summed
    // back into the FP64 work grid
    prof_count(c, ST_GRID);
    split3_kernel<<<grid_blocks(nw), 256, 0, c.stream>>>(nw, B, c.H32, c.D32);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(refined_solve3(c, c.H32, c.H32, c.D32, steps));
    prof_count(c, ST_GRID);
    sum3_kernel<<<grid_blocks(nw), 256, 0, c.stream>>>(nw, c.V32, c.U32, steps > 1 ? c.T32 : nullptr, B);
    KFBI_CUDA_TRY(cudaGetLastError());
  } else {
    KFBI_TRY(box_solve3_f64(c, B, B));
  }
  if (v_grid) {
    prof_count(c, ST_GRID);
    work_to_grid3_kernel<double><<<grid_blocks(ng), 256, 0, c.stream>>>(N, B, nullptr, v_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
  }
  return out ? interp3<double>(c, B, nullptr, out) : KFBI_OK;
}

kfbi_status combined_u3(Ctx& c, int precision, const double* dens, const double* f_grid,
                        const double* f_ctrl, double* u_grid) {
  const int N = c.N;
  const long ng = (long)(N + 1) * (N + 1) * (N + 1);
  KFBI_TRY(interface_solve3(c, precision, dens, f_grid, f_ctrl, nullptr, nullptr, nullptr));
  prof_count(c, ST_GRID);
  if (use_fp32(precision) && steps_of(precision) == 0)
    work_to_grid3_kernel<float><<<grid_blocks(ng), 256, 0, c.stream>>>(N, c.V32, c.inside, u_grid);
  else
    work_to_grid3_kernel<double><<<grid_blocks(ng), 256, 0, c.stream>>>(N, c.V64, c.inside, u_grid);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status box_solve_grid3(Ctx& c, int precision, const double* b_grid, double* v_grid) {
  const int N = c.N;
  const long nw = (long)N * N * N, ng = (long)(N + 1) * (N + 1) * (N + 1);
  const int steps = steps_of(precision);
  if (steps > 0) {                    // refined: exact FP32 pair of b, refined FP32 solves
    prof_count(c, ST_GRID, 4);
    grid_to_work3_kernel<double><<<grid_blocks(nw), 256, 0, c.stream>>>(N, b_grid, c.V64);
    split3_kernel<<<grid_blocks(nw), 256, 0, c.stream>>>(nw, c.V64, c.H32, c.D32);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(refined_solve3(c, c.H32, c.H32, c.D32, steps));
    sum3_kernel<<<grid_blocks(nw), 256, 0, c.stream>>>(nw, c.V32, c.U32, steps > 1 ? c.T32 : nullptr, c.V64);
    work_to_grid3_kernel<double><<<grid_blocks(ng), 256, 0, c.stream>>>(N, c.V64, nullptr, v_grid);
    KFBI_CUDA_TRY(cudaGetLastError());
    return KFBI_OK;
  }
  prof_count(c, ST_GRID, 2);
  if (precision != KFBI_FP64) {
    grid_to_work3_kernel<float><<<grid_blocks(nw), 256, 0, c.stream>>>(N, b_grid, c.V32);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(plain_solve3(c, precision, c.V32, c.V32));
    work_to_grid3_kernel<float><<<grid_blocks(ng), 256, 0, c.stream>>>(N, c.V32, nullptr, v_grid);
  } else {
    grid_to_work3_kernel<double><<<grid_blocks(nw), 256, 0, c.stream>>>(N, b_grid, c.V64);
    KFBI_CUDA_TRY(cudaGetLastError());
    KFBI_TRY(box_solve3_f64(c, c.V64, c.V64));
    work_to_grid3_kernel<double><<<grid_blocks(ng), 256, 0, c.stream>>>(N, c.V64, nullptr, v_grid);
  }
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status inside_mask3(Ctx& c, uint8_t* mask) {
  const long ng = (long)(c.N + 1) * (c.N + 1) * (c.N + 1);
  prof_count(c, ST_GRID);
  copy_bytes_kernel<<<grid_blocks(ng), 256, 0, c.stream>>>(ng, c.inside, mask);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace kfbi
