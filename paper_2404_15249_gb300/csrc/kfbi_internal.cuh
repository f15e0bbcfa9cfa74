// Internal definitions of the GB300 KFBI library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/kfbi.h"

namespace kfbi {

void set_error(const char* fmt, ...);
const char* last_error_message();          // this thread's last set_error text

#define KFBI_CUDA_TRY(expr)                                                          \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      ::kfbi::set_error("%s:%d: %s -> %s", __FILE__, __LINE__, #expr,                \
                        cudaGetErrorString(e_));                                     \
      return KFBI_ERR_CUDA;                                                          \
    }                                                                                \
  } while (0)

#define KFBI_TRY(expr)                 \
  do {                                 \
    kfbi_status s_ = (expr);           \
    if (s_ != KFBI_OK) return s_;      \
  } while (0)

// A kernel's dynamic shared-memory limit is an attribute of the kernel in one device's
// context.  It is recorded per (device, kernel address): a kernel template instantiated in
// several translation units (each compiled as its own module) is a distinct kernel in each,
// with its own attribute, so the record must not be keyed on the launching host template
// alone.  Two threads racing both set the same value, which is harmless.
kfbi_status set_smem_limit(const void* func, size_t bytes);
// ------------------------------------------------------------------ FFT plan
// Complex FFT of length N = 2^a or 3*2^a in shared memory.  Every thread of a line
// holds EPT values per stage; each stage radix divides EPT (16 for 2^a, 24 for 3*2^a).
struct FftPlan {
  int N;
  int ept;       // values per thread per stage
  int tpl;       // threads per line = N / ept
  int nst;       // number of stages
  int radix[12];
};

bool make_fft_plan(int N, FftPlan* p);

// Padded shared-memory index: one spare slot every 16 complex values keeps the
// stride-R writes of a Stockham stage free of bank conflicts.
__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int padded_len(int N) { return N + (N >> 4) + 1; }

// Device tables of one precision for the box solve on an N x N work grid.
template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

template <typename T>
struct BoxTables {
  typename Vec2<T>::type* tw;  // e^{-i pi t/N}, t < 2N
  T* lam;        // lambda_k = -(4/h^2) sin^2(pi k / 2N), k < N (lam[0] unused)
};

// ------------------------------------------------------------------ stage timers
enum Stage : int {
  ST_SETUP = 0, ST_CORR = 1, ST_ROWS32 = 2, ST_COLS32 = 3, ST_ROWS64 = 4, ST_COLS64 = 5,
  ST_INTERP = 6, ST_GRID = 7, ST_KRYLOV = 8, ST_REFINE = 9, ST_TRANS = 10, ST_SPARSE = 11,
  ST_TC = 12, ST_TRI = 13, ST_COUNT = 14   // ST_SPARSE: sparse first x-transform; ST_TC:
                                           // tensor-core GEMMs; ST_TRI: tridiagonal y-solves
};

struct Prof {
  bool on = false;
  bool hold = false;               // inside a span timed as a whole: count launches only
  std::vector<cudaEvent_t> ev;     // 2 per timed launch
  std::vector<int> stage;          // stage of each event pair
  int used = 0;
  double ms[KFBI_NSTAGES] = {};
  long long launches[KFBI_NSTAGES] = {};
};

// ------------------------------------------------------------------ context
constexpr int kStepGraphs = 5;   // precisions KFBI_FP64 .. KFBI_TF32X3
constexpr int kOpDirichlet = 0;  // GMRES operator: v^+ of the double layer (K_D)
constexpr int kOpNeumann = 1;    // GMRES operator: d_n v^+ of the single layer (K_N)
constexpr int kOps = 2;

struct Ctx {
  // problem (dim 2: M control points on a curve; dim 3: M grid-line intersection points)
  int dim = 2;
  int N = 0, M = 0;
  double lo = -1, hi = 1, h = 0, kappa = 0, kappa2 = 0;
  kfbi_options opt{};
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;              // second stream of the row-layout y-pass
  cudaStream_t own = nullptr;               // the context's stream for BVP solves
  cudaEvent_t own_in = nullptr, own_out = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  FftPlan plan{};

  // interface (device, FP64)
  double* pts = nullptr;      // M x 2
  double* nrm = nullptr;      // M x 2
  double* curv = nullptr;     // M

  // crossings: axis 0 = on vertical lines x = x_i, axis 1 = on horizontal lines y = y_j
  int ncross[2] = {0, 0};
  int* cr_line[2] = {nullptr, nullptr};
  int* cr_seg[2] = {nullptr, nullptr};
  double* cr_tau[2] = {nullptr, nullptr};
  double* cr_along[2] = {nullptr, nullptr};   // coordinate along the line (snapped)
  int* line_ptr[2] = {nullptr, nullptr};      // CSR over lines (N+2 entries), sorted by along
  int* cr_flip[2] = {nullptr, nullptr};       // arm index (lower node) each crossing belongs to

  uint8_t* inside = nullptr;                  // (N+1)^2 labels

  // irregular nodes and their crossed arms (CSR)
  int nirr = 0, narms = 0;
  int* irr_node = nullptr;                    // work-grid index j*N + i
  int* irr_rowptr = nullptr;                  // 2-D: row j's nodes [rowptr[j-1], rowptr[j])
  // work items of the sparse first x-transform (2-D), longest first: 8 ints each,
  // (row j, first node, end node, part, parts of the row, first scratch slot of the row,
  // arrival counter of the row, 0); a row with many irregular nodes is split into parts
  // whose partial rows are added by the last part to finish
  int spx_nitems = 0;
  int* spx_items = nullptr;
  float* spx_part = nullptr;                  // scratch rows of the split rows' parts
  unsigned* spx_cnt = nullptr;                // arrival counters of the split rows (zero at rest)
  int* arm_ptr = nullptr;                     // nirr + 1
  int* arm_seg = nullptr;                     // narms: segment of the crossing
  double* arm_wD = nullptr;                   // narms x 6: density -> correction (double layer)
  double* arm_wS = nullptr;                   // narms x 6: density -> correction (single layer)
  double* arm_wF = nullptr;                   // narms x 6: f on Gamma -> correction (volume)

  // control points: 6-node stencils
  int* ctrl_node = nullptr;                   // M x 6 work-grid index, -1 on the box boundary
  double* ctrl_w = nullptr;                   // M x 6 quadratic interpolation weights
  double* ctrl_cD = nullptr;                  // M x 6 density weights of the jump Taylor terms
  double* ctrl_cS = nullptr;                  // M x 6 (single layer)
  double* ctrl_eF = nullptr;                  // M   f(z) weight of the jump Taylor terms
  // stencil nodes of the control points by grid row (2-D): the plain FP32 apply's last
  // x-transform is evaluated only at these sn_count nodes, in sn_nitems work items
  int sn_count = 0, sn_nitems = 0;
  int* ctrl_slot = nullptr;                   // M x 6: slot of each stencil entry (-1: boundary)
  int* sn_col = nullptr;                      // column i of each node (sorted by row, column)
  int* sn_items = nullptr;                    // 4 ints each: row j, first node, end node, 0
                                              // (at most a few nodes each, longest first)
  float* sn_val = nullptr;                    // the values at the nodes (FP32 work values)
  // the same four for the normal derivative n . grad of the fitted quadratic at z
  double* ctrl_wn = nullptr;
  double* ctrl_cDn = nullptr;
  double* ctrl_cSn = nullptr;
  double* ctrl_eFn = nullptr;

  // 3-D interface: line CSR per axis, least-squares stencils, interpolation stencils
  int npts_axis[3] = {0, 0, 0};
  int* l3_ptr[3] = {nullptr, nullptr, nullptr};   // (N+1)^2 + 1 offsets per axis
  int* l3_pts[3] = {nullptr, nullptr, nullptr};   // points sorted by (line, coordinate)
  int* pt_edge = nullptr;                     // M: edge of the point on its line
  double* frame = nullptr;                    // M x 6: tangents t1, t2
  int* ls_ptr = nullptr;                      // M + 1
  int* ls_idx = nullptr;                      // neighbour points
  double* ls_w = nullptr;                     // 6 weights per neighbour (c0..c5)
  int* ip_node = nullptr;                     // M x 10 work-grid nodes
  double* ip_w = nullptr;                     // M x 10 interpolation weights
  double* ip_mom = nullptr;                   // M x 10 outside-node Taylor moments
  double* irr_sigma = nullptr;                // nirr: -1 inside, +1 outside
  int* arm3_pt = nullptr;                     // narms: point on the arm
  int* arm3_axis = nullptr;
  double* arm3_delta = nullptr;               // neighbour coordinate - point coordinate
  double* jmp3 = nullptr;                     // M x 10 jumps (J, G, H) scratch
  double* fit3 = nullptr;                     // M fitted density scratch

  // work grids (N^dim, index 0 along every axis identically zero)
  float* B32 = nullptr;  float* V32 = nullptr;     // sparse RHS (irregular entries only), work
  double* B64 = nullptr; double* V64 = nullptr;
  float* W32 = nullptr;                             // refinement residual (FP32)
  float* U32 = nullptr;                             // second FP32 solve of a refined solve
  float* T32 = nullptr;                             // third FP32 solve (two refinement steps)
  float* H32 = nullptr;                             // dense right-hand side, FP32 high part
  float* D32 = nullptr;                             // dense right-hand side, FP32 low part
  void* XT = nullptr;                               // transposed work grid (N x N, FP64 size)
  float* tc_shi = nullptr;                          // sine matrix, TF32 high part (N x N)
  float* tc_slo = nullptr;                          // sine matrix, TF32 low part
  void* tc_maps = nullptr;                          // TMA tensor maps of the GEMM operands
  int tri_k0 = 0;        // 2-D FP32: x-modes >= tri_k0 solved along y by elimination (N: none)
  int ypass_k0 = 0;      // 2-D FP32 row-layout y-pass: x-modes >= ypass_k0 by the filters (N: none)
  BoxTables<float> t32{};
  BoxTables<double> t64{};
  int rows_variant[2] = {0, 0};                     // row-pass variant per precision (autotuned)
  void* stw[4] = {nullptr, nullptr, nullptr, nullptr}; // stage twiddle tables (FP32/FP64 x EPT)
  int cols_variant[2] = {0, 0};                     // column-pass variant per precision (autotuned)

  // GMRES workspace (FP64)
  int gm_m = 0;
  double* basis = nullptr;     // (m+1) x M
  double* hess = nullptr;      // (m+1) x m, column major: hess[j*(m+1) + i]
  double* givens = nullptr;    // 2m (c, s)
  double* gvec = nullptr;      // m+1
  double* hcol = nullptr;      // m+1 scratch dot products
  double* scal = nullptr;      // 16 scalars
  double* vecs = nullptr;      // 6 x M scratch vectors
  double* yvec = nullptr;      // m
  double* h_pinned = nullptr;  // pinned host mirror of scal (16 doubles)
  cudaEvent_t gm_ev[2] = {nullptr, nullptr};   // Arnoldi steps done (their flags written)
  int* gm_j = nullptr;         // Arnoldi step index within the cycle (device)
  double* d_flags = nullptr;   // device address of h_pinned + 8 (host-mapped flag slots)
  // one captured CUDA graph per matvec precision for the whole Arnoldi step
  // (per BIE operator: kOpDirichlet, kOpNeumann)
  cudaGraphExec_t step_exec[kOps][kStepGraphs] = {};
  long long step_launches[kOps][kStepGraphs][KFBI_NSTAGES] = {};
  int gm_op = 0;               // operator of the solve in progress
  bool graphs_ok = true;       // false: direct launches (KFBI_GRAPHS=0, or capture failed)
  int graph_m = 0;             // restart length the graphs were captured with
  double* gm_part = nullptr;       // per-block partial dot products
  unsigned* gm_counter = nullptr;  // blocks done in the current multi-dot
  int* err_flag = nullptr;     // device error flags: [0] geometry, [2] bounded wait expired
  int poll_limit = 1 << 20;    // polls of a staged-copy wait before it gives up (a test
                               // lowers it through KFBI_TEST_POLL_LIMIT at setup)

  int64_t bytes = 0;
  int n_inside = 0;
  std::vector<void*> allocs;                  // device allocations owned by the context
  Prof prof;
};

// Launch bookkeeping: every kernel launch site calls prof_begin before and prof_end
// after the launch; the pair is timed with events only while profiling is on.
inline void prof_count(Ctx& c, int stage, int n = 1) { c.prof.launches[stage] += n; }
int prof_begin(Ctx& c, int stage);
void prof_end(Ctx& c, int pair);
// a span of several launches (possibly on two streams joined at its end) timed as one
// interval of `stage` on the context's stream; the launches inside are counted, not timed
int prof_span_begin(Ctx& c, int stage);
void prof_span_end(Ctx& c, int pair);
void prof_flush(Ctx& c);

// ------------------------------------------------------------------ stages
kfbi_status setup_geometry(Ctx& c);                 // setup2d.cu
kfbi_status alloc_bytes(Ctx& c, void** p, size_t bytes);

// box solve (dst.cu): three passes in place on the N x N work grid `work`, reading the
// right-hand side from `rhs` (may equal work).
kfbi_status box_solve_f32(Ctx& c, const float* rhs, float* work);
// the first pass of the FP32 box solve alone: the x-transform of every row of in into out
kfbi_status rows_pass_f32(Ctx& c, const float* in, float* out);
kfbi_status box_solve_f64(Ctx& c, const double* rhs, double* work);
// the y-transform pair with the spectral division on the transposed FP32 grid X in place,
// and the last half of the box solve: transpose X back into V and transform its rows
kfbi_status ylines_f32(Ctx& c, float* X);
kfbi_status x_pass_f32(Ctx& c, const float* X, float* V);
// FP32 2-D: the box solve after its first row pass (column pass variant + last row pass)
kfbi_status box_solve_after_rows_f32(Ctx& c, float* work);
// FP32 2-D y-pass on the row layout from V into Y (Y != V): recursive filters for the
// modes k >= ypass_k0, the transform pair (side stream) for the others (dst_ycol.cu); its
// result grid is ypass_out(c), the second half of the transposed scratch XT
kfbi_status ypass_rows_f32(Ctx& c, const float* V, float* Y);
// the transform pair along y (with the spectral division) of columns [0, ncols) of the
// row-layout FP32 grid V, written to the same columns of Y
kfbi_status ycol_lines_f32(Ctx& c, const float* V, float* Y, int ncols);
inline float* ypass_out(Ctx& c) { return reinterpret_cast<float*>(c.XT) + (size_t)c.N * c.N; }
kfbi_status init_box_tables(Ctx& c);
kfbi_status autotune_f32(Ctx& c);   // column-pass variant per precision, on scratch grids
kfbi_status autotune_f64(Ctx& c);

// apply stages (apply2d.cu)
enum class Layer { Double, Single };
// dn: the normal derivative d_n v^+ at the control points instead of v^+ (2-D)
kfbi_status apply_potential(Ctx& c, Layer layer, int precision, const double* dens, double* out,
                            bool dn = false);
// psi: single-layer density ([d_n v] = psi, 2-D), may be null
kfbi_status interface_solve(Ctx& c, int precision, const double* dens, const double* f_grid,
                            const double* f_ctrl, double* rhs_grid, double* v_grid,
                            double* out, const double* psi = nullptr, bool dn = false);
kfbi_status box_solve_grid(Ctx& c, int precision, const double* b_grid, double* v_grid);
kfbi_status inside_mask(Ctx& c, uint8_t* mask);
kfbi_status combined_u(Ctx& c, int precision, const double* dens, const double* f_grid,
                       const double* f_ctrl, double* u_grid, const double* psi = nullptr);
inline bool valid_precision(int p) {
  return p == KFBI_FP64 || p == KFBI_MIXED_FP32 || p == KFBI_FP32_REFINED ||
         p == KFBI_FP32_REFINED_ONCE || p == KFBI_TF32X3;
}

// dense tensor-core box solve (dst_tc.cu)
bool tc_supported(const Ctx& c);
kfbi_status init_tc_tables(Ctx& c);
kfbi_status box_solve_tc(Ctx& c, const float* rhs, float* work);
void free_tc(Ctx& c);

// tridiagonal y-solves of the well-conditioned x-modes (dst_tri.cu)
int tri_first_mode(const Ctx& c);
// first x-mode of the row-layout y-pass filters (dst_tri.cu)
int ypass_first_mode(const Ctx& c);
kfbi_status ytri_f32(Ctx& c, float* X, int k0);

// 3-D (kfbi3d.cu, dst3d.cu): setup and the same stages on the N^3 work grid
kfbi_status setup_geometry3(Ctx& c);
kfbi_status box_solve3_f32(Ctx& c, const float* rhs, float* work);
kfbi_status box_solve3_f64(Ctx& c, const double* rhs, double* work);
kfbi_status apply_potential3(Ctx& c, Layer layer, int precision, const double* dens, double* out);
kfbi_status interface_solve3(Ctx& c, int precision, const double* dens, const double* f_grid,
                             const double* f_ctrl, double* rhs_grid, double* v_grid, double* out);
kfbi_status combined_u3(Ctx& c, int precision, const double* dens, const double* f_grid,
                        const double* f_ctrl, double* u_grid);
kfbi_status box_solve_grid3(Ctx& c, int precision, const double* b_grid, double* v_grid);
kfbi_status inside_mask3(Ctx& c, uint8_t* mask);

// solver (gmres.cu)
kfbi_status solve_bvp(Ctx& c, const double* f_grid, const double* f_ctrl, const double* g_ctrl,
                      double* u_grid, double* dens_out, kfbi_solve_info* info, int op);
kfbi_status alloc_gmres(Ctx& c, int m);
void drop_step_graphs(Ctx& c);   // the captured Arnoldi-step graphs (recaptured on use)
kfbi_status batch_solve(kfbi_ctx* ctxs, int count, int nrhs, const double* const* f_grid,
                        const double* const* f_ctrl, const double* const* g_ctrl,
                        double* const* u_grid, double* const* dens_out, kfbi_solve_info* info,
                        cudaStream_t stream);

}  // namespace kfbi

struct kfbi_ctx_s {
  kfbi::Ctx c;
};
