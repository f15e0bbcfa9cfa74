// extern "C" entry points of libkfbi (declared and documented in include/kfbi.h).
#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "kfbi_internal.cuh"

namespace kfbi {

static thread_local char g_err[512] = "";

const char* last_error_message() { return g_err; }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

kfbi_status set_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;   // (device, kernel) -> bytes set
  int dev = 0;
  KFBI_CUDA_TRY(cudaGetDevice(&dev));
  const std::pair<int, const void*> key(dev, func);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return KFBI_OK;
  }
  KFBI_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  std::lock_guard<std::mutex> lock(mu);
  size_t& b = done[key];
  if (b < bytes) b = bytes;
  return KFBI_OK;
}

kfbi_status alloc_bytes(Ctx& c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    return KFBI_ERR_NOMEM;
  }
  c.allocs.push_back(*p);                    // recorded first: freed with the context on any error
  c.bytes += (int64_t)bytes;
  e = cudaMemsetAsync(*p, 0, bytes, c.stream);
  if (e != cudaSuccess) {
    set_error("cudaMemsetAsync failed: %s", cudaGetErrorString(e));
    return KFBI_ERR_CUDA;
  }
  return KFBI_OK;
}

}  // namespace kfbi

using kfbi::Ctx;

static void free_handle(kfbi_ctx_s* hd) {
  if (!hd) return;
  Ctx& c = hd->c;
  if (c.stream) cudaStreamSynchronize(c.stream);
  for (void* p : c.allocs) cudaFree(p);
  if (c.basis) {
    cudaFree(c.basis); cudaFree(c.hess); cudaFree(c.givens); cudaFree(c.gvec);
    cudaFree(c.hcol); cudaFree(c.yvec); cudaFree(c.gm_part); cudaFree(c.gm_counter);
  }
  kfbi::drop_step_graphs(c);
  if (c.gm_j) cudaFree(c.gm_j);
  if (c.h_pinned) cudaFreeHost(c.h_pinned);
  kfbi::free_tc(c);
  for (int i = 0; i < 2; ++i)
    if (c.gm_ev[i]) cudaEventDestroy(c.gm_ev[i]);
  if (c.own) cudaStreamSynchronize(c.own);
  if (c.fork_ev) cudaEventDestroy(c.fork_ev);
  if (c.own_in) cudaEventDestroy(c.own_in);
  if (c.own_out) cudaEventDestroy(c.own_out);
  if (c.own) cudaStreamDestroy(c.own);
  if (c.join_ev) cudaEventDestroy(c.join_ev);
  if (c.side) cudaStreamDestroy(c.side);
  delete hd;
}

extern "C" {

void kfbi_default_options(kfbi_options* o) {
  if (!o) return;
  o->dim = 2;
  o->N = 128;
  o->lo = -1.0;
  o->hi = 1.0;
  o->kappa = 0.0;
  o->precision = KFBI_FP64;
  o->gmres_m = 50;
  o->max_restarts = 20;
  o->tol = 1e-10;
  o->inner_tol = 1e-5;
}

const char* kfbi_status_string(kfbi_status s) {
  switch (s) {
    case KFBI_OK: return "ok";
    case KFBI_ERR_ARG: return "invalid argument";
    case KFBI_ERR_GEOMETRY: return "interface geometry rejected";
    case KFBI_ERR_NOMEM: return "out of device memory";
    case KFBI_ERR_CUDA: return "CUDA error";
    case KFBI_ERR_NOT_CONVERGED: return "GMRES did not converge";
    case KFBI_ERR_TIMEOUT: return "device wait timed out";
    case KFBI_ERR_NUMERIC: return "non-finite value in the iteration";
    case KFBI_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

const char* kfbi_last_error(void) { return kfbi::g_err; }

kfbi_status kfbi_setup(const kfbi_options* opt, int64_t M, const double* d_pts,
                       const double* d_normals, const double* d_curv, void* stream,
                       kfbi_ctx* out) {
  if (out) *out = nullptr;
  if (!opt || !out || !d_pts || !d_normals || !d_curv) {
    kfbi::set_error("kfbi_setup: null argument");
    return KFBI_ERR_ARG;
  }
  if (opt->dim != 2 && opt->dim != 3) {
    kfbi::set_error("kfbi_setup: dim = %d (2 or 3)", opt->dim);
    return KFBI_ERR_UNSUPPORTED;
  }
  const int dim = opt->dim;
  const int nmax = dim == 2 ? 8192 : 512;
  kfbi::FftPlan plan;
  if (!kfbi::make_fft_plan(opt->N, &plan) || opt->N > nmax) {
    kfbi::set_error("kfbi_setup: N = %d must be 2^a or 3*2^a with 32 <= N <= %d", opt->N, nmax);
    return KFBI_ERR_ARG;
  }
  if (M < 8 || M > (1 << 22) || !(opt->hi > opt->lo) || !(opt->kappa >= 0.0) ||
      opt->gmres_m < 1 || opt->gmres_m > 128 || opt->max_restarts < 0 || !(opt->tol > 0.0) ||
      !kfbi::valid_precision(opt->precision)) {
    kfbi::set_error("kfbi_setup: bad size or option");
    return KFBI_ERR_ARG;
  }
  kfbi_ctx_s* hd = new (std::nothrow) kfbi_ctx_s();
  if (!hd) {
    kfbi::set_error("kfbi_setup: host allocation of the context failed");
    return KFBI_ERR_NOMEM;
  }
  Ctx& c = hd->c;
  c.opt = *opt;
  c.N = opt->N;
  c.M = (int)M;
  c.lo = opt->lo;
  c.hi = opt->hi;
  c.h = (opt->hi - opt->lo) / opt->N;
  c.kappa = opt->kappa;
  c.kappa2 = opt->kappa * opt->kappa;
  c.stream = (cudaStream_t)stream;
  c.plan = plan;
  c.dim = dim;
  // KFBI_GRAPHS=0: the Arnoldi steps are launched kernel by kernel instead of as graphs
  if (const char* e = std::getenv("KFBI_GRAPHS"))
    if (e[0] == '0') c.graphs_ok = false;
  // KFBI_TEST_POLL_LIMIT (tests of the failure path only): polls of a staged-copy wait
  // before it records a timeout; 0 makes every such wait give up at once
  if (const char* e = std::getenv("KFBI_TEST_POLL_LIMIT")) {
    const long v = std::strtol(e, nullptr, 10);
    if (v >= 0 && v < (1 << 20)) c.poll_limit = (int)v;
  }
  if (opt->precision == KFBI_TF32X3 && !kfbi::tc_supported(c)) {
    kfbi::set_error("kfbi_setup: KFBI_TF32X3 needs N a multiple of 128, up to 8192 in 2-D and 512 in 3-D");
    free_handle(hd);
    return KFBI_ERR_UNSUPPORTED;
  }
  kfbi_status s = KFBI_OK;
  const size_t grid = (size_t)c.N * c.N * (dim == 3 ? (size_t)c.N : 1);
#define SETUP_TRY(expr)       \
  do {                        \
    s = (expr);               \
    if (s != KFBI_OK) {       \
      free_handle(hd);        \
      return s;               \
    }                         \
  } while (0)
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.err_flag, sizeof(int) * 4));
  if (cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c.own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.join_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.own_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c.own_out, cudaEventDisableTiming) != cudaSuccess) {
    kfbi::set_error("kfbi_setup: stream or event creation failed");
    free_handle(hd);
    return KFBI_ERR_CUDA;
  }
  // per point: dim coordinates, dim normal components, 1 curvature (2-D) or 6 packed
  // shape-operator entries (3-D)
  const size_t ncurv = dim == 2 ? 1 : 6;
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.pts, sizeof(double) * dim * M));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.nrm, sizeof(double) * dim * M));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.curv, sizeof(double) * ncurv * M));
  if (cudaMemcpyAsync(c.pts, d_pts, sizeof(double) * dim * M, cudaMemcpyDeviceToDevice, c.stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(c.nrm, d_normals, sizeof(double) * dim * M, cudaMemcpyDeviceToDevice,
                      c.stream) != cudaSuccess ||
      cudaMemcpyAsync(c.curv, d_curv, sizeof(double) * ncurv * M, cudaMemcpyDeviceToDevice,
                      c.stream) != cudaSuccess) {
    kfbi::set_error("kfbi_setup: copying the interface failed: %s",
                    cudaGetErrorString(cudaGetLastError()));
    free_handle(hd);
    return KFBI_ERR_CUDA;
  }
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.B32, sizeof(float) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.V32, sizeof(float) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.B64, sizeof(double) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.V64, sizeof(double) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.W32, sizeof(float) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.U32, sizeof(float) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.T32, sizeof(float) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.H32, sizeof(float) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.D32, sizeof(float) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, &c.XT, sizeof(double) * grid));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.scal, sizeof(double) * 16));
  SETUP_TRY(kfbi::alloc_bytes(c, (void**)&c.vecs, sizeof(double) * 8 * M));
  if (cudaMallocHost((void**)&c.h_pinned, sizeof(double) * 16) != cudaSuccess) {
    kfbi::set_error("kfbi_setup: pinned host allocation failed");
    free_handle(hd);
    return KFBI_ERR_NOMEM;
  }
  SETUP_TRY(kfbi::init_box_tables(c));
  if (dim == 2) {
    // KFBI_DST_VARIANTS="r32,c32,r64,c64" fixes the transform variants (profiling runs,
    // where the autotuner's timings would be distorted by the profiler)
    c.tri_k0 = kfbi::tri_first_mode(c);
    c.ypass_k0 = kfbi::ypass_first_mode(c);
    const char* fixed = std::getenv("KFBI_DST_VARIANTS");
    int v[4];
    if (fixed && std::sscanf(fixed, "%d,%d,%d,%d", &v[0], &v[1], &v[2], &v[3]) == 4 &&
        v[0] >= 0 && v[0] <= 1 && v[2] >= 0 && v[2] <= 1 && v[1] >= 0 && v[1] <= 8 &&
        v[3] >= 0 && v[3] <= 7 && (v[1] != 8 || (c.ypass_k0 > 0 && c.ypass_k0 < c.N))) {
      c.rows_variant[0] = v[0];
      c.cols_variant[0] = v[1];
      c.rows_variant[1] = v[2];
      c.cols_variant[1] = v[3];
    } else {
      SETUP_TRY(kfbi::autotune_f32(c));
      SETUP_TRY(kfbi::autotune_f64(c));
    }
    SETUP_TRY(kfbi::setup_geometry(c));
    SETUP_TRY(kfbi::init_tc_tables(c));
  } else {
    SETUP_TRY(kfbi::setup_geometry3(c));
    SETUP_TRY(kfbi::init_tc_tables(c));
  }
  SETUP_TRY(kfbi::alloc_gmres(c, c.opt.gmres_m));
  if (cudaStreamSynchronize(c.stream) != cudaSuccess) {
    kfbi::set_error("kfbi_setup: %s", cudaGetErrorString(cudaGetLastError()));
    free_handle(hd);
    return KFBI_ERR_CUDA;
  }
#undef SETUP_TRY
  *out = hd;
  return KFBI_OK;
}

static Ctx* ctx_of(kfbi_ctx h, cudaStream_t st) {
  if (!h) return nullptr;
  h->c.stream = st;
  return &h->c;
}

// the tensor-core precision exists for N a multiple of 128, up to 8192 in 2-D and 512 in 3-D
static bool tc_refused(const Ctx& c, int precision, const char* who) {
  if (precision != KFBI_TF32X3 || kfbi::tc_supported(c)) return false;
  kfbi::set_error("%s: KFBI_TF32X3 needs N a multiple of 128, up to 8192 in 2-D and 512 in 3-D", who);
  return true;
}

kfbi_status kfbi_apply_layer_potential(kfbi_ctx ctx, int layer, int precision,
                                       const double* d_density, double* d_out, void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !d_density || !d_out || (layer != KFBI_DOUBLE_LAYER && layer != KFBI_SINGLE_LAYER) ||
      !kfbi::valid_precision(precision)) {
    kfbi::set_error("kfbi_apply_layer_potential: bad argument");
    return KFBI_ERR_ARG;
  }
  if (tc_refused(*c, precision, "kfbi_apply_layer_potential")) return KFBI_ERR_UNSUPPORTED;
  return kfbi::apply_potential(*c, layer == KFBI_DOUBLE_LAYER ? kfbi::Layer::Double
                                                              : kfbi::Layer::Single,
                               precision, d_density, d_out);
}

kfbi_status kfbi_apply_volume(kfbi_ctx ctx, int precision, const double* d_f_grid,
                              const double* d_f_ctrl, double* d_out, void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !d_f_grid || !d_f_ctrl || !d_out ||
      !kfbi::valid_precision(precision)) {
    kfbi::set_error("kfbi_apply_volume: bad argument");
    return KFBI_ERR_ARG;
  }
  if (tc_refused(*c, precision, "kfbi_apply_volume")) return KFBI_ERR_UNSUPPORTED;
  return kfbi::interface_solve(*c, precision, nullptr, d_f_grid, d_f_ctrl, nullptr, nullptr,
                               d_out);
}

kfbi_status kfbi_interface_solve(kfbi_ctx ctx, int precision, const double* d_density,
                                 const double* d_f_grid, const double* d_f_ctrl,
                                 double* d_rhs_grid, double* d_v_grid, double* d_out,
                                 void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !kfbi::valid_precision(precision)) {
    kfbi::set_error("kfbi_interface_solve: bad argument");
    return KFBI_ERR_ARG;
  }
  if (tc_refused(*c, precision, "kfbi_interface_solve")) return KFBI_ERR_UNSUPPORTED;
  return kfbi::interface_solve(*c, precision, d_density, d_f_grid, d_f_ctrl, d_rhs_grid, d_v_grid,
                               d_out);
}

kfbi_status kfbi_box_solve(kfbi_ctx ctx, int precision, const double* d_b_grid, double* d_v_grid,
                           void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !d_b_grid || !d_v_grid || !kfbi::valid_precision(precision)) {
    kfbi::set_error("kfbi_box_solve: bad argument");
    return KFBI_ERR_ARG;
  }
  if (tc_refused(*c, precision, "kfbi_box_solve")) return KFBI_ERR_UNSUPPORTED;
  return kfbi::box_solve_grid(*c, precision, d_b_grid, d_v_grid);
}

kfbi_status kfbi_solve_bvp(kfbi_ctx ctx, const double* d_f_grid, const double* d_f_ctrl,
                           const double* d_g_ctrl, double* d_u_grid, double* d_density_out,
                           kfbi_solve_info* h_info, void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !d_f_grid || !d_f_ctrl || !d_g_ctrl) {
    kfbi::set_error("kfbi_solve_bvp: bad argument");
    return KFBI_ERR_ARG;
  }
  return kfbi::solve_bvp(*c, d_f_grid, d_f_ctrl, d_g_ctrl, d_u_grid, d_density_out, h_info,
                         kfbi::kOpDirichlet);
}

kfbi_status kfbi_solve_neumann_bvp(kfbi_ctx ctx, const double* d_f_grid, const double* d_f_ctrl,
                                   const double* d_gn_ctrl, double* d_u_grid,
                                   double* d_density_out, kfbi_solve_info* h_info, void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !d_f_grid || !d_f_ctrl || !d_gn_ctrl) {
    kfbi::set_error("kfbi_solve_neumann_bvp: bad argument");
    return KFBI_ERR_ARG;
  }
  if (c->dim != 2) {
    kfbi::set_error("kfbi_solve_neumann_bvp: 2-D only");
    return KFBI_ERR_UNSUPPORTED;
  }
  if (!(c->kappa > 0.0)) {              // kappa = 0: u fixed only up to a constant, K_N singular
    kfbi::set_error("kfbi_solve_neumann_bvp: kappa must be positive");
    return KFBI_ERR_ARG;
  }
  return kfbi::solve_bvp(*c, d_f_grid, d_f_ctrl, d_gn_ctrl, d_u_grid, d_density_out, h_info,
                         kfbi::kOpNeumann);
}

kfbi_status kfbi_apply_layer_potential_dn(kfbi_ctx ctx, int layer, int precision,
                                          const double* d_density, double* d_out, void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !d_density || !d_out || (layer != KFBI_DOUBLE_LAYER && layer != KFBI_SINGLE_LAYER) ||
      !kfbi::valid_precision(precision)) {
    kfbi::set_error("kfbi_apply_layer_potential_dn: bad argument");
    return KFBI_ERR_ARG;
  }
  if (c->dim != 2) {
    kfbi::set_error("kfbi_apply_layer_potential_dn: 2-D only");
    return KFBI_ERR_UNSUPPORTED;
  }
  if (tc_refused(*c, precision, "kfbi_apply_layer_potential_dn")) return KFBI_ERR_UNSUPPORTED;
  return kfbi::apply_potential(*c, layer == KFBI_DOUBLE_LAYER ? kfbi::Layer::Double
                                                              : kfbi::Layer::Single,
                               precision, d_density, d_out, true);
}

kfbi_status kfbi_apply_volume_dn(kfbi_ctx ctx, int precision, const double* d_f_grid,
                                 const double* d_f_ctrl, double* d_out, void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !d_f_grid || !d_f_ctrl || !d_out || !kfbi::valid_precision(precision)) {
    kfbi::set_error("kfbi_apply_volume_dn: bad argument");
    return KFBI_ERR_ARG;
  }
  if (c->dim != 2) {
    kfbi::set_error("kfbi_apply_volume_dn: 2-D only");
    return KFBI_ERR_UNSUPPORTED;
  }
  if (tc_refused(*c, precision, "kfbi_apply_volume_dn")) return KFBI_ERR_UNSUPPORTED;
  return kfbi::interface_solve(*c, precision, nullptr, d_f_grid, d_f_ctrl, nullptr, nullptr, d_out,
                               nullptr, true);
}

kfbi_status kfbi_get_inside_mask(kfbi_ctx ctx, uint8_t* d_mask, void* stream) {
  Ctx* c = ctx_of(ctx, (cudaStream_t)stream);
  if (!c || !d_mask) {
    kfbi::set_error("kfbi_get_inside_mask: null argument");
    return KFBI_ERR_ARG;
  }
  return kfbi::inside_mask(*c, d_mask);
}

kfbi_status kfbi_get_info(kfbi_ctx ctx, kfbi_ctx_info* info) {
  if (!ctx || !info) {
    kfbi::set_error("kfbi_get_info: null argument");
    return KFBI_ERR_ARG;
  }
  const Ctx& c = ctx->c;
  info->N = c.N;
  info->M = c.M;
  info->dim = c.dim;
  info->n_crossings_x = c.dim == 2 ? c.ncross[0] : c.npts_axis[0];
  info->n_crossings_y = c.dim == 2 ? c.ncross[1] : c.npts_axis[1];
  info->n_crossings_z = c.dim == 2 ? 0 : c.npts_axis[2];
  // the split of the y-pass variant in use: the row-layout filters (variant bit 8) start
  // at c <= 0.9, the transposed elimination at c <= 0.825
  info->tri_first_mode = c.dim != 2 ? c.N : (c.cols_variant[0] & 8) ? c.ypass_k0 : c.tri_k0;
  info->n_irregular = c.nirr;
  info->n_inside = c.n_inside;
  info->device_bytes = c.bytes + (int64_t)sizeof(double) * ((int64_t)(c.gm_m + 1) * c.M);
  info->dst_variant[0] = c.rows_variant[0];
  info->dst_variant[1] = c.cols_variant[0];
  info->dst_variant[2] = c.rows_variant[1];
  info->dst_variant[3] = c.cols_variant[1];
  return KFBI_OK;
}

kfbi_status kfbi_set_solver(kfbi_ctx ctx, int precision, int gmres_m, int max_restarts,
                            double tol, double inner_tol) {
  if (!ctx || !kfbi::valid_precision(precision) || gmres_m < 1 ||
      gmres_m > 128 || max_restarts < 0 || !(tol > 0) || !(inner_tol > 0)) {
    kfbi::set_error("kfbi_set_solver: bad argument");
    return KFBI_ERR_ARG;
  }
  Ctx& c = ctx->c;
  if (tc_refused(c, precision, "kfbi_set_solver")) return KFBI_ERR_UNSUPPORTED;
  c.opt.precision = precision;
  c.opt.gmres_m = gmres_m;
  c.opt.max_restarts = max_restarts;
  c.opt.tol = tol;
  c.opt.inner_tol = inner_tol;
  return kfbi::alloc_gmres(c, gmres_m);
}

kfbi_status kfbi_destroy(kfbi_ctx ctx) {
  if (!ctx) {
    kfbi::set_error("kfbi_destroy: null context");
    return KFBI_ERR_ARG;
  }
  free_handle(ctx);
  return KFBI_OK;
}

// ---------------------------------------------------------------- batches
struct kfbi_batch_s {
  std::vector<kfbi_ctx> ctxs;
};

kfbi_status kfbi_batch_create(const kfbi_ctx* ctxs, int count, kfbi_batch* out) {
  if (out) *out = nullptr;
  if (!ctxs || !out || count < 1) {
    kfbi::set_error("kfbi_batch_create: bad argument");
    return KFBI_ERR_ARG;
  }
  kfbi_batch_s* b = new (std::nothrow) kfbi_batch_s();
  if (!b) {
    kfbi::set_error("kfbi_batch_create: host allocation failed");
    return KFBI_ERR_NOMEM;
  }
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) {
      delete b;
      kfbi::set_error("kfbi_batch_create: null context %d", i);
      return KFBI_ERR_ARG;
    }
    b->ctxs.push_back(ctxs[i]);
  }
  // a context listed twice would be driven by two workers at once (one workspace, one
  // stream): refused
  std::vector<kfbi_ctx> sorted(b->ctxs);
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
    delete b;
    kfbi::set_error("kfbi_batch_create: a context is listed more than once");
    return KFBI_ERR_ARG;
  }
  *out = b;
  return KFBI_OK;
}

kfbi_status kfbi_batch_solve(kfbi_batch b, int nrhs, const double* const* d_f_grid,
                             const double* const* d_f_ctrl, const double* const* d_g_ctrl,
                             double* const* d_u_grid, double* const* d_density_out,
                             kfbi_solve_info* h_info, void* stream) {
  if (!b || nrhs < 1 || !d_f_grid || !d_f_ctrl || !d_g_ctrl || !d_u_grid) {
    kfbi::set_error("kfbi_batch_solve: bad argument");
    return KFBI_ERR_ARG;
  }
  return kfbi::batch_solve(b->ctxs.data(), (int)b->ctxs.size(), nrhs, d_f_grid, d_f_ctrl,
                           d_g_ctrl, d_u_grid, d_density_out, h_info, (cudaStream_t)stream);
}

kfbi_status kfbi_batch_destroy(kfbi_batch b) {
  if (!b) {
    kfbi::set_error("kfbi_batch_destroy: null batch");
    return KFBI_ERR_ARG;
  }
  delete b;
  return KFBI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- stage timers
namespace kfbi {

static const int kProfPairs = 4096;

void prof_flush(Ctx& c) {
  Prof& p = c.prof;
  if (p.used == 0) return;
  cudaStreamSynchronize(c.stream);
  for (int i = 0; i < p.used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]) == cudaSuccess)
      p.ms[p.stage[i]] += ms;
  }
  p.used = 0;
}

static int prof_record(Ctx& c, int stage) {
  Prof& p = c.prof;
  if (p.used == kProfPairs) prof_flush(c);
  const int i = p.used++;
  p.stage[i] = stage;
  cudaEventRecord(p.ev[2 * i], c.stream);
  return i;
}

int prof_span_begin(Ctx& c, int stage) {
  Prof& p = c.prof;
  if (!p.on || p.hold) return -1;
  const int i = prof_record(c, stage);
  p.hold = true;
  return i;
}

void prof_span_end(Ctx& c, int pair) {
  if (pair < 0) return;
  c.prof.hold = false;
  cudaEventRecord(c.prof.ev[2 * pair + 1], c.stream);
}

int prof_begin(Ctx& c, int stage) {
  Prof& p = c.prof;
  ++p.launches[stage];
  if (!p.on || p.hold) return -1;
  return prof_record(c, stage);
}

void prof_end(Ctx& c, int pair) {
  if (pair >= 0) cudaEventRecord(c.prof.ev[2 * pair + 1], c.stream);
}

}  // namespace kfbi

extern "C" {

kfbi_status kfbi_profile(kfbi_ctx ctx, int enable) {
  if (!ctx) {
    kfbi::set_error("kfbi_profile: null context");
    return KFBI_ERR_ARG;
  }
  kfbi::Ctx& c = ctx->c;
  kfbi::Prof& p = c.prof;
  if (enable) {
    if (p.ev.empty()) {
      p.ev.resize(2 * kfbi::kProfPairs);
      p.stage.resize(kfbi::kProfPairs);
      for (auto& e : p.ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
          kfbi::set_error("kfbi_profile: cudaEventCreate failed");
          return KFBI_ERR_CUDA;
        }
    }
    p.used = 0;
    for (int s = 0; s < KFBI_NSTAGES; ++s) { p.ms[s] = 0.0; p.launches[s] = 0; }
    p.on = true;
  } else {
    kfbi::prof_flush(c);
    p.on = false;
  }
  return KFBI_OK;
}

kfbi_status kfbi_profile_read(kfbi_ctx ctx, kfbi_stage_times* out) {
  if (!ctx || !out) {
    kfbi::set_error("kfbi_profile_read: null argument");
    return KFBI_ERR_ARG;
  }
  kfbi::Ctx& c = ctx->c;
  kfbi::prof_flush(c);
  for (int s = 0; s < KFBI_NSTAGES; ++s) {
    out->ms[s] = c.prof.ms[s];
    out->launches[s] = c.prof.launches[s];
  }
  out->nstages = kfbi::ST_COUNT;
  return KFBI_OK;
}

const char* kfbi_stage_name(int s) {
  static const char* names[] = {"setup", "correction", "dst_rows_f32", "dst_cols_f32",
                                "dst_rows_f64", "dst_cols_f64", "interpolation", "grid",
                                "krylov", "refine", "transpose", "sparse_x_f32", "dst_tc_tf32x3", "dst_tri_f32"};
  return (s >= 0 && s < kfbi::ST_COUNT) ? names[s] : "unused";
}

}  // extern "C"
