// Box solve of Alg. 4 without a context and without any device allocation: the work grid
// and the transform tables live in one library-static device array per device.  The
// transforms are the kernels of the context box solve (dst_impl.cuh) in their default
// variants; only the home of their workspace differs.
#include <mutex>

#include "dst_impl.cuh"

namespace kfbi {
namespace boxstatic {

using dst::cplan;
using dst::cx;
using dst::default_ept;

constexpr int kMaxN = KFBI_STATIC_MAX_N;
constexpr size_t kScratchBytes = KFBI_STATIC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch array.  Nothing in the work area has to start at zero: every call writes the
// tables and the whole work grid before any kernel reads them.  The last kCtlBytes hold the
// error word (an int set when a bounded wait of a transform kernel gave up); it starts at
// zero (device statics are zero-initialised at load) and only kfbi_box_solve_static_check
// clears it again.
static __device__ __align__(256) unsigned char g_box_scratch[kScratchBytes];
constexpr size_t kCtlBytes = 256;
constexpr size_t kWorkBytes = kScratchBytes - kCtlBytes;

std::mutex g_lock;
unsigned char* g_base[kMaxDevices];   // device address of g_box_scratch, per device

constexpr size_t round256(size_t n) { return (n + 255) / 256 * 256; }

// scratch layout for (T, N): work grid N x N, tw (2N), lam (N), stage twiddles
template <typename T, int N>
constexpr size_t bytes_needed() {
  constexpr dst::CPlan P = cplan(N, default_ept(N));
  return round256(sizeof(T) * (size_t)N * N) + round256(sizeof(cx<T>) * 2 * (size_t)N) +
         round256(sizeof(T) * (size_t)N) +
         round256(sizeof(cx<T>) * (size_t)(P.twtotal > 0 ? P.twtotal : 1));
}
static_assert(bytes_needed<double, kMaxN>() <= kWorkBytes, "scratch too small for max N");
static_assert(bytes_needed<double, 768>() <= kWorkBytes, "scratch too small for N = 768");

// twiddles tw[s] = e^{-i pi s/N} (s < 2N) and eigenvalues lam[k] = -(4/h^2) sin^2(pi k/2N)
// of the 1-D second difference, computed in FP64 and rounded to T
template <typename T>
__global__ void tables_kernel(int N, double h, cx<T>* __restrict__ tw, T* __restrict__ lam) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < 2 * N) {
    double sn, cs;
    sincospi((double)s / (double)N, &sn, &cs);
    tw[s] = cx<T>{(T)cs, (T)-sn};
  }
  if (s < N) {
    const double sk = sinpi((double)s / (2.0 * N));
    lam[s] = (T)(-(4.0 / (h * h)) * sk * sk);
  }
}

// (N+1)^2 FP64 grid -> N x N work grid (row 0 and column 0 zero, boundary of b ignored)
template <typename T>
__global__ void load_kernel(int N, const double* __restrict__ b, T* __restrict__ w) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
    w[(size_t)j * N + i] = (i > 0 && j > 0) ? (T)b[(size_t)j * (N + 1) + i] : T(0);
}

// work grid -> (N+1)^2 FP64 grid with v = 0 on the box boundary
template <typename T>
__global__ void store_kernel(int N, const T* __restrict__ w, double* __restrict__ v) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= N; i += gridDim.x * blockDim.x)
    v[(size_t)j * (N + 1) + i] = (i < N && j < N) ? (double)w[(size_t)j * N + i] : 0.0;
}

template <typename T, int N>
struct Launch {
  static constexpr int E = default_ept(N);
  static constexpr dst::CPlan P = cplan(N, E);
  static constexpr int LPC = P.tpl >= 256 ? 1 : 256 / P.tpl;        // rows per CTA
  static constexpr int L = dst::cols_L<T, N, E, 512>();              // columns per CTA
  static constexpr size_t rows_smem = dst::rows_smem<T, N, E>(LPC);
  static constexpr size_t cols_smem = dst::cols_smem<T, N, E, 512>();

  static kfbi_status attributes() {
    KFBI_CUDA_TRY(cudaFuncSetAttribute(dst::rows_kernel<T, N, E>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem));
    KFBI_CUDA_TRY(cudaFuncSetAttribute(dst::cols_kernel<T, N, E, 512>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cols_smem));
    return KFBI_OK;
  }

  static kfbi_status solve(unsigned char* base, double h, double kappa2, const double* b,
                           double* v, cudaStream_t s) {
    size_t off = 0;
    auto take = [&](size_t n) { unsigned char* p = base + off; off += round256(n); return p; };
    T* work = reinterpret_cast<T*>(take(sizeof(T) * (size_t)N * N));
    cx<T>* tw = reinterpret_cast<cx<T>*>(take(sizeof(cx<T>) * 2 * (size_t)N));
    T* lam = reinterpret_cast<T*>(take(sizeof(T) * (size_t)N));
    cx<T>* stw = reinterpret_cast<cx<T>*>(take(sizeof(cx<T>) * (size_t)(P.twtotal > 0 ? P.twtotal : 1)));

    tables_kernel<T><<<(2 * N + 255) / 256, 256, 0, s>>>(N, h, tw, lam);
    KFBI_CUDA_TRY(cudaGetLastError());
    if (P.twtotal > 0) {
      dst::stage_twiddles_kernel<T, N, E><<<(P.twtotal + 255) / 256, 256, 0, s>>>(tw, stw);
      KFBI_CUDA_TRY(cudaGetLastError());
    }
    const dim3 gg((N + 256) / 256 < 8 ? (N + 256) / 256 : 8, N + 1);
    load_kernel<T><<<dim3(gg.x, N), 256, 0, s>>>(N, b, work);
    KFBI_CUDA_TRY(cudaGetLastError());
    const int row_blocks = (N + LPC - 1) / LPC;
    int* err = reinterpret_cast<int*>(base + kWorkBytes);
    dst::rows_kernel<T, N, E><<<row_blocks, LPC * P.tpl, rows_smem, s>>>(work, work, stw, tw, T(1), N, err,
                                                                      dst::kPollLimit);
    KFBI_CUDA_TRY(cudaGetLastError());
    dst::cols_kernel<T, N, E, 512><<<N / L, L * P.tpl, cols_smem, s>>>(
        work, stw, tw, lam, T(kappa2), T((2.0 / N) * (2.0 / N)));
    KFBI_CUDA_TRY(cudaGetLastError());
    dst::rows_kernel<T, N, E><<<row_blocks, LPC * P.tpl, rows_smem, s>>>(work, work, stw, tw, T(1), N, err,
                                                                      dst::kPollLimit);
    KFBI_CUDA_TRY(cudaGetLastError());
    store_kernel<T><<<gg, 256, 0, s>>>(N, work, v);
    KFBI_CUDA_TRY(cudaGetLastError());
    return KFBI_OK;
  }
};

#define KFBI_STATIC_SIZES(X) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

// one-time work per device: the scratch address and the kernels' shared-memory limits
kfbi_status device_setup(unsigned char** base) {
  int dev = 0;
  KFBI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("kfbi_box_solve_static: device ordinal %d above %d", dev, kMaxDevices - 1);
    return KFBI_ERR_ARG;
  }
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_base[dev]) {
    void* p = nullptr;
    KFBI_CUDA_TRY(cudaGetSymbolAddress(&p, g_box_scratch));
#define KFBI_ATTR(n)                                    \
  KFBI_TRY((Launch<float, n>::attributes()));           \
  KFBI_TRY((Launch<double, n>::attributes()));
    KFBI_STATIC_SIZES(KFBI_ATTR)
#undef KFBI_ATTR
    g_base[dev] = static_cast<unsigned char*>(p);
  }
  *base = g_base[dev];
  return KFBI_OK;
}

template <typename T>
kfbi_status solve_any(int N, unsigned char* base, double h, double kappa2, const double* b,
                      double* v, cudaStream_t s) {
  switch (N) {
#define KFBI_CASE(n) \
  case n: return Launch<T, n>::solve(base, h, kappa2, b, v, s);
    KFBI_STATIC_SIZES(KFBI_CASE)
#undef KFBI_CASE
  }
  set_error("kfbi_box_solve_static: no plan for N = %d", N);
  return KFBI_ERR_ARG;
}

bool supported_n(int N) {
  switch (N) {
#define KFBI_CASE(n) case n:
    KFBI_STATIC_SIZES(KFBI_CASE)
#undef KFBI_CASE
    return true;
  }
  return false;
}

}  // namespace boxstatic
}  // namespace kfbi

extern "C" kfbi_status kfbi_box_solve_static(int N, double lo, double hi, double kappa,
                                             int precision, const double* d_b_grid,
                                             double* d_v_grid, void* stream) {
  using namespace kfbi::boxstatic;
  if (N > kMaxN) {
    kfbi::set_error("kfbi_box_solve_static: N = %d exceeds the static scratch limit N <= %d "
                    "(%zu bytes); use kfbi_setup and kfbi_box_solve", N, kMaxN, kScratchBytes);
    return KFBI_ERR_ARG;
  }
  if (!supported_n(N)) {
    kfbi::set_error("kfbi_box_solve_static: N = %d is not 2^a or 3*2^a with 32 <= N <= %d", N,
                    kMaxN);
    return KFBI_ERR_ARG;
  }
  if (!d_b_grid || !d_v_grid || !(hi > lo) || !(kappa >= 0.0) ||
      (precision != KFBI_FP64 && precision != KFBI_MIXED_FP32)) {
    kfbi::set_error("kfbi_box_solve_static: bad argument (null grid, hi <= lo, kappa < 0 or "
                    "precision not KFBI_FP64 / KFBI_MIXED_FP32)");
    return KFBI_ERR_ARG;
  }
  unsigned char* base = nullptr;
  KFBI_TRY(device_setup(&base));
  const double h = (hi - lo) / N;
  const cudaStream_t s = (cudaStream_t)stream;
  if (precision == KFBI_FP64)
    return solve_any<double>(N, base, h, kappa * kappa, d_b_grid, d_v_grid, s);
  return solve_any<float>(N, base, h, kappa * kappa, d_b_grid, d_v_grid, s);
}

extern "C" kfbi_status kfbi_box_solve_static_check(void* stream) {
  using namespace kfbi::boxstatic;
  unsigned char* base = nullptr;
  KFBI_TRY(device_setup(&base));
  const cudaStream_t s = (cudaStream_t)stream;
  KFBI_CUDA_TRY(cudaStreamSynchronize(s));
  int err = 0;                          // host stack word: a synchronous 4-byte copy
  KFBI_CUDA_TRY(cudaMemcpy(&err, base + kWorkBytes, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    KFBI_CUDA_TRY(cudaMemset(base + kWorkBytes, 0, sizeof(int)));
    kfbi::set_error("kfbi_box_solve_static: a staged line copy of an earlier call did not "
                    "complete (bounded wait expired); its output is wrong");
    return KFBI_ERR_TIMEOUT;
  }
  return KFBI_OK;
}
