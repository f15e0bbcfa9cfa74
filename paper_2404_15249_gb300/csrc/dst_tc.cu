// Box solve of Alg. 4 in its dense form on the tensor cores: with the sine matrix
// S[l][i] = sin(pi l i / N) (zero in row and column 0, so the N x N work grid is used as
// it is), the full diagonalisation is four GEMMs
//     T1 = (B S)^T,  X2 = (T1 S) / (lambda_l + lambda_m - kappa^2) (2/N)^2,
//     T3 = (X2 S)^T, V = T3 S,
// each C = A S^T (S symmetric) with A and S K-major.  The GEMMs run on tcgen05: operands
// in shared memory in the canonical K-major layout without swizzle (core matrices of
// 8 rows x 16 bytes), the FP32 accumulator in tensor memory, MMAs issued by one thread and
// tracked by an mbarrier per shared-memory stage (two stages: the next K chunk is staged
// while the MMAs of the current one run).  TF32 with a three-term split
// (A_hi S_hi + A_hi S_lo + A_lo S_hi, hi = TF32 rounding, lo = TF32 of the remainder) keeps
// FP32-class accuracy.  Every wait is bounded; tensor memory is released on every path.
#include <atomic>

#include "kfbi_internal.cuh"

namespace kfbi {
namespace {

constexpr int BM = 128, BN = 64, KC = 32;          // CTA tile and K chunk
constexpr int A_BYTES = BM * KC * 4, B_BYTES = BN * KC * 4;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // A hi, A lo, S hi, S lo
constexpr int SMEM_BYTES = 2 * STAGE_BYTES;               // two stages: 96 KB
constexpr int TC_THREADS = 128;

__device__ __forceinline__ uint32_t sm_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of an R x KC chunk, k a multiple of 4 (16-byte group)
__device__ __forceinline__ int canon(int r, int k) {
  return (((r >> 3) * (KC / 4) + (k >> 2)) << 7) + ((r & 7) << 4);
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  constexpr uint32_t LBO = 128, SBO = (KC / 4) * 128;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(LBO >> 4) << 16) |
         ((uint64_t)(SBO >> 4) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, M = 128, N = 64
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ float tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = sm_addr(bar);
  for (int i = 0; i < (1 << 20); ++i) {
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

// S hi / lo tables, S[l][i] = sin(pi l i / N) for l, i >= 1 (row and column 0 zero)
__global__ void sine_split_kernel(int N, float* shi, float* slo) {
  const long n = (long)N * N;
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const int l = (int)(q / N), i = (int)(q - (q / N) * N);
    double s = 0.0;
    if (l > 0 && i > 0) s = sinpi((double)(((long)l * i) % (2L * N)) / (double)N);
    const float hi = tf32((float)s);
    shi[q] = hi;
    slo[q] = tf32((float)(s - (double)hi));
  }
}

// C[r][c] = sum_k A[r][k] S[c][k] on the tile rows [m0, m0+128), columns [n0, n0+64).
// mode 0: out[r][c] = C;  mode 1: out[c][r] = C;  mode 2: out[r][c] = C * scale /
// (lam[r] + lam[c] - kappa2), zero where r or c is 0.
__global__ void __launch_bounds__(TC_THREADS, 1)
    dst_gemm_kernel(const float* __restrict__ A, const float* __restrict__ shi,
                    const float* __restrict__ slo, float* __restrict__ out, int N, int mode,
                    const float* __restrict__ lam, float kappa2, float scale, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sm_addr(&tbase)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sm_addr(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  const int nchunks = N / KC;
  int uses[2] = {0, 0}, waits[2] = {0, 0};
  bool ok = true;

  auto stage = [&](int s, int kc) {
    unsigned char* base = smem + s * STAGE_BYTES;
    unsigned char* ahi = base;
    unsigned char* alo = base + A_BYTES;
    unsigned char* bhi = base + 2 * A_BYTES;
    unsigned char* blo = base + 2 * A_BYTES + B_BYTES;
    // A: thread t takes row t, eight groups of 4 values (one 128-byte row segment)
    const float* arow = A + (size_t)(m0 + tid) * N + kc;
#pragma unroll
    for (int g = 0; g < KC / 4; ++g) {
      const float4 v = *reinterpret_cast<const float4*>(arow + 4 * g);
      const float4 h = make_float4(tf32(v.x), tf32(v.y), tf32(v.z), tf32(v.w));
      const float4 l = make_float4(tf32(v.x - h.x), tf32(v.y - h.y), tf32(v.z - h.z), tf32(v.w - h.w));
      const int o = canon(tid, 4 * g);
      *reinterpret_cast<float4*>(ahi + o) = h;
      *reinterpret_cast<float4*>(alo + o) = l;
    }
    // S: threads 0..63 take rows n0 + t of the hi table, 64..127 those of the lo table
    const int r = tid & (BN - 1);
    const float* srow = (tid < BN ? shi : slo) + (size_t)(n0 + r) * N + kc;
    unsigned char* dst = tid < BN ? bhi : blo;
#pragma unroll
    for (int g = 0; g < KC / 4; ++g)
      *reinterpret_cast<float4*>(dst + canon(r, 4 * g)) = *reinterpret_cast<const float4*>(srow + 4 * g);
  };

  auto issue = [&](int s, bool first) {
    unsigned char* base = smem + s * STAGE_BYTES;
    const uint32_t ahi = sm_addr(base), alo = ahi + A_BYTES;
    const uint32_t bhi = sm_addr(base + 2 * A_BYTES), blo = bhi + B_BYTES;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int term = 0; term < 3; ++term) {
      const uint32_t a = term == 2 ? alo : ahi;
      const uint32_t b = term == 1 ? blo : bhi;
#pragma unroll
      for (int ks = 0; ks < KC / 8; ++ks) {
        const uint64_t ad = smem_desc(a + ks * 256), bd = smem_desc(b + ks * 256);
        const uint32_t acc = (first && term == 0 && ks == 0) ? 0u : 1u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     sm_addr(&bar[s]))
                 : "memory");
  };

  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;
    if (uses[s] > waits[s]) {                 // the MMAs that read this stage are done
      ok = bar_wait(&bar[s], (uint32_t)(waits[s] & 1)) && ok;
      ++waits[s];
    }
    stage(s, c * KC);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) issue(s, c == 0);
    ++uses[s];
  }
  for (int s = 0; s < 2; ++s)
    while (uses[s] > waits[s]) {
      ok = bar_wait(&bar[s], (uint32_t)(waits[s] & 1)) && ok;
      ++waits[s];
    }
  if (!ok && lane == 0) atomicOr(err, 2);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // epilogue: warp w holds rows m0 + 32 w + lane, 16 columns per load
  const int row = m0 + warp * 32 + lane;
  const float lr = (mode == 2) ? lam[row] - kappa2 : 0.f;
#pragma unroll
  for (int c0 = 0; c0 < BN; c0 += 16) {
    uint32_t v[16];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (mode == 1) {
#pragma unroll
      for (int j = 0; j < 16; ++j) out[(size_t)(n0 + c0 + j) * N + row] = __uint_as_float(v[j]);
    } else {
      float x[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        x[j] = __uint_as_float(v[j]);
        if (mode == 2) {
          const int col = n0 + c0 + j;
          x[j] = (row == 0 || col == 0) ? 0.f : x[j] * scale / (lr + lam[col]);
        }
      }
      float4* o = reinterpret_cast<float4*>(out + (size_t)row * N + n0 + c0);
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN)
                 : "memory");
}

kfbi_status gemm(Ctx& c, const float* A, float* out, int mode) {
  static std::atomic<bool> attr{false};
  if (!attr) {
    KFBI_CUDA_TRY(cudaFuncSetAttribute(dst_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES));
    attr = true;
  }
  const int N = c.N;
  const float scale = (float)((2.0 / N) * (2.0 / N));
  const int pr = prof_begin(c, ST_TC);
  dst_gemm_kernel<<<dim3(N / BN, N / BM), TC_THREADS, SMEM_BYTES, c.stream>>>(
      A, c.tc_shi, c.tc_slo, out, N, mode, c.t32.lam, (float)c.kappa2, scale, c.err_flag + 2);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

}  // namespace

bool tc_supported(const Ctx& c) { return c.dim == 2 && c.N % BM == 0 && c.N <= 4096; }

kfbi_status init_tc_tables(Ctx& c) {
  if (!tc_supported(c)) return KFBI_OK;
  const size_t n = (size_t)c.N * c.N;
  KFBI_TRY(alloc_bytes(c, (void**)&c.tc_shi, sizeof(float) * n));
  KFBI_TRY(alloc_bytes(c, (void**)&c.tc_slo, sizeof(float) * n));
  prof_count(c, ST_SETUP);
  sine_split_kernel<<<4096, 256, 0, c.stream>>>(c.N, c.tc_shi, c.tc_slo);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status box_solve_tc(Ctx& c, const float* rhs, float* work) {
  if (!tc_supported(c) || !c.tc_shi) {
    set_error("tensor-core box solve: 2-D grids with N a multiple of %d up to 4096 only", BM);
    return KFBI_ERR_UNSUPPORTED;
  }
  float* X = reinterpret_cast<float*>(c.XT);
  KFBI_TRY(gemm(c, rhs, X, 1));     // T1 = (B S)^T
  KFBI_TRY(gemm(c, X, work, 2));    // X2 = T1 S / (lambda_l + lambda_m - kappa^2) (2/N)^2
  KFBI_TRY(gemm(c, work, X, 1));    // T3 = (X2 S)^T
  return gemm(c, X, work, 0);       // V = T3 S
}

}  // namespace kfbi
