// Box solve of Alg. 4 in its dense form on the tensor cores: with the sine matrix
// S[l][i] = sin(pi l i / N) (zero in row and column 0, so the work grid is used as it is),
// the full diagonalisation is a chain of GEMMs C = A S^T (S symmetric, A and S K-major).
// 2-D (B[j][i]):  T1 = (B S)^T,  X2 = (T1 S) / (lambda_l + lambda_m - kappa^2) (2/N)^2,
//                 T3 = (X2 S)^T, V = T3 S.
// 3-D (B[k][j][i] as an N^2 x N matrix): each GEMM transforms the fastest axis and writes
// its result transposed (N x N^2), which moves the next axis to the front:
//   (k,j,i) -> (l,k,j) -> (m,l,k) -> (n,m,l) with the division by
//   lambda_l + lambda_m + lambda_n - kappa^2 and (2/N)^3 in the third epilogue, then the
//   three inverse transforms back to (k,j,i).  TF32 with a three-term split
// (A_hi S_hi + A_hi S_lo + A_lo S_hi, hi = TF32 rounding, lo = TF32 of the exact FP32
// remainder) keeps FP32-class accuracy.  Every operand is kept in global memory as its
// (hi, lo) pair: S once at setup, the right-hand side by one split pass, and each GEMM's
// epilogue writes the pair of its output for the next GEMM, so the main loop only copies.
//
// GEMM kernel: one 128 x BN output tile per CTA, warp-specialised.  The producer fills a
// ring of ST shared-memory stages with K chunks of 16 and signals each stage on its "full"
// mbarrier: either one thread issuing four TMA tensor loads per chunk (64-byte swizzled
// K-major tiles, completion counted in bytes on the mbarrier), or two producer warps with
// 16-byte cp.async into the canonical K-major no-swizzle form (core matrices of 8 rows x
// 16 bytes; copy q of a tile lands at byte 16 q).  One thread of warp 4 waits on it,
// issues the tcgen05.mma (kind::tf32) of the chunk with the FP32 accumulators in tensor
// memory and commits them to the stage's "empty" mbarrier, which the producers wait on
// before they refill the stage; warps 0-3 then read the accumulators for the epilogue.
// Every mbarrier wait is bounded; tensor memory is released on every path.
#include <cuda.h>

#include <atomic>
#include <cstdlib>

#include "kfbi_internal.cuh"

namespace kfbi {
namespace {

constexpr int BM = 128, KC = 16;
constexpr int A_BYTES = BM * KC * 4;                // one part (hi or lo) of an A chunk

template <int BN>
struct Tile {
  static constexpr int B_BYTES = BN * KC * 4;
  static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;     // A hi, A lo, S hi, S lo
  static constexpr int ST = (192 * 1024) / STAGE;              // stages in 192 KB
  static constexpr int SMEM = ST * STAGE;
  // partial accumulators in tensor memory (all 512 columns): chunk c adds into c % NACC.
  // The tensor core's FP32 accumulation is not round-to-nearest; splitting the K sum
  // into NACC partial sums, added in the epilogue, divides its systematic drift by NACC.
  static constexpr int NACC = 512 / BN;
  // instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, M = 128, N = BN
  static constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static_assert(ST >= 3, "pipeline depth");
};

__device__ __forceinline__ uint32_t sm_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  constexpr uint32_t LBO = 128, SBO = (KC / 4) * 128;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(LBO >> 4) << 16) |
         ((uint64_t)(SBO >> 4) << 32) | ((uint64_t)1 << 46);
}

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

// FP32 values -> TF32 (hi, lo) pair
__global__ void split_tf32_kernel(long n, const float* __restrict__ x, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const float v = x[q], h = tf32(v);
    hi[q] = h;
    lo[q] = tf32(v - h);
  }
}

constexpr int PRODUCERS = 64;                  // warps 5 and 6
constexpr int GEMM_THREADS = 128 + 32 + PRODUCERS;   // epilogue warps 0-3, MMA warp 4

// copy rows [r0, r0 + R) x columns [kc, kc + KC) of a row-major N x N matrix into the
// canonical layout at dst: copy q (row r0 + 8 (q / (2 KC)) + q % 8, column group
// (q / 8) % (KC / 4)) lands at byte 16 q; producer thread pt takes q = pt, pt + 64, ...
template <int R>
__device__ __forceinline__ void copy_tile(uint32_t dst, const float* __restrict__ src, int N,
                                          int r0, int kc, int pt) {
#pragma unroll
  for (int it = 0; it < R * (KC / 4) / PRODUCERS; ++it) {
    const int q = it * PRODUCERS + pt;
    const int r = r0 + (q / (2 * KC)) * 8 + (q & 7), g = (q >> 3) & (KC / 4 - 1);
    const float* p = src + (size_t)r * N + kc + 4 * g;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * q), "l"(p)
                 : "memory");
  }
}

// shared-memory descriptor of a K-major tile written by TMA with the 64-byte swizzle: rows
// of 64 bytes (KC = 16 values), 8-row atoms of 512 bytes, descriptor version 1
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}

// TMA: rows [y, y + box) x columns [x, x + KC) of the tensor map's matrix into dst
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(sm_addr(bar))
      : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(bar)), "r"(count) : "memory");
}

// C[r][c] = sum_k A[r][k] S[c][k] on the tile rows [m0, m0+128), columns [n0, n0+BN) of
// an M x N result (A: M x N, S: N x N), A and S given as TF32 (hi, lo) pairs.
// mode 0: out[r][c] = C (M = N);  mode 1: out[c][r] = C;  mode 2 (M = N): out[r][c] =
// C * scale / (lam[r] + lam[c] - kappa2), zero where r or c is 0;  mode 3 (M = N^2):
// out[c][r] = C * scale / (lam[r % N] + lam[r / N] + lam[c] - kappa2), zero where any of
// the three indices is 0.  With out_lo non-null the output is written as its TF32 pair
// (out, out_lo), else as FP32 values.
template <int BN, bool TMA>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    dst_gemm_kernel(const float* __restrict__ ahi, const float* __restrict__ alo,
                    const float* __restrict__ shi, const float* __restrict__ slo,
                    const __grid_constant__ CUtensorMap map_ahi,
                    const __grid_constant__ CUtensorMap map_alo,
                    const __grid_constant__ CUtensorMap map_shi,
                    const __grid_constant__ CUtensorMap map_slo,
                    float* __restrict__ out, float* __restrict__ out_lo, int M, int N, int mode,
                    const float* __restrict__ lam, float kappa2, float scale, int* err) {
  using TL = Tile<BN>;
  constexpr int ST = TL::ST;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[ST];
  __shared__ __align__(8) uint64_t empty[ST];
  __shared__ __align__(8) uint64_t done;
  __shared__ uint32_t tbase;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     sm_addr(&tbase)),
                 "r"(BN * TL::NACC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      bar_init(&full[s], TMA ? 1 : PRODUCERS);
      bar_init(&empty[s], 1);
    }
    bar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tbase;
  const uint32_t sbase = sm_addr(smem);
  const int nchunks = N / KC;
  bool ok = true;
  // the swizzled TMA tiles need stage bases on 512-byte boundaries
  const bool aligned = !TMA || (sbase & 511u) == 0;

  if (TMA && tid == 160) {
    if (!aligned) atomicOr(err, 4);
#pragma unroll 1
    for (int c = 0; aligned && c < nchunks; ++c) {
      const int s = c % ST;
      if (c >= ST) ok = bar_wait(&empty[s], (uint32_t)((c / ST - 1) & 1)) && ok;
      const uint32_t st = sbase + (uint32_t)(s * TL::STAGE);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(&full[s])),
                   "r"((uint32_t)TL::STAGE)
                   : "memory");
      const int kc = c * KC;
      tma_load(st, &map_ahi, kc, m0, &full[s]);
      tma_load(st + A_BYTES, &map_alo, kc, m0, &full[s]);
      tma_load(st + 2 * A_BYTES, &map_shi, kc, n0, &full[s]);
      tma_load(st + 2 * A_BYTES + TL::B_BYTES, &map_slo, kc, n0, &full[s]);
    }
  } else if (!TMA && tid >= 160) {
    // producers: chunk c into stage c % ST once the MMAs of chunk c - ST have read it
    const int pt = tid - 160;
#pragma unroll 1
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % ST;
      if (c >= ST) ok = bar_wait(&empty[s], (uint32_t)((c / ST - 1) & 1)) && ok;
      const uint32_t st = sbase + (uint32_t)(s * TL::STAGE);
      const int kc = c * KC;
      copy_tile<BM>(st, ahi, N, m0, kc, pt);
      copy_tile<BM>(st + A_BYTES, alo, N, m0, kc, pt);
      copy_tile<BN>(st + 2 * A_BYTES, shi, N, n0, kc, pt);
      copy_tile<BN>(st + 2 * A_BYTES + TL::B_BYTES, slo, N, n0, kc, pt);
      // arrives on full[s] once this thread's copies so far have landed
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(sm_addr(&full[s]))
                   : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (tid == 128) {
    // MMA issuer (warp 4, one thread)
#pragma unroll 1
    for (int c = 0; aligned && c < nchunks; ++c) {
      const int s = c % ST;
      ok = bar_wait(&full[s], (uint32_t)((c / ST) & 1)) && ok;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t st = sbase + (uint32_t)(s * TL::STAGE);
      const uint32_t a_hi = st, a_lo = st + A_BYTES;
      const uint32_t b_hi = st + 2 * A_BYTES, b_lo = b_hi + TL::B_BYTES;
      const uint32_t d = tmem + (uint32_t)((c % TL::NACC) * BN);
#pragma unroll
      for (int term = 0; term < 3; ++term) {
        const uint32_t a = term == 2 ? a_lo : a_hi;
        const uint32_t b = term == 1 ? b_lo : b_hi;
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          // K step of 8 values: 32 bytes along a swizzled row, or two core matrices
          const uint64_t ad = TMA ? smem_desc_sw64(a + ks * 32) : smem_desc(a + ks * 256);
          const uint64_t bd = TMA ? smem_desc_sw64(b + ks * 32) : smem_desc(b + ks * 256);
          const uint32_t acc = (c < TL::NACC && term == 0 && ks == 0) ? 0u : 1u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
              "l"(ad), "l"(bd), "r"(TL::IDESC), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       sm_addr(&empty[s]))
                   : "memory");
    }
    // completes once every MMA above has
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     sm_addr(&done))
                 : "memory");
  }
  if (tid < 128) {
    ok = bar_wait(&done, 0u) && ok;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok) atomicOr(err, 2);

  if (tid < 128) {
    // epilogue: warp w holds rows m0 + 32 w + lane, 16 columns per load; the partial sums
    // are added pairwise
    const int row = m0 + warp * 32 + lane;
    // row part of the divisor; zero_row: a boundary mode in the row index
    float lr = 0.f;
    bool zero_row = false;
    if (mode == 2) {
      lr = lam[row] - kappa2;
      zero_row = row == 0;
    } else if (mode == 3) {
      const int ri = row % N, rj = row / N;
      lr = lam[ri] + lam[rj] - kappa2;
      zero_row = ri == 0 || rj == 0;
    }
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float x[16];
      float part[TL::NACC][16];
#pragma unroll
      for (int a = 0; a < TL::NACC; ++a) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(a * BN + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
            "[%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
              "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) part[a][j] = __uint_as_float(v[j]);
      }
#pragma unroll
      for (int w = 1; w < TL::NACC; w *= 2)
#pragma unroll
        for (int a = 0; a + w < TL::NACC; a += 2 * w)
#pragma unroll
          for (int j = 0; j < 16; ++j) part[a][j] += part[a + w][j];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        x[j] = part[0][j];
        if (mode >= 2) {
          const int col = n0 + c0 + j;
          float r;
          asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(lr + lam[col]));
          x[j] = (zero_row || col == 0) ? 0.f : x[j] * scale * r;
        }
      }
      if (mode == 1 || mode == 3) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const size_t o = (size_t)(n0 + c0 + j) * M + row;
          if (out_lo) {
            const float h = tf32(x[j]);
            out[o] = h;
            out_lo[o] = tf32(x[j] - h);
          } else {
            out[o] = x[j];
          }
        }
      } else {
        const size_t o = (size_t)row * N + n0 + c0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          float4 w = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
          if (out_lo) {
            const float4 h = make_float4(tf32(w.x), tf32(w.y), tf32(w.z), tf32(w.w));
            *reinterpret_cast<float4*>(out_lo + o + 4 * j) =
                make_float4(tf32(w.x - h.x), tf32(w.y - h.y), tf32(w.z - h.z), tf32(w.w - h.w));
            w = h;
          }
          *reinterpret_cast<float4*>(out + o + 4 * j) = w;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(BN * TL::NACC)
                 : "memory");
}

// Tensor maps of the GEMM operands (2-D views, rows x N values, 64-byte swizzle, boxes of
// KC columns): the TF32 pairs in (H32, D32) and in the two halves of XT with 128-row boxes,
// the sine tables with BN-row boxes.  Encoded once at setup through the driver entry point.
struct TcMaps {
  CUtensorMap a_hi[2], a_lo[2], s_hi, s_lo;
  const float* a_base[2];          // H32 and the first half of XT: which pair a GEMM reads
  int bn;
};

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool encode_map(EncodeTiled enc, CUtensorMap* m, const float* base, long rows, int cols,
                int box_rows) {
  const cuuint64_t dim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t stride[1] = {(cuuint64_t)cols * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dim, stride, box,
             estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tile width of the context: 128 x 256 where it fills the GPU (2-D N >= 2048, 3-D N^2 rows),
// else 128 x 64
int tile_bn(const Ctx& c) {
  const bool wide = c.N >= 2048 || c.dim == 3;
  return wide ? (c.N % 256 == 0 ? 256 : 128) : 64;
}

template <int BN>
kfbi_status gemm_n(Ctx& c, const float* ahi, const float* alo, float* out, float* out_lo,
                   int mode) {
  static_assert(BN == 64 || BN == 128 || BN == 256, "tile width");
  KFBI_TRY(set_smem_limit((const void*)dst_gemm_kernel<BN, true>, Tile<BN>::SMEM));
  KFBI_TRY(set_smem_limit((const void*)dst_gemm_kernel<BN, false>, Tile<BN>::SMEM));
  const int N = c.N, M = c.dim == 3 ? N * N : N;
  const double s1 = 2.0 / N;
  const float scale = (float)(c.dim == 3 ? s1 * s1 * s1 : s1 * s1);
  // TMA loads when the operand pair has tensor maps (KFBI_TC_CPASYNC=1 forces the cp.async
  // producers, for comparison)
  static const bool force_cpasync = [] {
    const char* e = std::getenv("KFBI_TC_CPASYNC");
    return e && e[0] == '1';
  }();
  const TcMaps* tm = reinterpret_cast<const TcMaps*>(c.tc_maps);
  const int pair = (tm && ahi == tm->a_base[0]) ? 0 : ((tm && ahi == tm->a_base[1]) ? 1 : -1);
  const bool tma = tm && pair >= 0 && tm->bn == BN && !force_cpasync;
  static const CUtensorMap zero_map{};
  const int pr = prof_begin(c, ST_TC);
  if (tma)
    dst_gemm_kernel<BN, true><<<dim3(N / BN, M / BM), GEMM_THREADS, Tile<BN>::SMEM, c.stream>>>(
        ahi, alo, c.tc_shi, c.tc_slo, tm->a_hi[pair], tm->a_lo[pair], tm->s_hi, tm->s_lo, out,
        out_lo, M, N, mode, c.t32.lam, (float)c.kappa2, scale, c.err_flag + 2);
  else
    dst_gemm_kernel<BN, false><<<dim3(N / BN, M / BM), GEMM_THREADS, Tile<BN>::SMEM, c.stream>>>(
        ahi, alo, c.tc_shi, c.tc_slo, zero_map, zero_map, zero_map, zero_map, out, out_lo, M, N,
        mode, c.t32.lam, (float)c.kappa2, scale, c.err_flag + 2);
  prof_end(c, pr);
  KFBI_CUDA_TRY(cudaGetLastError());
  return KFBI_OK;
}

kfbi_status gemm(Ctx& c, const float* ahi, const float* alo, float* out, float* out_lo, int mode) {
  switch (tile_bn(c)) {
    case 256: return gemm_n<256>(c, ahi, alo, out, out_lo, mode);
    case 128: return gemm_n<128>(c, ahi, alo, out, out_lo, mode);
    default: return gemm_n<64>(c, ahi, alo, out, out_lo, mode);
  }
}

}  // namespace

// 2-D: N a multiple of 128 up to 8192; 3-D: N a multiple of 128 up to 512
bool tc_supported(const Ctx& c) {
  return c.N % BM == 0 && ((c.dim == 2 && c.N <= 8192) || (c.dim == 3 && c.N <= 512));
}

kfbi_status init_tc_tables(Ctx& c) {
  if (!tc_supported(c)) return KFBI_OK;
  const size_t n = (size_t)c.N * c.N;
  KFBI_TRY(alloc_bytes(c, (void**)&c.tc_shi, sizeof(float) * n));
  KFBI_TRY(alloc_bytes(c, (void**)&c.tc_slo, sizeof(float) * n));
  prof_count(c, ST_SETUP);
  sine_split_kernel<<<4096, 256, 0, c.stream>>>(c.N, c.tc_shi, c.tc_slo);
  KFBI_CUDA_TRY(cudaGetLastError());
  // tensor maps for the TMA producer; without the driver entry point the GEMMs fall back to
  // the cp.async producers
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return KFBI_OK;
  }
  const EncodeTiled enc = reinterpret_cast<EncodeTiled>(fn);
  TcMaps* tm = new (std::nothrow) TcMaps();
  if (!tm) return KFBI_OK;
  const long rows = c.dim == 3 ? (long)c.N * c.N : c.N;
  const long total = rows * c.N;
  const float* xt = reinterpret_cast<const float*>(c.XT);
  tm->bn = tile_bn(c);
  tm->a_base[0] = c.H32;
  tm->a_base[1] = xt;
  const bool ok = encode_map(enc, &tm->a_hi[0], c.H32, rows, c.N, BM) &&
                  encode_map(enc, &tm->a_lo[0], c.D32, rows, c.N, BM) &&
                  encode_map(enc, &tm->a_hi[1], xt, rows, c.N, BM) &&
                  encode_map(enc, &tm->a_lo[1], xt + total, rows, c.N, BM) &&
                  encode_map(enc, &tm->s_hi, c.tc_shi, c.N, c.N, tm->bn) &&
                  encode_map(enc, &tm->s_lo, c.tc_slo, c.N, c.N, tm->bn);
  if (!ok) {
    delete tm;
    return KFBI_OK;
  }
  c.tc_maps = tm;
  return KFBI_OK;
}

void free_tc(Ctx& c) {
  delete reinterpret_cast<TcMaps*>(c.tc_maps);
  c.tc_maps = nullptr;
}

// rhs and work: FP32 work grids (N^2 or N^3, may be the same buffer).  Scratch: the TF32
// pairs live in H32 / D32 and in the two halves of XT.
kfbi_status box_solve_tc(Ctx& c, const float* rhs, float* work) {
  if (!tc_supported(c) || !c.tc_shi) {
    set_error("tensor-core box solve: N a multiple of %d, up to 8192 in 2-D and 512 in 3-D", BM);
    return KFBI_ERR_UNSUPPORTED;
  }
  const long n = (long)c.N * c.N * (c.dim == 3 ? c.N : 1);
  float* phi = c.H32;
  float* plo = c.D32;
  float* qhi = reinterpret_cast<float*>(c.XT);
  float* qlo = qhi + n;
  prof_count(c, ST_TC);
  split_tf32_kernel<<<(int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192), 256, 0, c.stream>>>(
      n, rhs, phi, plo);
  KFBI_CUDA_TRY(cudaGetLastError());
  if (c.dim == 2) {
    KFBI_TRY(gemm(c, phi, plo, qhi, qlo, 1));     // T1 = (B S)^T
    KFBI_TRY(gemm(c, qhi, qlo, phi, plo, 2));     // X2 = T1 S / (lambda_l + lambda_m - kappa^2) (2/N)^2
    KFBI_TRY(gemm(c, phi, plo, qhi, qlo, 1));     // T3 = (X2 S)^T
    return gemm(c, qhi, qlo, work, nullptr, 0);   // V = T3 S
  }
  KFBI_TRY(gemm(c, phi, plo, qhi, qlo, 1));       // (k,j,i) -> (l,k,j)
  KFBI_TRY(gemm(c, qhi, qlo, phi, plo, 1));       // -> (m,l,k)
  KFBI_TRY(gemm(c, phi, plo, qhi, qlo, 3));       // -> (n,m,l), divided
  KFBI_TRY(gemm(c, qhi, qlo, phi, plo, 1));       // inverse: -> (i,n,m)
  KFBI_TRY(gemm(c, phi, plo, qhi, qlo, 1));       // -> (j,i,n)
  return gemm(c, qhi, qlo, work, nullptr, 1);     // -> (k,j,i)
}

}  // namespace kfbi
