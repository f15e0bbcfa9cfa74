// Host-side helpers of the box solver: supported grid sizes and the device tables
// (twiddles e^{-i pi s/N}, eigenvalues of the 1-D second difference).  The kernels are in
// dst_impl.cuh, instantiated per precision by dst_f32.cu and dst_f64.cu.
#include "kfbi_internal.cuh"

namespace kfbi {

// ---------------------------------------------------------------------------- plan
bool make_fft_plan(int N, FftPlan* p) {
  // grid sizes with a compiled plan: 2^a (32..8192) and 3 * 2^a (48..6144)
  if (N < 32 || N > 8192) return false;
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

}  // namespace kfbi
