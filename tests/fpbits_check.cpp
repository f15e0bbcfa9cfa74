// Host-side check of the integer bit conversions in csrc/fpbits.cuh against the hardware
// conversions: random bit patterns of every exponent, values at every scale, rounding ties
// and carries, zeros, subnormals, infinities, NaN and the FP32 range edges.  Built and run by
// tests/test_fpbits_host.py; exits nonzero on any mismatch.
#include "fpbits.cuh"
#include <cstdio>
#include <cmath>
#include <random>
#include <limits>
using namespace kfbi;
static bool same(float a, float b) { return fpb_bits(a) == fpb_bits(b) || (std::isnan(a) && std::isnan(b)); }
static bool samed(double a, double b) { return fpb_bits(a) == fpb_bits(b) || (std::isnan(a) && std::isnan(b)); }
int main() {
  long bad = 0, n = 0;
  auto check = [&](double v) {
    float h, l; f64_to_f32_pair(v, h, l);
    const float rh = (float)v; const float rl = (float)(v - (double)rh);
    ++n;
    if (!same(h, rh) || !same(l, rl)) { if (bad < 10) std::printf("pair bad %.17g: %.9g %.9g vs %.9g %.9g\n", v, h, l, rh, rl); ++bad; }
  };
  auto checkf = [&](float f) {
    ++n;
    if (!samed(f32_to_f64(f), (double)f)) { if (bad < 10) std::printf("f2d bad %.9g\n", f); ++bad; }
  };
  std::mt19937_64 rng(7);
  for (int i = 0; i < 4000000; ++i) {            // random bit patterns: every exponent
    const uint64_t u = rng();
    check(fpb_double(u));
    checkf(fpb_float((uint32_t)u));
  }
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (int k = -200; k <= 200; ++k)              // moderate values at every scale
    for (int i = 0; i < 20000; ++i) { const double v = std::ldexp(U(rng), k); check(v); checkf((float)v); }
  // ties and carries: patterns with the low 29 bits at the halfway point, all ones, zero
  for (int i = 0; i < 200000; ++i) {
    uint64_t u = rng() & ~((1ull << 29) - 1);
    const uint64_t lows[] = {0ull, (1ull << 28), (1ull << 28) - 1, (1ull << 28) + 1, (1ull << 29) - 1};
    for (uint64_t lo : lows) { check(fpb_double(u | lo)); }
    // all-ones fraction (carry into the exponent)
    check(fpb_double((u & 0xfff0000000000000ull) | 0x000fffffffffffffull));
  }
  const double sp[] = {0.0, -0.0, 1.0, -1.0, std::numeric_limits<double>::infinity(), -std::numeric_limits<double>::infinity(),
                       std::numeric_limits<double>::quiet_NaN(), std::numeric_limits<double>::denorm_min(), 1e-300, 1e300,
                       (double)std::numeric_limits<float>::max(), (double)std::numeric_limits<float>::min(),
                       std::ldexp(1.0, 127), std::ldexp(1.0, 128), std::ldexp(1.0, -126), std::ldexp(1.0, -149), std::ldexp(1.0, -150),
                       std::nextafter((double)std::numeric_limits<float>::max(), 1e300)};
  for (double v : sp) { check(v); checkf((float)v); }
  std::printf("%ld checks, %ld mismatches\n", n, bad);
  return bad != 0;
}
