// Host check of narrow_f64_bits (the integer FP64 -> binary32 / bfloat16
// rounding of the mixed-precision copies) against independent references:
// the host's own FP64 -> FP32 conversion (IEEE 754 round to nearest even),
// and for bfloat16 a rounding written from the definition (the two
// neighbouring representable values, the nearer one, ties to the even
// significand).  Prints "ok <cases>" or the first mismatches; exit status 1
// on any mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "spfd_internal.cuh"

static unsigned ref_bf16(double x) {
  uint64_t u;
  std::memcpy(&u, &x, 8);
  const unsigned sign = (unsigned)(u >> 63) << 15;
  const double ax = std::fabs(x);
  if (std::isinf(ax)) return sign | 0x7f80u;
  if (ax == 0.0) return sign;
  int ex;
  std::frexp(ax, &ex);                      // ax = f * 2^ex, f in [0.5, 1)
  int eq = ex - 8;                          // spacing of 8 significant bits
  if (ex < -125) eq = -133;                 // subnormal spacing
  const double scaled = std::ldexp(ax, -eq);  // exact: a power-of-two scaling
  const double fl = std::floor(scaled), rem = scaled - fl;
  uint64_t q = (uint64_t)fl;
  if (rem > 0.5 || (rem == 0.5 && (q & 1))) ++q;
  const double val = std::ldexp((double)q, eq);
  if (val >= std::ldexp(1.0, 128)) return sign | 0x7f80u;
  const float fv = (float)val;              // exactly representable
  unsigned fb;
  std::memcpy(&fb, &fv, 4);
  return sign | (fb >> 16);
}

int main() {
  long n = 0, bad32 = 0, bad16 = 0;
  auto check = [&](double x) {
    uint64_t u;
    std::memcpy(&u, &x, 8);
    const unsigned g32 = spfd::narrow_f64_bits<23>(u), g16 = spfd::narrow_f64_bits<7>(u);
    if (std::isnan(x)) {
      if (((g32 >> 23) & 0xffu) != 0xffu || !(g32 & 0x7fffffu)) ++bad32;
      if (((g16 >> 7) & 0xffu) != 0xffu || !(g16 & 0x7fu)) ++bad16;
    } else {
      const float f = (float)x;
      unsigned fb;
      std::memcpy(&fb, &f, 4);
      if (g32 != fb && bad32++ < 5) std::printf("binary32 %a: %08x, want %08x\n", x, g32, fb);
      const unsigned r16 = ref_bf16(x);
      if (g16 != r16 && bad16++ < 5) std::printf("bfloat16 %a: %04x, want %04x\n", x, g16, r16);
    }
    ++n;
  };
  std::mt19937_64 rng(2010);
  for (long i = 0; i < 1000000; ++i) {  // uniform bit patterns: every exponent
    const uint64_t u = rng();
    double x;
    std::memcpy(&x, &u, 8);
    check(x);
  }
  std::uniform_real_distribution<double> ud(-1.0, 1.0);
  for (long i = 0; i < 1000000; ++i)  // the target formats' range, subnormals included
    check(ud(rng) * std::ldexp(1.0, (int)(rng() % 300) - 160));
  for (int e = -160; e < 130; ++e)  // exact ties and their neighbours
    for (int k = 0; k < 64; ++k) {
      const double base = std::ldexp(1.0 + k / 64.0, e);
      const double t32 = base + std::ldexp(1.0, e - 24), t16 = base + std::ldexp(1.0, e - 8);
      check(t32); check(-t32); check(std::nextafter(t32, 0.0)); check(std::nextafter(t32, 1e300));
      check(t16); check(-t16); check(std::nextafter(t16, 0.0)); check(std::nextafter(t16, 1e300));
    }
  const double special[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, 3.4028235677973366e38,
                            3.4028234663852886e38, 1.4e-45, 7e-46, 1.1754943508222875e-38,
                            1.1754942106924411e-38, 9.2e-41, 5e-324, -5e-324};
  for (double x : special) check(x);
  if (bad32 || bad16) {
    std::printf("mismatch binary32 %ld bfloat16 %ld of %ld\n", bad32, bad16, n);
    return 1;
  }
  std::printf("ok %ld\n", n);
  return 0;
}
