// Host driver: the integer FP64 -> FP32 conversions of
// paper_1905_01331_gb300/csrc/f64_bits.cuh against the converting casts
// (round to nearest even) on random bit patterns, values of ordinary
// magnitude and exact ties, and the FP32 -> FP64 conversion on random FP32
// bit patterns (exact, bit for bit).  Prints "<mismatches> <cases>".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#include "../paper_1905_01331_gb300/csrc/f64_bits.cuh"

using namespace ttn::f64b;

int main(int argc, char** argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 1000000;
  std::mt19937_64 g(3);
  long bad = 0, cases = 0;
  auto check = [&](double x) {
    float h, l;
    split(x, h, l);
    const float rh = (float)x, rl = (float)(x - (double)rh), t = to_f32(x);
    ++cases;
    if (std::memcmp(&h, &rh, 4) || std::memcmp(&l, &rl, 4) || std::memcmp(&t, &rh, 4)) ++bad;
  };
  for (long i = 0; i < n; ++i) {
    const uint64_t b = g();
    double x;
    std::memcpy(&x, &b, 8);
    if (!std::isnan(x)) check(x);
    const double y = std::ldexp((double)(g() >> 11) / 9007199254740992.0, (int)(g() % 120) - 80);
    check((g() & 1) ? -y : y);
    const uint64_t t = (g() & 0x800FFFFFE0000000ull) | (1ull << 28) | ((uint64_t)(900 + g() % 300) << 52);
    std::memcpy(&x, &t, 8);
    check(x);
  }
  check(0.0);
  check(-0.0);
  auto check32 = [&](float f) {
    const double d = from_f32(f), r = (double)f;
    ++cases;
    if (std::memcmp(&d, &r, 8)) ++bad;
  };
  for (long i = 0; i < n; ++i) {
    const uint32_t b = (uint32_t)g();
    float f;
    std::memcpy(&f, &b, 4);
    if (!std::isnan(f)) check32(f);
  }
  check32(0.f);
  check32(-0.f);
  std::printf("%ld %ld\n", bad, cases);
  return 0;
}
