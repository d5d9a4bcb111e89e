// Host check of the double-float arithmetic and its FP64 conversions (eq_dd.cuh, host branches):
// prints the worst errors found against long double on seeded random operands, then the round
// trips of special values.  Compiled and run by tests/test_dd_host.py.
#include <cmath>
#include <cstdio>
#include <random>

#include "eq_dd.cuh"

using eqk::dd;

int main() {
  std::mt19937_64 rng(20210501);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double conv = 0, trip = 0, add = 0, mul = 0, conv2 = 0, agree = 0;
  for (int i = 0; i < 1000000; ++i) {
    const double a = U(rng) * std::pow(10.0, static_cast<int>(rng() % 30) - 15);
    const double b = U(rng) * std::pow(10.0, static_cast<int>(rng() % 30) - 15);
    const dd A = eqk::dd_from_bits(a), B = eqk::dd_from_bits(b);
    const double ra = eqk::dd_to_bits(A), rb = eqk::dd_to_bits(B);
    conv = std::fmax(conv, std::fabs(ra - a) / std::fabs(a));
    // the FP64-instruction forms: conversion error and agreement with the bit forms
    const double r2 = eqk::dd_to_f64(eqk::dd_from_f64(a));
    conv2 = std::fmax(conv2, std::fabs(r2 - a) / std::fabs(a));
    agree = std::fmax(agree, std::fabs(eqk::dd_to_f64(A) - ra) / std::fabs(ra));
    // a double-float that came from a double goes back and forth unchanged
    trip = std::fmax(trip, std::fabs(eqk::dd_to_bits(eqk::dd_from_bits(ra)) - ra) / std::fabs(ra));
    const long double se = static_cast<long double>(ra) + rb, pe = static_cast<long double>(ra) * rb;
    const double s = eqk::dd_to_bits(A + B), p = eqk::dd_to_bits(A * B);
    add = std::fmax(add, static_cast<double>(std::fabs(s - se) / (std::fabs(static_cast<long double>(ra)) + std::fabs(static_cast<long double>(rb)))));
    if (std::fabs(pe) > 1e-25L) mul = std::fmax(mul, static_cast<double>(std::fabs(p - pe) / std::fabs(pe)));
  }
  std::printf("conv %.6g\ntrip %.6g\nadd %.6g\nmul %.6g\nconv2 %.6g\nagree %.6g\n", conv, trip, add, mul,
              conv2, agree);
  const double sp2[] = {INFINITY, -1e300, 1e-300};
  for (double v : sp2)
    std::printf("special2 %.17g %.17g\n", v, eqk::dd_to_f64(eqk::dd_from_f64(v)));
  const double sp[] = {0.0, -0.0, 1.0, -2.5, 0.1, 1e30, -1e-30, 123456789.123456789, INFINITY, -INFINITY};
  for (double v : sp) std::printf("special %.17g %.17g\n", v, eqk::dd_to_bits(eqk::dd_from_bits(v)));
  const dd n = eqk::dd_from_bits(NAN);
  std::printf("nan %d\n", std::isnan(eqk::dd_to_bits(n)) ? 1 : 0);
  return 0;
}
