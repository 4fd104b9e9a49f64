// Host check of the register FFT's 16-point butterflies (dft16 and the FMA-folded
// dft16_fma of paper_1907_13428_gb300/csrc/fftreg.cuh) against the definition of
// the DFT, X_k = sum_j x_j exp(-+2 pi i j k / 16), forward and inverse, in float
// and double. Prints one line per case: "<case> <max relative error>".
#include <cmath>
#include <cstdio>
#include <random>

#include "../paper_1907_13428_gb300/csrc/fftreg.cuh"

using namespace fde;

template <typename C, bool INV, bool FMA>
static double worst_error(std::mt19937_64& gen) {
  using R = decltype(C::x);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  const double pi = 3.14159265358979323846264338327950288;
  double worst = 0.0;
  for (int trial = 0; trial < 500; ++trial) {
    C v[16];
    double xr[16], xi[16];
    for (int j = 0; j < 16; ++j) {
      v[j] = mk<C>((R)u(gen), (R)u(gen));
      xr[j] = (double)v[j].x;
      xi[j] = (double)v[j].y;
    }
    if (FMA)
      dft16_fma<C, INV>(v);
    else
      dft16<C, INV>(v);
    double scale = 0.0, err = 0.0;
    for (int k = 0; k < 16; ++k) {
      long double re = 0.0L, im = 0.0L;
      for (int j = 0; j < 16; ++j) {
        const long double a = (INV ? 2.0L : -2.0L) * (long double)pi * (long double)((j * k) % 16) / 16.0L;
        re += (long double)xr[j] * cosl(a) - (long double)xi[j] * sinl(a);
        im += (long double)xr[j] * sinl(a) + (long double)xi[j] * cosl(a);
      }
      scale = std::fmax(scale, (double)sqrtl(re * re + im * im));
      err = std::fmax(err, std::hypot((double)v[k].x - (double)re, (double)v[k].y - (double)im));
    }
    worst = std::fmax(worst, err / scale);
  }
  return worst;
}

int main() {
  std::mt19937_64 gen(1907);
  std::printf("dft16_double_fwd %.3e\n", worst_error<double2, false, false>(gen));
  std::printf("dft16_double_inv %.3e\n", worst_error<double2, true, false>(gen));
  std::printf("dft16_fma_double_fwd %.3e\n", worst_error<double2, false, true>(gen));
  std::printf("dft16_fma_double_inv %.3e\n", worst_error<double2, true, true>(gen));
  std::printf("dft16_float_fwd %.3e\n", worst_error<float2, false, false>(gen));
  std::printf("dft16_float_inv %.3e\n", worst_error<float2, true, false>(gen));
  std::printf("dft16_fma_float_fwd %.3e\n", worst_error<float2, false, true>(gen));
  std::printf("dft16_fma_float_inv %.3e\n", worst_error<float2, true, true>(gen));
  return 0;
}
