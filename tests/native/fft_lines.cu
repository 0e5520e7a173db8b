// Host check of the library's register line FFTs (csrc/fft.cuh, compiled here for the CPU
// through their __host__ paths): every supported length, both directions, FP64 and FP32,
// against the direct DFT sum_n x[n] exp(DIR 2 pi i k n / N) in long double.  Prints one
// line per case: N DIR precision max|X - X_ref| / max|X_ref|.
#include <cmath>
#include <complex>
#include <cstdio>

#include "fft.cuh"

using namespace ltmp2;

template <typename T, int N, int DIR> double check() {
  cpx<T> a[N];
  std::complex<long double> x[N];
  for (int n = 0; n < N; ++n) {
    const T re = (T)std::sin(1.3 * n + 0.1), im = (T)std::cos(0.7 * n * n + 0.2);
    a[n] = {re, im};
    x[n] = {(long double)re, (long double)im};
  }
  LineFFT<T, N, DIR>::run(a);
  const long double two_pi = 6.283185307179586476925286766559L;
  long double err = 0, norm = 0;
  for (int k = 0; k < N; ++k) {
    std::complex<long double> X = 0;
    for (int n = 0; n < N; ++n) {
      const long double ang = DIR * two_pi * (long double)((k * n) % N) / N;
      X += x[n] * std::complex<long double>(std::cos(ang), std::sin(ang));
    }
    const std::complex<long double> got((long double)a[k].x, (long double)a[k].y);
    err = std::fmax(err, std::abs(got - X));
    norm = std::fmax(norm, std::abs(X));
  }
  return (double)(err / norm);
}

template <int N> void row() {
  std::printf("%d -1 f64 %.3e\n", N, check<double, N, -1>());
  std::printf("%d 1 f64 %.3e\n", N, check<double, N, 1>());
  std::printf("%d -1 f32 %.3e\n", N, check<float, N, -1>());
  std::printf("%d 1 f32 %.3e\n", N, check<float, N, 1>());
}

int main() {
  fill_host_twiddles();
  row<8>(); row<10>(); row<12>(); row<16>(); row<18>(); row<20>(); row<24>();
  row<25>(); row<27>(); row<30>(); row<32>(); row<36>(); row<40>();
  return 0;
}
