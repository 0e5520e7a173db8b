// Register-resident mixed-radix line FFTs (radices 2, 3, 4, 5) for the batched
// 3D FFTs of the LTMP2 hot path: orbitals and transformed states to real space
// (Sec. II A, the inverse transform of the plane-wave coefficients) and the
// co-density transforms of Eq. (SCHovrlp) applied to phi_i^* w_j (Sec. II B).
//
// One thread owns one line of N points in registers.  The Cooley-Tukey split
// N = R * M (decimation in time) is unrolled at compile time, so every twiddle
// index is a constant and the twiddle operand comes straight from the
// constant bank.  Conventions (unnormalised both ways):
//   forward  X[k] = sum_n x[n] exp(-2 pi i k n / N)      (DIR = -1)
//   inverse  x[n] = sum_k X[k] exp(+2 pi i k n / N)      (DIR = +1)
#pragma once
#include <cuda_runtime.h>
#include <cmath>

namespace ltmp2 {

// Aligned to its full size, so that a complex value moves as one 64-bit (float) or 128-bit
// (double) access in shared and global memory: with 4-byte alignment every complex load
// split into two 32-bit accesses, which 2-way bank-conflict at the even word strides of the
// plane and column layouts.
template <typename T> struct alignas(2 * sizeof(T)) cpx { T x, y; };

template <typename T> __host__ __device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __host__ __device__ __forceinline__ cpx<T> cmulconj(cpx<T> a, cpx<T> b) {  // a * conj(b)
  return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename T> __host__ __device__ __forceinline__ cpx<T> cconj(cpx<T> a) { return {a.x, -a.y}; }
template <typename T> __host__ __device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return {a.x * s, a.y * s}; }
// multiply by DIR * i  (DIR = -1: -i, DIR = +1: +i)
template <int DIR, typename T> __host__ __device__ __forceinline__ cpx<T> mul_i(cpx<T> a) {
  return DIR > 0 ? cpx<T>{-a.y, a.x} : cpx<T>{a.y, -a.x};
}

// ---------------------------------------------------------------- twiddle tables
// Supported line lengths (5-smooth).  The table holds exp(-2 pi i k / N),
// k = 0..N-1, for each N, filled once per device from host double cos/sin.
constexpr int kFftSizes[] = {8, 10, 12, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40};
constexpr int kNumFftSizes = sizeof(kFftSizes) / sizeof(int);
__host__ __device__ constexpr int tw_size_at(int i) {
  return i == 0 ? 8 : i == 1 ? 10 : i == 2 ? 12 : i == 3 ? 16 : i == 4 ? 18 : i == 5 ? 20 : i == 6 ? 24
       : i == 7 ? 25 : i == 8 ? 27 : i == 9 ? 30 : i == 10 ? 32 : i == 11 ? 36 : i == 12 ? 40 : 0;
}
__host__ __device__ constexpr int tw_offset(int n) {
  int off = 0;
  for (int i = 0; i < kNumFftSizes; ++i) {
    if (tw_size_at(i) == n) return off;
    off += tw_size_at(i);
  }
  return -1;
}
constexpr int kTwTotal = tw_offset(40) + 40;
__host__ __device__ constexpr bool fft_size_supported(int n) { return tw_offset(n) >= 0; }

// Each translation unit that launches FFT kernels owns its own copy of the
// constant tables and uploads them with upload_twiddles() (once per device).
static __constant__ double2 c_tw64[kTwTotal];
static __constant__ float2 c_tw32[kTwTotal];
// host copies (same values), used by host-side callers and by the upload
inline double2 h_tw64[kTwTotal];
inline float2 h_tw32[kTwTotal];

inline void fill_host_twiddles() {
  static bool done = false;
  if (done) return;
  const double two_pi = 6.283185307179586476925286766559;
  int off = 0;
  for (int s = 0; s < kNumFftSizes; ++s) {
    const int n = kFftSizes[s];
    for (int k = 0; k < n; ++k) {
      // exact values on the axes, cos/sin of the host math library elsewhere
      double c, sn;
      if ((4 * k) % n == 0) {
        const int q = (4 * k) / n;
        c = (q == 0) ? 1.0 : (q == 2) ? -1.0 : 0.0;
        sn = (q == 1) ? 1.0 : (q == 3) ? -1.0 : 0.0;
      } else {
        c = std::cos(two_pi * k / n);
        sn = std::sin(two_pi * k / n);
      }
      h_tw64[off + k] = make_double2(c, -sn);
      h_tw32[off + k] = make_float2((float)c, (float)-sn);
    }
    off += n;
  }
  done = true;
}

static inline cudaError_t upload_twiddles() {
  fill_host_twiddles();
  cudaError_t e = cudaMemcpyToSymbol(c_tw64, h_tw64, sizeof(h_tw64));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_tw32, h_tw32, sizeof(h_tw32));
}

template <typename T> struct TwTable;
template <> struct TwTable<double> {
  static __host__ __device__ __forceinline__ cpx<double> get(int i) {
#ifdef __CUDA_ARCH__
    double2 v = c_tw64[i];
#else
    double2 v = h_tw64[i];
#endif
    return {v.x, v.y};
  }
};
template <> struct TwTable<float> {
  static __host__ __device__ __forceinline__ cpx<float> get(int i) {
#ifdef __CUDA_ARCH__
    float2 v = c_tw32[i];
#else
    float2 v = h_tw32[i];
#endif
    return {v.x, v.y};
  }
};

// exp(DIR * 2 pi i e / N) for a table length NT that holds exp(-2 pi i k / NT)
template <typename T, int NT, int DIR> __host__ __device__ __forceinline__ cpx<T> twiddle(int e) {
  constexpr int off = tw_offset(NT);
  static_assert(off >= 0, "unsupported line length");
  cpx<T> w = TwTable<T>::get(off + (e % NT));
  return DIR < 0 ? w : cconj(w);
}

// v * exp(DIR * 2 pi i e / NT).  e is a compile-time constant once the callers' loops are
// unrolled; multiples of a quarter turn become exact swaps and sign changes (no multiply).
template <typename T, int NT, int DIR> __host__ __device__ __forceinline__ cpx<T> twiddle_mul(cpx<T> v, int e) {
  e %= NT;
  if ((4 * e) % NT == 0) {
    switch ((4 * e) / NT) {
      case 0: return v;
      case 1: return mul_i<DIR>(v);               // exp(DIR i pi / 2) = DIR i
      case 2: return {-v.x, -v.y};
      default: return mul_i<-DIR>(v);             // exp(DIR 3 i pi / 2) = -DIR i
    }
  }
  return cmul(v, twiddle<T, NT, DIR>(e));
}

// ---------------------------------------------------------------- radix kernels
template <typename T, int R, int DIR> struct Radix;

template <typename T, int DIR> struct Radix<T, 2, DIR> {
  static __host__ __device__ __forceinline__ void run(cpx<T> (&v)[2]) {
    cpx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename T, int DIR> struct Radix<T, 4, DIR> {
  static __host__ __device__ __forceinline__ void run(cpx<T> (&v)[4]) {
    cpx<T> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    cpx<T> s13 = cadd(v[1], v[3]), d13 = mul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

template <typename T, int DIR> struct Radix<T, 3, DIR> {
  static __host__ __device__ __forceinline__ void run(cpx<T> (&v)[3]) {
    const T h = T(0.5), s3 = T(0.86602540378443864676372317075294);  // sin(2 pi / 3)
    cpx<T> t = cadd(v[1], v[2]);
    cpx<T> d = csub(v[1], v[2]);
    cpx<T> m = {v[0].x - h * t.x, v[0].y - h * t.y};
    cpx<T> r = mul_i<DIR>(cscale(d, s3));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};

template <typename T, int DIR> struct Radix<T, 5, DIR> {
  static __host__ __device__ __forceinline__ void run(cpx<T> (&v)[5]) {
    const T c1 = T(0.30901699437494742410229341718282);   // cos(2 pi / 5)
    const T c2 = T(-0.80901699437494742410229341718282);  // cos(4 pi / 5)
    const T s1 = T(0.95105651629515357211643933337938);   // sin(2 pi / 5)
    const T s2 = T(0.58778525229247312916870595463907);   // sin(4 pi / 5)
    cpx<T> t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    cpx<T> t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    cpx<T> b1 = {v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y};
    cpx<T> b2 = {v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y};
    cpx<T> q1 = {s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y};
    cpx<T> q2 = {s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y};
    cpx<T> r1 = mul_i<DIR>(q1), r2 = mul_i<DIR>(q2);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(b1, r1);
    v[4] = csub(b1, r1);
    v[2] = cadd(b2, r2);
    v[3] = csub(b2, r2);
  }
};

__host__ __device__ constexpr int pick_radix(int n) {
  return (n % 4 == 0) ? 4 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : (n % 2 == 0) ? 2 : n;
}

// Coprime split N = N1 N2 for the prime-factor (Good-Thomas) algorithm, which needs no
// twiddle factors between its two passes: N1 = the power-of-two part of N, or for odd N
// the power-of-three part; 0 when N is a prime power (Cooley-Tukey then).
__host__ __device__ constexpr int pfa_n1(int n) {
  int p2 = 1, m = n;
  while (m % 2 == 0) { m /= 2; p2 *= 2; }
  if (p2 > 1 && p2 < n) return p2;
  int p3 = 1;
  m = n;
  while (m % 3 == 0) { m /= 3; p3 *= 3; }
  if (p3 > 1 && p3 < n) return p3;
  return 0;
}
// x with a x = 1 (mod m), m >= 2 and gcd(a, m) = 1
__host__ __device__ constexpr int inv_mod(int a, int m) {
  int x = 1;
  while ((a * x) % m != 1) ++x;
  return x;
}

// ---------------------------------------------------------------- line FFT
// In place on a[0..N-1].  NT is the length of the full line (for the twiddle table).
// Coprime N = N1 N2 (prime-factor algorithm): with n = (N2 n1 + N1 n2) mod N and
// k = (N2 a k1 + N1 b k2) mod N, a = N2^-1 mod N1, b = N1^-1 mod N2, the kernel factors as
// W_N^{nk} = W_N1^{n1 k1} W_N2^{n2 k2}: length-N1 transforms along n1, then length-N2
// transforms along n2, with no twiddle factors between them.
// Otherwise (Cooley-Tukey, decimation in time) N = R * M; n = M n1 + n2, k = k1 + R k2:
//   X[k1 + R k2] = sum_n2 W_M^{n2 k2} W_N^{n2 k1} sum_n1 x[M n1 + n2] W_R^{n1 k1}
template <typename T, int N, int DIR, int NT = N> struct LineFFT {
  static constexpr int P1 = pfa_n1(N);
  static constexpr int R = pick_radix(N);
  static constexpr int M = N / R;
  static __host__ __device__ __forceinline__ void run(cpx<T> (&a)[N]) {
    if constexpr (P1 > 0) {
      constexpr int N1 = P1, N2 = N / P1;
      constexpr int A = inv_mod(N2 % N1, N1), B = inv_mod(N1 % N2, N2);
      cpx<T> t[N];   // t[k1 N2 + n2]: after the length-N1 transforms
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) {
        cpx<T> v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = a[(N2 * n1 + N1 * n2) % N];
        LineFFT<T, N1, DIR, NT>::run(v);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) t[k1 * N2 + n2] = v[k1];
      }
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        cpx<T> u[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[n2] = t[k1 * N2 + n2];
        LineFFT<T, N2, DIR, NT>::run(u);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) a[(N2 * A * k1 + N1 * B * k2) % N] = u[k2];
      }
      return;
    } else {
      run_ct(a);
    }
  }
  static __host__ __device__ __forceinline__ void run_ct(cpx<T> (&a)[N]) {
    static_assert(R == 2 || R == 3 || R == 4 || R == 5, "line length must be 5-smooth");
#pragma unroll
    for (int n2 = 0; n2 < M; ++n2) {
      cpx<T> v[R];
#pragma unroll
      for (int n1 = 0; n1 < R; ++n1) v[n1] = a[M * n1 + n2];
      Radix<T, R, DIR>::run(v);
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) {
        // W_N^{n2 k1} = W_NT^{n2 k1 NT / N}
        if (n2 * k1 != 0) v[k1] = twiddle_mul<T, NT, DIR>(v[k1], (n2 * k1 * (NT / N)) % NT);
        a[M * k1 + n2] = v[k1];
      }
    }
    if constexpr (M > 1) {
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) {
        cpx<T>(&sub)[M] = *reinterpret_cast<cpx<T>(*)[M]>(&a[M * k1]);
        LineFFT<T, M, DIR, NT>::run(sub);
      }
      // a[M k1 + k2] holds X[k1 + R k2]: transpose to natural order
      cpx<T> tmp[N];
#pragma unroll
      for (int i = 0; i < N; ++i) tmp[i] = a[i];
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < M; ++k2) a[k1 + R * k2] = tmp[M * k1 + k2];
    }
  }
};

// index helpers: frequency m (|m| < N/2) <-> storage slot
__host__ __device__ __forceinline__ int wrap_idx(int m, int n) { return m < 0 ? m + n : m; }

}  // namespace ltmp2
