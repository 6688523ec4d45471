// Discrete Fourier transforms of compile-time length held in registers (float2 arrays),
// mixed radix 2, 3, 4, 5, 7, unnormalised:
//   forward  X[k] = sum_n x[n] exp(-2 pi i n k / N),   inverse  with exp(+2 pi i n k / N).
// Composite lengths split N = P M by decimation in time (P sub-sequences x[P m + r] of length
// M, twiddles exp(-+2 pi i r k / N), then P-point transforms across r); primes 3, 5, 7 use
// the symmetric form that pairs x[j] with x[N - j]. The roots are compile-time constants:
// cos and sin of 2 pi j / N evaluated by Taylor series in double precision and rounded to
// float when the table is built (constexpr), so no trigonometric call runs on the device.
// Usable from host code as well (the same template compiles for the CPU), which is how the
// transforms are checked against a reference FFT without a GPU.
#pragma once

#include <vector_types.h>

#ifdef __CUDACC__
#define DFT_HD __host__ __device__ __forceinline__
#define DFT_CX __host__ __device__ constexpr
#else
#define DFT_HD inline
#define DFT_CX constexpr
#endif

namespace lps {
namespace dftr {

constexpr double kPi = 3.14159265358979323846264338327950288;

// sin and cos on [-pi/4, pi/4] by their Taylor series (terms to x^27: error below 1e-19).
DFT_CX double sin_small(double x) {
  double t = x, s = x;
  for (int k = 1; k < 14; ++k) {
    t *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    s += t;
  }
  return s;
}
DFT_CX double cos_small(double x) {
  double t = 1.0, s = 1.0;
  for (int k = 1; k < 14; ++k) {
    t *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    s += t;
  }
  return s;
}
// cos and sin of 2 pi j / n for integers 0 <= j < n, reduced by octant symmetry.
DFT_CX void root_cs(int j, int n, double* c, double* s) {
  // angle = 2 pi j / n = (pi / 4) * q with q = 8 j / n in [0, 8)
  const double q = 8.0 * j / n;
  int oct = (int)q;
  if (oct > 7) oct = 7;
  const double r = (q - oct) * (kPi / 4.0);   // in [0, pi/4)
  double cc = 0, ss = 0;
  // rotate by octant: angle = oct * pi/4 + r
  const double c0 = cos_small(r), s0 = sin_small(r);
  const double h = 0.70710678118654752440084436210484903928;   // cos(pi/4) = sin(pi/4)
  switch (oct) {
    case 0: cc = c0; ss = s0; break;
    case 1: cc = h * (c0 - s0); ss = h * (c0 + s0); break;
    case 2: cc = -s0; ss = c0; break;
    case 3: cc = -h * (c0 + s0); ss = h * (c0 - s0); break;
    case 4: cc = -c0; ss = -s0; break;
    case 5: cc = -h * (c0 - s0); ss = -h * (c0 + s0); break;
    case 6: cc = s0; ss = -c0; break;
    default: cc = h * (c0 + s0); ss = -h * (c0 - s0); break;
  }
  *c = cc;
  *s = ss;
}

template <int N>
struct Roots {
  float c[N];
  float s[N];
  DFT_CX Roots() : c(), s() {
    for (int j = 0; j < N; ++j) {
      double cc = 0, ss = 0;
      // exact values where the root lies on an axis
      if ((4 * j) % N == 0) {
        const int a = (4 * j) / N;
        cc = a == 0 ? 1.0 : (a == 2 ? -1.0 : 0.0);
        ss = a == 1 ? 1.0 : (a == 3 ? -1.0 : 0.0);
      } else {
        root_cs(j, N, &cc, &ss);
      }
      c[j] = (float)cc;
      s[j] = (float)ss;
    }
  }
};

DFT_HD float2 f2(float x, float y) {
  float2 r;
  r.x = x;
  r.y = y;
  return r;
}
DFT_HD float2 add(float2 a, float2 b) { return f2(a.x + b.x, a.y + b.y); }
DFT_HD float2 sub(float2 a, float2 b) { return f2(a.x - b.x, a.y - b.y); }
// a * exp(-+2 pi i j / N) for the root j of length N (forward: minus sign)
template <int N, bool INV>
DFT_HD float2 rot(float2 a, int j) {
  constexpr Roots<N> R{};
  if (j == 0) return a;
  if (4 * j == N) return INV ? f2(-a.y, a.x) : f2(a.y, -a.x);   // * (+-i)
  if (2 * j == N) return f2(-a.x, -a.y);
  if (4 * j == 3 * N) return INV ? f2(a.y, -a.x) : f2(-a.y, a.x);
  const float c = R.c[j], s = INV ? R.s[j] : -R.s[j];
  return f2(a.x * c - a.y * s, a.x * s + a.y * c);
}

template <int N>
DFT_CX int radix_of() {
  return (N % 4 == 0 && N > 4) ? 4 : (N % 2 == 0 && N > 2) ? 2 : (N % 3 == 0 && N > 3) ? 3
                                                            : (N % 5 == 0 && N > 5) ? 5 : (N % 7 == 0 && N > 7) ? 7 : 0;
}

template <int N, bool INV>
DFT_HD void dft(float2 (&v)[N]);

// Odd prime N (3, 5, 7): pairs a_j = x_j + x_{N-j}, b_j = x_j - x_{N-j};
// X[k] = x_0 + sum_j a_j cos(2 pi j k / N) -+ i sum_j b_j sin(2 pi j k / N), X[N-k] with +-.
template <int N, bool INV>
DFT_HD void dft_prime(float2 (&v)[N]) {
  constexpr Roots<N> R{};
  constexpr int H = (N - 1) / 2;
  float2 a[H + 1], b[H + 1];
#pragma unroll
  for (int j = 1; j <= H; ++j) {
    a[j] = add(v[j], v[N - j]);
    b[j] = sub(v[j], v[N - j]);
  }
  float2 out[N];
  float2 s0 = v[0];
#pragma unroll
  for (int j = 1; j <= H; ++j) s0 = add(s0, a[j]);
  out[0] = s0;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    float2 t = v[0], u = f2(0.f, 0.f);
#pragma unroll
    for (int j = 1; j <= H; ++j) {
      const int q = (j * k) % N;
      t.x += a[j].x * R.c[q];
      t.y += a[j].y * R.c[q];
      u.x += b[j].x * R.s[q];
      u.y += b[j].y * R.s[q];
    }
    // forward: X[k] = t - i u, X[N-k] = t + i u; inverse swaps them
    const float2 mi = f2(t.x + u.y, t.y - u.x);   // t - i u
    const float2 pi = f2(t.x - u.y, t.y + u.x);   // t + i u
    out[k] = INV ? pi : mi;
    out[N - k] = INV ? mi : pi;
  }
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = out[k];
}

template <int N, bool INV>
DFT_HD void dft(float2 (&v)[N]) {
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = add(a, b);
    v[1] = sub(a, b);
  } else if constexpr (N == 4) {
    const float2 s02 = add(v[0], v[2]), d02 = sub(v[0], v[2]);
    const float2 s13 = add(v[1], v[3]), d13 = sub(v[1], v[3]);
    // forward: X1 = d02 - i d13, X3 = d02 + i d13
    const float2 mi = f2(d02.x + d13.y, d02.y - d13.x);
    const float2 pi = f2(d02.x - d13.y, d02.y + d13.x);
    v[0] = add(s02, s13);
    v[2] = sub(s02, s13);
    v[1] = INV ? pi : mi;
    v[3] = INV ? mi : pi;
  } else if constexpr (N == 3 || N == 5 || N == 7) {
    dft_prime<N, INV>(v);
  } else {
    constexpr int P = radix_of<N>();
    static_assert(P > 0, "length must factor into 2, 3, 5, 7");
    constexpr int M = N / P;
    float2 s[P][M];
#pragma unroll
    for (int r = 0; r < P; ++r)
#pragma unroll
      for (int m = 0; m < M; ++m) s[r][m] = v[P * m + r];
#pragma unroll
    for (int r = 0; r < P; ++r) dft<M, INV>(s[r]);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      float2 t[P];
#pragma unroll
      for (int r = 0; r < P; ++r) t[r] = rot<N, INV>(s[r][k], r * k);
      dft<P, INV>(t);
#pragma unroll
      for (int q = 0; q < P; ++q) v[k + M * q] = t[q];
    }
  }
}

}  // namespace dftr
}  // namespace lps
