// Register-resident complex DFT of one line of compile-time length N (N = 2^a 3^b 5^c).
//
// Used for the one-dimensional passes of the 3D transform of paper Sec. 4
// (Eqs. zfft, yfft, xfft and fwFFT): every line is owned by one thread and lives in
// registers.  The factorisation is a two-level Cooley-Tukey split N = R * M applied
// recursively (R = 4, 2, 3 or 5), with explicit radix-2/3/4/5 butterflies.  Every index
// is a compile-time constant after unrolling, and every twiddle factor is a compile-time
// constant computed below from its Taylor series (no table, no library call).
//
// Sign convention: DIR = +1 computes X_k = sum_n x_n e^{+2 pi i n k / N} (the inverse
// transform of the paper, no normalisation); DIR = -1 computes the forward sum with
// e^{-2 pi i n k / N} (the 1/N_r factor is applied by the caller).
//
// Output order: the transform is computed in place; X_k is left in register slot
// fft_out_slot<N>(k).  Inputs are in natural order.
#pragma once
#include <cuda_runtime.h>

#include <utility>

// host-and-device, always inlined: lets the CPU self-test exercise the same templates
#define PWK_HD __host__ __device__ __forceinline__

namespace pwk {

// ------------------------------------------------------------------ compile-time trig
constexpr double kPi = 3.14159265358979323846264338327950288;

__host__ __device__ constexpr double taylor_sin(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int n = 1; n < 14; ++n) {
    term *= -x2 / double((2 * n) * (2 * n + 1));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int n = 1; n < 14; ++n) {
    term *= -x2 / double((2 * n - 1) * (2 * n));
    sum += term;
  }
  return sum;
}
// cos(2 pi e / n) with exact rational reduction to |angle| <= pi/4.
__host__ __device__ constexpr double cos2pi(long e, long n) {
  e %= n;
  if (e < 0) e += n;
  if (2 * e > n) e = n - e;                  // cos(2pi f) = cos(2pi (1-f))
  double sgn = 1.0;
  if (4 * e > n) {                           // cos(2pi f) = -cos(2pi (1/2 - f))
    sgn = -1.0;
    long ne = n - 2 * e, nn = 2 * n;         // (1/2 - f) = (n - 2e) / 2n
    e = ne;
    n = nn;
  }
  if (8 * e > n)                             // cos(2pi f) = sin(2pi (1/4 - f))
    return sgn * taylor_sin(2.0 * kPi * double(n - 4 * e) / double(4 * n));
  return sgn * taylor_cos(2.0 * kPi * double(e) / double(n));
}
// sin(2 pi e / n) = cos(2 pi (e/n - 1/4)) = cos2pi(4e - n, 4n)
__host__ __device__ constexpr double sin2pi(long e, long n) { return cos2pi(4 * e - n, 4 * n); }

// ------------------------------------------------------------------ complex helpers
template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };
template <typename T> using c2_t = typename C2<T>::type;

template <typename V> PWK_HD V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> PWK_HD V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V, typename T> PWK_HD V cscale(V a, T s) { return V{a.x * s, a.y * s}; }
// a * (i * s), s = +-1
template <typename V> PWK_HD V cmul_i(V a, int s) {
  return s > 0 ? V{-a.y, a.x} : V{a.y, -a.x};
}

// ------------------------------------------------------------------ compile-time loops
// static_for<N>(f) calls f(std::integral_constant<int, 0>) ... f(<N-1>): the index is a
// constant expression, so register arrays indexed by it (or by constexpr functions of it)
// never fall back to local memory.
template <typename F, int... I>
PWK_HD void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
PWK_HD void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}
// PWK_SFOR(N, j, body): body repeated for the constant j = 0 .. N-1
#define PWK_SFOR(NN, j, ...) \
  ::pwk::static_for<NN>([&](auto j##_c) { constexpr int j = decltype(j##_c)::value; __VA_ARGS__; })

// ------------------------------------------------------------------ factorisation
__host__ __device__ constexpr int first_radix(int n) {
  return (n % 4 == 0 && n != 8) ? 4 : (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : (n % 5 == 0) ? 5 : n;
}
// register slot holding X_k after an in-place transform of length n
__host__ __device__ constexpr int fft_out_slot(int n, int k) {
  return (n == 2 || n == 3 || n == 4 || n == 5)
             ? k
             : (n / first_radix(n)) * (k % first_radix(n)) +
                   fft_out_slot(n / first_radix(n), k / first_radix(n));
}

// X_k of a length-n transform, k a compile-time constant
template <int n, int k>
struct OutSlot {
  static constexpr int value = fft_out_slot(n, k);
};

// multiply v by W_N^E = e^{DIR 2 pi i E / N}; E, N compile time
template <typename T, int N, int E, int DIR>
PWK_HD c2_t<T> twiddle(c2_t<T> v) {
  constexpr int e = ((E % N) + N) % N;
  if constexpr (e == 0) {
    return v;
  } else if constexpr (4 * e == N) {
    return cmul_i(v, DIR);
  } else if constexpr (2 * e == N) {
    return c2_t<T>{-v.x, -v.y};
  } else if constexpr (4 * e == 3 * N) {
    return cmul_i(v, -DIR);
  } else {
    constexpr T c = T(cos2pi(e, N));
    constexpr T s = T(DIR * sin2pi(e, N));
    return c2_t<T>{v.x * c - v.y * s, v.x * s + v.y * c};
  }
}

// ------------------------------------------------------------------ butterflies
template <typename T, int R, int DIR> struct Butterfly;

template <typename T, int DIR> struct Butterfly<T, 2, DIR> {
  using V = c2_t<T>;
  template <int S>
  static PWK_HD void run(V* x) {
    V a = x[0], b = x[S];
    x[0] = cadd(a, b);
    x[S] = csub(a, b);
  }
};

template <typename T, int DIR> struct Butterfly<T, 4, DIR> {
  using V = c2_t<T>;
  template <int S>
  static PWK_HD void run(V* x) {
    V a = x[0], b = x[S], c = x[2 * S], d = x[3 * S];
    V ac = cadd(a, c), amc = csub(a, c), bd = cadd(b, d), bmd = cmul_i(csub(b, d), DIR);
    x[0] = cadd(ac, bd);
    x[2 * S] = csub(ac, bd);
    x[S] = cadd(amc, bmd);
    x[3 * S] = csub(amc, bmd);
  }
};

template <typename T, int DIR> struct Butterfly<T, 3, DIR> {
  using V = c2_t<T>;
  template <int S>
  static PWK_HD void run(V* x) {
    constexpr T h = T(0.5);
    constexpr T s3 = T(DIR * 0.86602540378443864676372317075293618);  // sin(2pi/3)
    V a = x[0], b = x[S], c = x[2 * S];
    V t = cadd(b, c);
    V m = V{a.x - h * t.x, a.y - h * t.y};
    V d = csub(b, c);
    V r = V{-s3 * d.y, s3 * d.x};  // i * s3 * (b - c)
    x[0] = cadd(a, t);
    x[S] = cadd(m, r);
    x[2 * S] = csub(m, r);
  }
};

template <typename T, int DIR> struct Butterfly<T, 5, DIR> {
  using V = c2_t<T>;
  template <int S>
  static PWK_HD void run(V* x) {
    constexpr T c1 = T(cos2pi(1, 5)), c2 = T(cos2pi(2, 5));
    constexpr T s1 = T(DIR * sin2pi(1, 5)), s2 = T(DIR * sin2pi(2, 5));
    V a = x[0], b = x[S], c = x[2 * S], d = x[3 * S], e = x[4 * S];
    V t1 = cadd(b, e), t2 = cadd(c, d), t3 = csub(b, e), t4 = csub(c, d);
    V p1 = V{a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y};
    V p2 = V{a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y};
    // q1 = i (s1 t3 + s2 t4), q2 = i (s2 t3 - s1 t4)
    V u1 = V{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y};
    V u2 = V{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y};
    V q1 = V{-u1.y, u1.x}, q2 = V{-u2.y, u2.x};
    x[0] = cadd(a, cadd(t1, t2));
    x[S] = cadd(p1, q1);
    x[4 * S] = csub(p1, q1);
    x[2 * S] = cadd(p2, q2);
    x[3 * S] = csub(p2, q2);
  }
};

// ------------------------------------------------------------------ recursive line FFT
// In-place transform of the N values x[0], x[1], ..., x[N-1] (contiguous register slots).
template <typename T, int N, int DIR> struct LineFFT {
  using V = c2_t<T>;
  static constexpr int R = first_radix(N);
  static constexpr int M = N / R;
  static PWK_HD void run(V* x) {
    if constexpr (M == 1) {
      Butterfly<T, R, DIR>::template run<1>(x);
    } else {
      // step A: for each n2 < M, a length-R DFT over n1 of x[M n1 + n2]; y[n2][k1] -> slot M k1 + n2
      static_for<M>([&](auto n2) { Butterfly<T, R, DIR>::template run<M>(x + decltype(n2)::value); });
      // step B: twiddle y[n2][k1] *= W_N^{n2 k1}
      apply_twiddles(x, std::make_integer_sequence<int, N>{});
      // step C: for each k1 < R, a length-M DFT of the contiguous block x[M k1 .. M k1 + M)
      static_for<R>([&](auto k1) { LineFFT<T, M, DIR>::run(x + M * decltype(k1)::value); });
    }
  }
  template <int... I>
  static PWK_HD void apply_twiddles(V* x, std::integer_sequence<int, I...>) {
    // slot I = M k1 + n2 carries exponent n2 * k1
    ((x[I] = twiddle<T, N, (I % M) * (I / M), DIR>(x[I])), ...);
  }
};

// ------------------------------------------------------------------ known-zero inputs
// A radix-R butterfly whose inputs n with bit n of ZM set are known to be zero (compile-time
// mask; the zero inputs must hold zeros).  IEEE arithmetic forbids dropping "x + 0" (the
// sign of a zero), so the compiler cannot prune these operations itself: when at most half
// the inputs are present the butterfly becomes the direct sum over them, with trivial
// twiddles (+-1, +-i) free; otherwise the full butterfly runs on the zeros.
__host__ __device__ constexpr int popcount_bits(unsigned m) { return m == 0u ? 0 : int(m & 1u) + popcount_bits(m >> 1); }

template <typename T, int R, int DIR, unsigned ZM>
struct ButterflyZ {
  using V = c2_t<T>;
  template <int S>
  static PWK_HD void run(V* x) {
    if constexpr (2 * (R - popcount_bits(ZM)) > R) {
      Butterfly<T, R, DIR>::template run<S>(x);   // more than half the inputs present
    } else if constexpr (ZM == (1u << R) - 1u) {
      static_for<R>([&](auto kc) { x[decltype(kc)::value * S] = V{T(0), T(0)}; });
    } else {
      V in[R];
      static_for<R>([&](auto nc) {
        constexpr int n = decltype(nc)::value;
        if constexpr (!((ZM >> n) & 1u)) in[n] = x[n * S];
      });
      static_for<R>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        V acc{T(0), T(0)};
        bool first = true;
        static_for<R>([&](auto nc) {
          constexpr int n = decltype(nc)::value;
          if constexpr (!((ZM >> n) & 1u)) {
            const V t = twiddle<T, R, n * k, DIR>(in[n]);
            acc = first ? t : cadd(acc, t);
            first = false;
          }
        });
        x[k * S] = acc;
      });
    }
  }
};

// The line transform of LineFFT (same factorisation, same output slots) when the inputs x[i]
// with Z::zero(i) true are known to be zero: only the first butterfly stage sees them, and
// it is pruned; the twiddles and the inner transforms are those of LineFFT.
template <typename T, int N, int DIR, typename Z>
struct LineFFTZ {
  using V = c2_t<T>;
  static constexpr int R = first_radix(N);
  static constexpr int M = N / R;
  template <int n2>
  __host__ __device__ static constexpr unsigned mask() {
    unsigned m = 0;
    for (int n1 = 0; n1 < R; ++n1)
      if (Z::zero(M * n1 + n2)) m |= 1u << n1;
    return m;
  }
  static PWK_HD void run(V* x) {
    if constexpr (M == 1) {
      ButterflyZ<T, R, DIR, mask<0>()>::template run<1>(x);
    } else {
      static_for<M>([&](auto n2) {
        constexpr int j = decltype(n2)::value;
        ButterflyZ<T, R, DIR, mask<j>()>::template run<M>(x + j);
      });
      LineFFT<T, N, DIR>::apply_twiddles(x, std::make_integer_sequence<int, N>{});
      static_for<R>([&](auto k1) { LineFFT<T, M, DIR>::run(x + M * decltype(k1)::value); });
    }
  }
};

}  // namespace pwk
