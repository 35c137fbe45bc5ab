// Host check of the register line transforms of csrc/fft_line.cuh (the same templates the
// kernels run): LineFFT<T, N, DIR> against the direct DFT sum in long double, and LineFFTZ (the
// first butterfly stage pruned for the known-zero inputs outside the window |m| <= N/4)
// against LineFFT on inputs that are zero there.  Prints one line per grid size:
//   N <n> <f64 inverse> <f64 forward> <f32 inverse> <f32 forward> <zf64 inv> <zf64 fwd> <zf32 inv> <zf32 fwd>
// (relative max-norm errors).
#include <cmath>
#include <complex>
#include <cstdio>

#include "../../paper_2412_01695_gb300/csrc/fft_line.cuh"

using namespace pwk;
using cld = std::complex<long double>;

template <int N>
struct OutsideWindow {
  __host__ __device__ static constexpr bool zero(int i) { return !(i <= N / 4 || i >= N - N / 4); }
};

// deterministic test input (no random generator needed)
static void input(int n, double& re, double& im) {
  re = std::sin(1.3 * n + 0.2);
  im = std::cos(0.7 * n * n + 0.1);
}

template <typename T, int N, int DIR>
double versus_direct_sum() {
  using V = c2_t<T>;
  V x[N];
  cld in[N];
  for (int n = 0; n < N; ++n) {
    double a, b;
    input(n, a, b);
    x[n] = V{(T)a, (T)b};
    in[n] = cld((long double)(T)a, (long double)(T)b);
  }
  LineFFT<T, N, DIR>::run(x);
  const long double two_pi = 6.283185307179586476925286766559L;
  double err = 0, nrm = 0;
  for (int k = 0; k < N; ++k) {
    cld s = 0;
    for (int n = 0; n < N; ++n) {
      const long double ang = DIR * two_pi * (long double)((n * k) % N) / N;
      s += in[n] * cld(std::cos(ang), std::sin(ang));
    }
    const V o = x[fft_out_slot(N, k)];
    err = std::fmax(err, (double)std::abs(cld(o.x, o.y) - s));
    nrm = std::fmax(nrm, (double)std::abs(s));
  }
  return err / nrm;
}

template <typename T, int N, int DIR>
double pruned_versus_full() {
  using V = c2_t<T>;
  V x[N], y[N];
  for (int n = 0; n < N; ++n) {
    double a, b;
    input(n, a, b);
    if (OutsideWindow<N>::zero(n)) a = b = 0;
    x[n] = y[n] = V{(T)a, (T)b};
  }
  LineFFT<T, N, DIR>::run(x);
  LineFFTZ<T, N, DIR, OutsideWindow<N>>::run(y);
  double err = 0, nrm = 0;
  for (int k = 0; k < N; ++k) {
    const V a = x[fft_out_slot(N, k)], b = y[fft_out_slot(N, k)];
    err = std::fmax(err, std::hypot((double)a.x - (double)b.x, (double)a.y - (double)b.y));
    nrm = std::fmax(nrm, std::hypot((double)a.x, (double)a.y));
  }
  return err / nrm;
}

template <int N>
void line() {
  std::printf("N %d %.3e %.3e %.3e %.3e %.3e %.3e %.3e %.3e\n", N, versus_direct_sum<double, N, 1>(),
              versus_direct_sum<double, N, -1>(), versus_direct_sum<float, N, 1>(), versus_direct_sum<float, N, -1>(),
              pruned_versus_full<double, N, 1>(), pruned_versus_full<double, N, -1>(),
              pruned_versus_full<float, N, 1>(), pruned_versus_full<float, N, -1>());
}

int main() {
  // every grid size the library instantiates
  line<12>(); line<15>(); line<16>(); line<18>(); line<20>(); line<24>(); line<25>();
  line<27>(); line<30>(); line<32>(); line<36>(); line<40>(); line<45>(); line<48>();
  return 0;
}
