// Line FFTs of compile-time length N for the plane-wave transforms.
//
// A line of length N = N1 * N2 (N1 a multiple of N2) is owned by N2 threads.  Writing
// i = t + N2 m and k = k1 + N1 k2 (t, k2 < N2; m, k1 < N1),
//
//   X[k1 + N1 k2] = sum_t w_N2^{t k2} w_N^{t k1} sum_m x[t + N2 m] w_N1^{m k1},
//
// so thread t first forms the N1-point DFT of its strided values in registers and applies
// the twiddles w_N^{t k1} (step 1), the values go through shared memory once, and thread t
// then forms the N2-point DFTs of the columns k1 = t + N2 j (j < N1 / N2), again in
// registers (step 2).  The register DFTs split coprime lengths by the prime-factor
// (Good-Thomas) index map, which needs no twiddles, and the rest by mixed-radix
// Cooley-Tukey, with every index known at compile time.  Twiddles come from a per-line table tw[e] = e^{-2 pi i e / N} in
// shared memory; all threads of a warp read the same entry (broadcast).
//
// Convention: forward X_k = sum_j x_j e^{-2 pi i k j / N}, inverse with +i; neither is
// normalised.
//
// Thread layout: line index fastest.  With L lines in flight, thread i works on line
// i % L at slot i / L, so the 16 (FP32) or 8 (FP64) threads of one shared-memory
// wavefront touch 16 or 8 distinct lines at the same element index; line pitches are odd
// in elements, which puts them in distinct banks.
#pragma once
#include "common.cuh"

namespace eacg {

// Plan variant 0 exists for every supported N; variant 1 (a second split N1 x N2) where one
// is worth trying.  The autotuner picks between them per system and precision.
template <int N, int PV = 0>
struct LinePlan;
#define EACG_LINE_PLAN(N_, PV_, A_, B_)        \
  template <>                                  \
  struct LinePlan<N_, PV_> {                   \
    static constexpr int N1 = A_, N2 = B_;     \
  };
EACG_LINE_PLAN(8, 0, 4, 2)
EACG_LINE_PLAN(12, 0, 6, 2)
EACG_LINE_PLAN(16, 0, 4, 4)
EACG_LINE_PLAN(20, 0, 10, 2)
EACG_LINE_PLAN(24, 0, 12, 2)
EACG_LINE_PLAN(32, 0, 8, 4)
EACG_LINE_PLAN(36, 0, 12, 3)
EACG_LINE_PLAN(40, 0, 20, 2)
EACG_LINE_PLAN(48, 0, 12, 4)
EACG_LINE_PLAN(64, 0, 16, 4)
EACG_LINE_PLAN(72, 0, 12, 6)
EACG_LINE_PLAN(80, 0, 20, 4)
EACG_LINE_PLAN(96, 0, 24, 4)
EACG_LINE_PLAN(128, 0, 16, 8)
EACG_LINE_PLAN(16, 1, 8, 2)
EACG_LINE_PLAN(32, 1, 16, 2)
EACG_LINE_PLAN(36, 1, 6, 6)
EACG_LINE_PLAN(48, 1, 24, 2)
EACG_LINE_PLAN(64, 1, 8, 8)
EACG_LINE_PLAN(72, 1, 24, 3)
#undef EACG_LINE_PLAN

// The supported line lengths (every N with a LinePlan), for host-side checks and dispatch,
// and those with a second plan variant.
#define EACG_FOR_EACH_N(X) X(8) X(12) X(16) X(20) X(24) X(32) X(36) X(40) X(48) X(64) X(72) X(80) X(96) X(128)
#define EACG_FOR_EACH_N_PLAN1(X) X(16) X(32) X(36) X(48) X(64) X(72)

template <int R, bool INV, typename V>
__device__ __forceinline__ void dft_small(V* v) {
  using T = decltype(v[0].x);
  if constexpr (R == 2) {
    V a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else if constexpr (R == 3) {
    constexpr T h = T(0.86602540378443864676372317075293618);  // sin(2 pi / 3)
    V t1 = v[1] + v[2];
    V t2 = v[0] - cscale(t1, T(0.5));
    V d = mul_mi<INV>(cscale(v[1] - v[2], h));
    v[0] = v[0] + t1;
    v[1] = t2 + d;
    v[2] = t2 - d;
  } else if constexpr (R == 4) {
    V t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3];
    V t3 = mul_mi<INV>(v[1] - v[3]);
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    v[1] = t1 + t3;
    v[3] = t1 - t3;
  } else if constexpr (R == 5) {
    constexpr T c1 = T(0.30901699437494742410229341718281906);   // cos(2 pi / 5)
    constexpr T c2 = T(-0.80901699437494742410229341718281906);  // cos(4 pi / 5)
    constexpr T s1 = T(0.95105651629515357211643933337938214);   // sin(2 pi / 5)
    constexpr T s2 = T(0.58778525229247312916870595463907277);   // sin(4 pi / 5)
    V t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
    V a1 = v[0] + cscale(t1, c1) + cscale(t2, c2);
    V a2 = v[0] + cscale(t1, c2) + cscale(t2, c1);
    V b1 = mul_mi<INV>(cscale(t3, s1) + cscale(t4, s2));
    V b2 = mul_mi<INV>(cscale(t3, s2) - cscale(t4, s1));
    v[0] = v[0] + t1 + t2;
    v[1] = a1 + b1;
    v[4] = a1 - b1;
    v[2] = a2 + b2;
    v[3] = a2 - b2;
  }
}

// x * w_N^e (conjugated for the inverse), e in [0, N) known at compile time or uniform.
template <int N, bool INV, typename V>
__device__ __forceinline__ V twiddle(V x, int e, const V* tw) {
  V w = tw[e];
  if (INV) w.y = -w.y;
  return cmul(x, w);
}

// First factor R of a register DFT of length M = R Q: a base radix coprime to Q when one
// exists (prime-factor split, no twiddles), else 4 or 2 (Cooley-Tukey split).
template <int A, int B>
struct Gcd {
  static constexpr int value = Gcd<B, A % B>::value;
};
template <int A>
struct Gcd<A, 0> {
  static constexpr int value = A;
};
template <int M>
struct FirstRadix {
  static constexpr int R = (M % 4 == 0 && Gcd<4, M / 4>::value == 1)   ? 4
                           : (M % 3 == 0 && Gcd<3, M / 3>::value == 1) ? 3
                           : (M % 5 == 0 && Gcd<5, M / 5>::value == 1) ? 5
                           : (M % 4 == 0)                               ? 4
                           : (M % 2 == 0)                               ? 2
                           : (M % 3 == 0)                               ? 3
                                                                        : 5;
};
// X^{-1} mod Mod for gcd(X, Mod) = 1 (Mod <= 8 here)
template <int X, int Mod, int T = 1>
struct ModInv {
  static constexpr int value = ((X % Mod) * T) % Mod == 1 % Mod ? T : ModInv<X, Mod, T + 1>::value;
};
template <int X, int Mod>
struct ModInv<X, Mod, 9> {
  static constexpr int value = 0;
};

// In-register DFT of length M (M divides N) on a[0..M), natural order in and out.
// Coprime M = R Q (prime-factor algorithm): with n = (Q r + R q) mod M and
// k = (Q (Q^-1 mod R) k_r + R (R^-1 mod Q) k_q) mod M the DFT is an R x Q two-dimensional DFT
// without twiddles.  Otherwise M = R Q with m = r + R q, k = u + Q s (Cooley-Tukey):
// A[u + Q s] = sum_r w_R^{r s} w_M^{r u} (DFT_Q a[r + R .])[u].
template <int M, int N, bool INV, typename V>
__device__ __forceinline__ void reg_dft(V* a, const V* tw) {
  if constexpr (M == 2 || M == 3 || M == 4 || M == 5) {
    dft_small<M, INV>(a);
  } else if constexpr (M > 1) {
    constexpr int R = FirstRadix<M>::R, Q = M / R;
    if constexpr (Gcd<R, Q>::value == 1) {
      constexpr int QI = ModInv<Q, R>::value, RI = ModInv<R, Q>::value;
      V c[R][Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        V t[R];
#pragma unroll
        for (int r = 0; r < R; ++r) t[r] = a[(Q * r + R * q) % M];
        dft_small<R, INV>(t);
#pragma unroll
        for (int r = 0; r < R; ++r) c[r][q] = t[r];
      }
#pragma unroll
      for (int kr = 0; kr < R; ++kr) reg_dft<Q, N, INV>(c[kr], tw);
#pragma unroll
      for (int kr = 0; kr < R; ++kr)
#pragma unroll
        for (int kq = 0; kq < Q; ++kq) a[(Q * QI * kr + R * RI * kq) % M] = c[kr][kq];
    } else {
      V c[R][Q];
#pragma unroll
      for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int q = 0; q < Q; ++q) c[r][q] = a[r + R * q];
        reg_dft<Q, N, INV>(c[r], tw);
#pragma unroll
        for (int u = 1; u < Q; ++u) {
          const int e = (r * u) % M;
          if (e == 0) continue;
          if (4 * e == M) {
            c[r][u] = mul_mi<INV>(c[r][u]);
          } else if (2 * e == M) {
            c[r][u].x = -c[r][u].x;
            c[r][u].y = -c[r][u].y;
          } else if (4 * e == 3 * M) {
            c[r][u] = mul_mi<!INV>(c[r][u]);
          } else {
            c[r][u] = twiddle<N, INV>(c[r][u], e * (N / M), tw);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < Q; ++u) {
        V d[R];
#pragma unroll
        for (int r = 0; r < R; ++r) d[r] = c[r][u];
        dft_small<R, INV>(d);
#pragma unroll
        for (int s = 0; s < R; ++s) a[u + Q * s] = d[s];
      }
    }
  }
}

// Step 1 of slot t: a[m] = x[t + N2 m] in; a[k1] = w_N^{t k1} sum_m x[t + N2 m] w_N1^{m k1} out.
template <int N, int PV, bool INV, typename V>
__device__ __forceinline__ void line_step1(V* a, int t, const V* tw) {
  constexpr int N1 = LinePlan<N, PV>::N1;
  reg_dft<N1, N, INV>(a, tw);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) a[k1] = twiddle<N, INV>(a[k1], t * k1, tw);  // t k1 < N
}

// Step 2 of slot t: a[j N2 + tt] = step-1 value of slot tt at k1 = t + N2 j in;
// a[j N2 + k2] = X[(t + N2 j) + N1 k2] out.
template <int N, int PV, bool INV, typename V>
__device__ __forceinline__ void line_step2(V* a, const V* tw) {
  constexpr int N1 = LinePlan<N, PV>::N1, N2 = LinePlan<N, PV>::N2;
#pragma unroll
  for (int j = 0; j < N1 / N2; ++j) reg_dft<N2, N, INV>(a + j * N2, tw);
}

// One transform phase over nlines lines (nlines <= lines in flight = blockDim.x / N2).
// Step-1 inputs come from load(l, i); step-1 outputs go to *scratch(l, position); step-2
// outputs X[o] go to store(l, o, X[o], q), q < N1 being the output's ordinal within the
// thread (the same for every call).  The CTA synchronises between the steps and after the
// phase, and with MIDSYNC also between the step-2 loads and the stores (needed when the
// scratch slots of a line are the places its outputs are stored to).  Every thread must
// call it.
template <int N, int PV, bool INV, bool MIDSYNC, typename V, typename Scratch, typename Load, typename Store>
__device__ __forceinline__ void fft_phase(int nlines, const V* tw, const Scratch& scratch, const Load& load,
                                          const Store& store) {
  constexpr int N1 = LinePlan<N, PV>::N1, N2 = LinePlan<N, PV>::N2;
  const int L = blockDim.x / N2;
  const int l = threadIdx.x % L, t = threadIdx.x / L;
  const bool act = t < N2 && l < nlines;
  V a[N1];
  if (act) {
#pragma unroll
    for (int m = 0; m < N1; ++m) a[m] = load(l, t + N2 * m);
    line_step1<N, PV, INV>(a, t, tw);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) *scratch(l, t + N2 * k1) = a[k1];
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int j = 0; j < N1 / N2; ++j)
#pragma unroll
      for (int tt = 0; tt < N2; ++tt) a[j * N2 + tt] = *scratch(l, tt + N2 * (t + N2 * j));
    line_step2<N, PV, INV>(a, tw);
  }
  if (MIDSYNC) __syncthreads();
  if (act) {
#pragma unroll
    for (int j = 0; j < N1 / N2; ++j)
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) store(l, (t + N2 * j) + N1 * k2, a[j * N2 + k2], j * N2 + k2);
  }
  __syncthreads();
}

// Scratch lines A[l * AP + position] (AP odd) distinct from the phase's inputs and outputs.
template <typename V>
struct PitchedScratch {
  V* A;
  int AP;
  __device__ __forceinline__ V* operator()(int l, int pos) const { return A + (size_t)l * AP + pos; }
};

}  // namespace eacg
