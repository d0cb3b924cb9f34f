// Shared-memory Stockham FFT passes for one line of length N = prod(radices).
//
// A line lives in shared memory; TPL = N / E threads own it.  In every pass of
// radix R each thread loads E values (E / R butterflies) into registers, the
// CTA synchronises, then each thread twiddles, applies the radix-R DFT and
// stores its outputs in the autosorted position.  The whole CTA calls every
// pass (the barriers are uniform); threads without a line pass active=false.
//
// Transform convention: forward X_m = sum_j x_j e^{-2 pi i m j / N}, inverse
// with +i; neither is normalised.  The twiddle table tw[k] = e^{-2 pi i k / N}
// (k < N) is read from shared memory and conjugated for the inverse.
#pragma once
#include "common.cuh"

namespace eacg {

struct FftPlan {
  int N;      // line length
  int E;      // values per thread (template argument of the kernels)
  int TPL;    // threads per line = N / E
  int npass;  // number of radix passes
  int radix[8];
  int ns[8];  // product of the radices of the earlier passes
};

template <int R, bool INV, typename V>
__device__ __forceinline__ void dft_small(V* v) {
  using T = decltype(v[0].x);
  if constexpr (R == 2) {
    V a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else if constexpr (R == 3) {
    const T h = (T)0.86602540378443864676372317075293618;  // sin(2 pi / 3)
    V t1 = v[1] + v[2];
    V t2 = v[0] - cscale(t1, (T)0.5);
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
    const T c1 = (T)0.30901699437494742410229341718281906;   // cos(2 pi / 5)
    const T c2 = (T)-0.80901699437494742410229341718281906;  // cos(4 pi / 5)
    const T s1 = (T)0.95105651629515357211643933337938214;   // sin(2 pi / 5)
    const T s2 = (T)0.58778525229247312916870595463907277;   // sin(4 pi / 5)
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

template <typename V, int E, int R, bool INV>
__device__ __forceinline__ void fft_pass(V* line, int es, int t, int TPL, int N, int Ns, const V* tw,
                                         bool active) {
  constexpr int B = E / R;
  V v[E];
  const int NR = N / R;
  if (active) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * TPL;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b * R + r] = line[(j + r * NR) * es];
    }
  }
  __syncthreads();
  if (active) {
    const int step = N / (Ns * R);
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = t + b * TPL;
      const int jm = j % Ns;
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V w = tw[r * jm * step];
        if (INV) w.y = -w.y;
        v[b * R + r] = cmul(v[b * R + r], w);
      }
      dft_small<R, INV>(&v[b * R]);
      const int d = (j / Ns) * Ns * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) line[(d + r * Ns) * es] = v[b * R + r];
    }
  }
  __syncthreads();
}

// Full transform of one line (all passes).  Must be reached by every thread of the CTA.
template <typename V, int E, bool INV>
__device__ __forceinline__ void fft_line(V* line, int es, int t, const FftPlan& pl, const V* tw, bool active) {
  for (int s = 0; s < pl.npass; ++s) {
    const int R = pl.radix[s], Ns = pl.ns[s];
    if (R == 2) {
      if constexpr (E % 2 == 0) fft_pass<V, E, 2, INV>(line, es, t, pl.TPL, pl.N, Ns, tw, active);
    } else if (R == 3) {
      if constexpr (E % 3 == 0) fft_pass<V, E, 3, INV>(line, es, t, pl.TPL, pl.N, Ns, tw, active);
    } else if (R == 4) {
      if constexpr (E % 4 == 0) fft_pass<V, E, 4, INV>(line, es, t, pl.TPL, pl.N, Ns, tw, active);
    } else if (R == 5) {
      if constexpr (E % 5 == 0) fft_pass<V, E, 5, INV>(line, es, t, pl.TPL, pl.N, Ns, tw, active);
    }
  }
}

// Transform nlines lines of one CTA: line l starts at base + l * lstride, elements es apart.
// Threads are grouped TPL per line; the trip count is uniform across the CTA.
template <typename V, int E, bool INV>
__device__ __forceinline__ void fft_lines(V* base, int nlines, int lstride, int es, const FftPlan& pl,
                                          const V* tw) {
  const int TPL = pl.TPL;
  const int per = blockDim.x / TPL;
  const int g = threadIdx.x / TPL, t = threadIdx.x - g * TPL;
  for (int l0 = 0; l0 < nlines; l0 += per) {
    const int l = l0 + g;
    const bool active = (g < per) && (l < nlines);
    fft_line<V, E, INV>(base + (size_t)(active ? l : 0) * lstride, es, t, pl, tw, active);
  }
}

// Same with a list of line offsets (lines that are not equally spaced).
template <typename V, int E, bool INV>
__device__ __forceinline__ void fft_lines_list(V* base, const int* offs, int nlines, int es, const FftPlan& pl,
                                               const V* tw) {
  const int TPL = pl.TPL;
  const int per = blockDim.x / TPL;
  const int g = threadIdx.x / TPL, t = threadIdx.x - g * TPL;
  for (int l0 = 0; l0 < nlines; l0 += per) {
    const int l = l0 + g;
    const bool active = (g < per) && (l < nlines);
    fft_line<V, E, INV>(base + (active ? offs[l] : 0), es, t, pl, tw, active);
  }
}

}  // namespace eacg
