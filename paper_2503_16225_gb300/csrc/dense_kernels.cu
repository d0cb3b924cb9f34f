// Dense kernels of libeacg (sm_103a, FP64 complex), batched over k-points:
// Gram-type products A^H B with a long reduction, block updates A B with a small
// right factor, small Hermitian eigen-decompositions (parallel cyclic Jacobi),
// inverses, Lyapunov solves, pairings and norms, and the projected shifted
// solves of the block FOM.  Every matrix is column-major: A_ij = A[j * ld + i].
// All reductions run over fixed chunks combined in a fixed order, so results do
// not depend on scheduling.
#include <math.h>

#include <algorithm>
#include <array>
#include <map>
#include <mutex>

#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.h"

namespace eacg {

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // c + a * b
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 c) {  // c + conj(a) * b
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// FP64 reciprocal square root and reciprocal by Newton-Raphson from an FP32 seed: two steps
// take the seed's ~1e-7 relative error to FP64 rounding (quadratic convergence), using only
// multiply-adds, which GB300 executes far faster than its FP64 divide and square-root
// sequences.  The argument (positive, normal) is first scaled by an exact power of two into
// [1, 4) so that the FP32 seed never under- or overflows.
//   y <- y (3 - x y^2) / 2          for 1 / sqrt(x)
//   y <- y (2 - x y)                for 1 / x
__device__ __forceinline__ double pow2(int e) {  // 2^e for -1022 <= e <= 1023
  return __longlong_as_double((long long)(e + 1023) << 52);
}
__device__ __forceinline__ int exponent_of(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  const int half = exponent_of(x) >> 1;  // floor(e / 2)
  const double xs = x * pow2(-2 * half);  // in [1, 4)
  double y = (double)rsqrtf((float)xs);
  y = y * fma(-0.5 * xs * y, y, 1.5);
  y = y * fma(-0.5 * xs * y, y, 1.5);
  return y * pow2(-half);
}
__device__ __forceinline__ double rcp_nr(double x) {
  const int e = exponent_of(x);
  const double xs = x * pow2(-e);  // in [1, 2)
  double y = (double)(1.0f / (float)xs);
  y = y * fma(-xs, y, 2.0);
  y = y * fma(-xs, y, 2.0);
  return y * pow2(-e);
}

// ----------------------------------------------------------------------------- A^H B
// Templated on the block precision T (double or float): A and B are cplx<T>, the products
// are accumulated in T within a chunk of rows, the chunk partials and the result are FP64.
// A CTA computes one 16 x 16 tile of C over one chunk of CN_CHUNK rows.  The chunk is read in
// rounds of CN_LANES stages of CN_SUB rows; stage v of every round belongs to summation lane v,
// whose products accumulate in their own T-precision sum, and the lane sums are added in FP64
// in lane order at the end.  G = 1, 2 or 4 groups of 256 threads share the lanes (group g takes
// lanes g, g + G, ...), so every G performs the same additions in the same order and gives
// bitwise the same partial: the tile choice (dense_tune_cn, timed at system set-up and cached
// for the process; untuned shapes use 4) changes only the speed.
constexpr int CN_TILE = 16;
constexpr int CN_CHUNK = 1024;  // largest number of rows per partial
constexpr int CN_SUB = 16;      // rows per stage
constexpr int CN_LANES = 4;     // summation lanes (stages per round)
// CTAs a small-problem GEMM launch aims at (two per SM): GB300 executes 2 FP64 FMA per
// SM-clock, so an FP64 contraction confined to a few CTAs leaves almost all of its FP64
// throughput unused.
constexpr int GEMM_TARGET_CTAS = 2 * 152;

// Rows per partial of A^H B: CN_CHUNK, or fewer (a multiple of CN_SUB * CN_LANES) when the
// tiles of all k-points would not fill GEMM_TARGET_CTAS CTAs.  Depends on the shape only.
static int cn_chunk(int K, int L, int m, int n) {
  const int tiles = ((m + CN_TILE - 1) / CN_TILE) * ((n + CN_TILE - 1) / CN_TILE);
  const long long have = (long long)tiles * K;
  const int want = (int)std::min<long long>(GEMM_TARGET_CTAS, (GEMM_TARGET_CTAS + have - 1) / have);
  constexpr int R = CN_SUB * CN_LANES;
  int chunk = (L + want - 1) / want;
  chunk = ((chunk + R - 1) / R) * R;
  return std::max(R, std::min(CN_CHUNK, chunk));
}

size_t dense_cn_work(int K, int L, int m, int n) {
  // at most ceil(L / CN_CHUNK) partials per element for large tile counts; otherwise at most
  // ceil(GEMM_TARGET_CTAS / (tiles K)) + 1 of them, with m n <= tiles * CN_TILE^2
  const int nch = (L + CN_CHUNK - 1) / CN_CHUNK;
  return (size_t)K * (nch + 1) * m * n + (size_t)GEMM_TARGET_CTAS * CN_TILE * CN_TILE;
}

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float2 cfmac(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
// double-float complex multiply-adds (FP64-accurate products and sums on the FP32 pipe)
__device__ __forceinline__ dcomplex cfma(dcomplex a, dcomplex b, dcomplex c) {  // c + a * b
  return {c.x + (a.x * b.x - a.y * b.y), c.y + (a.x * b.y + a.y * b.x)};
}
__device__ __forceinline__ dcomplex cfmac(dcomplex a, dcomplex b, dcomplex c) {  // c + conj(a) * b
  return {c.x + (a.x * b.x + a.y * b.y), c.y + (a.x * b.y - a.y * b.x)};
}

template <typename T, typename TM, int CN_GROUPS>
__global__ void __launch_bounds__(CN_TILE * CN_TILE * CN_GROUPS)
    k_gemm_cn_partial(int L, int m, int n, const cplx<T>* __restrict__ A, size_t sA, int lda,
                      const cplx<T>* __restrict__ B, size_t sB, int ldb, double2* __restrict__ part,
                      const int* __restrict__ kactive, int chunk) {
  using V = cplx<TM>;  // arithmetic type (the storage type T, or double-float for FP64 storage)
  constexpr int PER = CN_LANES / CN_GROUPS;  // lanes per group
  constexpr int NT = CN_TILE * CN_TILE * CN_GROUPS;
  const int k = blockIdx.z;
  if (kactive && !kactive[k]) return;
  const int tiles_m = (m + CN_TILE - 1) / CN_TILE;
  const int tm = blockIdx.x % tiles_m, tn = blockIdx.x / tiles_m;
  const int ch = blockIdx.y, nch = gridDim.y;
  const int g = threadIdx.x / (CN_TILE * CN_TILE), t = threadIdx.x % (CN_TILE * CN_TILE);
  const int ti = t % CN_TILE, tj = t / CN_TILE;
  const int i0 = tm * CN_TILE, j0 = tn * CN_TILE;
  __shared__ V sa[CN_LANES][CN_SUB][CN_TILE + 1];
  __shared__ V sb[CN_LANES][CN_SUB][CN_TILE + 1];
  const cplx<T>* Ak = A + k * sA;
  const cplx<T>* Bk = B + k * sB;
  const V zero = czero<V>();
  V acc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) acc[i] = zero;
  const int l_beg = ch * chunk, l_end = min(L, l_beg + chunk);
  for (int s0 = l_beg; s0 < l_end; s0 += CN_SUB * CN_LANES) {  // uniform trip count over the CTA
    for (int e = threadIdx.x; e < CN_LANES * CN_SUB * CN_TILE; e += NT) {
      const int v = e / (CN_SUB * CN_TILE), w = e - v * (CN_SUB * CN_TILE);
      const int c = w / CN_SUB, r = w - c * CN_SUB;
      const int l = s0 + v * CN_SUB + r;
      sa[v][r][c] = (l < l_end && i0 + c < m) ? cvt<V>(Ak[(size_t)(i0 + c) * lda + l]) : zero;
      sb[v][r][c] = (l < l_end && j0 + c < n) ? cvt<V>(Bk[(size_t)(j0 + c) * ldb + l]) : zero;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int v = g + i * CN_GROUPS;
#pragma unroll
      for (int r = 0; r < CN_SUB; ++r) acc[i] = cfmac(sa[v][r][ti], sb[v][r][tj], acc[i]);
    }
    __syncthreads();
  }
  // lane sums added in lane order (CN_LANES * 256 values fit in sa)
  V* red = &sa[0][0][0];
#pragma unroll
  for (int i = 0; i < PER; ++i) red[(g + i * CN_GROUPS) * CN_TILE * CN_TILE + t] = acc[i];
  __syncthreads();
  if (g == 0 && i0 + ti < m && j0 + tj < n) {
    double2 sum = to_d(red[t]);
    for (int v = 1; v < CN_LANES; ++v) sum = sum + to_d(red[v * CN_TILE * CN_TILE + t]);
    part[(((size_t)k * nch + ch) * n + (j0 + tj)) * m + (i0 + ti)] = sum;
  }
}

__global__ void k_gemm_cn_reduce(int m, int n, int nch, const double2* __restrict__ part, double2* __restrict__ C,
                                 size_t sC, int ldc, double2 alpha, double2 beta, const int* __restrict__ kactive) {
  const int k = blockIdx.y;
  if (kactive && !kactive[k]) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * n; e += gridDim.x * blockDim.x) {
    const int j = e / m, i = e - j * m;
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < nch; ++c) s = s + part[(((size_t)k * nch + c) * n + j) * m + i];
    double2* cp = C + k * sC + (size_t)j * ldc + i;
    double2 r = cmul(alpha, s);
    if (beta.x != 0.0 || beta.y != 0.0) r = r + cmul(beta, *cp);
    *cp = r;
  }
}

namespace {
std::mutex g_cn_mu;
std::map<std::array<int, 5>, int> g_cn_groups;  // (device, element bytes, m, n, row chunks) buckets -> G

int pow2_bucket(int x) {
  int b = 16;
  while (b < x && b < 4096) b <<= 1;
  return b;
}
std::array<int, 5> cn_key(size_t es, int m, int n, int L) {
  int dev = 0;
  cudaGetDevice(&dev);
  return {dev, (int)es, pow2_bucket(m), pow2_bucket(n), std::min(8, (L + CN_CHUNK - 1) / CN_CHUNK)};
}
int g_cn_force = 0;  // 1, 2 or 4 overrides the tuned choice for every shape
int cn_groups_for(size_t es, int m, int n, int L) {
  std::lock_guard<std::mutex> lock(g_cn_mu);
  if (g_cn_force) return g_cn_force;
  auto it = g_cn_groups.find(cn_key(es, m, n, L));
  return it == g_cn_groups.end() ? 4 : it->second;
}
}  // namespace

template <typename T, typename TM>
static void gemm_cn_partial_launch(int G, dim3 g1, int L, int m, int n, const cplx<T>* A, size_t sA, int lda,
                                   const cplx<T>* B, size_t sB, int ldb, double2* work, const int* kactive,
                                   int chunk, cudaStream_t st) {
  if (G == 1)
    k_gemm_cn_partial<T, TM, 1><<<g1, CN_TILE * CN_TILE, 0, st>>>(L, m, n, A, sA, lda, B, sB, ldb, work, kactive,
                                                                   chunk);
  else if (G == 2)
    k_gemm_cn_partial<T, TM, 2><<<g1, CN_TILE * CN_TILE * 2, 0, st>>>(L, m, n, A, sA, lda, B, sB, ldb, work,
                                                                       kactive, chunk);
  else
    k_gemm_cn_partial<T, TM, 4><<<g1, CN_TILE * CN_TILE * 4, 0, st>>>(L, m, n, A, sA, lda, B, sB, ldb, work,
                                                                       kactive, chunk);
  count_launch();
}

void dense_cn_reduce(int K, int m, int n, int nch, const double2* work, double2* C, size_t sC, int ldc,
                     double2 alpha, double2 beta, const int* kactive, cudaStream_t st) {
  if (K <= 0 || m <= 0 || n <= 0) return;
  dim3 g2((m * n + 255) / 256, K);
  k_gemm_cn_reduce<<<g2, 256, 0, st>>>(m, n, nch, work, C, sC, ldc, alpha, beta, kactive);
  count_launch();
}

template <typename T, typename TM = T>
static void gemm_cn_t(int K, int L, int m, int n, const cplx<T>* A, size_t sA, int lda, const cplx<T>* B, size_t sB,
                      int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta, double2* work,
                      const int* kactive, cudaStream_t st, int G = 0) {
  if (K <= 0 || m <= 0 || n <= 0) return;
  const int chunk = cn_chunk(K, L, m, n);
  const int nch = (L + chunk - 1) / chunk;
  const int tiles = ((m + CN_TILE - 1) / CN_TILE) * ((n + CN_TILE - 1) / CN_TILE);
  dim3 g1(tiles, nch > 0 ? nch : 1, K);
  if (nch > 0)
    gemm_cn_partial_launch<T, TM>(G > 0 ? G : cn_groups_for(sizeof(cplx<T>), m, n, L), g1, L, m, n, A, sA, lda, B,
                                  sB, ldb, work, kactive, chunk, st);
  dim3 g2((m * n + 255) / 256, K);
  k_gemm_cn_reduce<<<g2, 256, 0, st>>>(m, n, nch, work, C, sC, ldc, alpha, beta, kactive);
  count_launch();
}

// Times G = 1, 2, 4 on the given operands (Kt k-points) and records the fastest for the shape
// bucket of (element size, m, n, L); a bucket already tuned is kept.
template <typename T>
static void tune_cn_t(int Kt, int L, int m, int n, const cplx<T>* A, size_t sA, int lda, const cplx<T>* B,
                      size_t sB, int ldb, double2* C, double2* work, cudaStream_t st) {
  const auto key = cn_key(sizeof(cplx<T>), m, n, L);
  {
    std::lock_guard<std::mutex> lock(g_cn_mu);
    if (g_cn_groups.count(key)) return;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const double2 one = make_double2(1.0, 0.0), zero = make_double2(0.0, 0.0);
  int best_g = 4;
  float best = 0.f;
  for (int G : {4, 2, 1}) {
    gemm_cn_t<T>(Kt, L, m, n, A, sA, lda, B, sB, ldb, C, (size_t)m * n, m, one, zero, work, nullptr, st, G);
    cudaEventRecord(a, st);
    for (int r = 0; r < 3; ++r)
      gemm_cn_t<T>(Kt, L, m, n, A, sA, lda, B, sB, ldb, C, (size_t)m * n, m, one, zero, work, nullptr, st, G);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (G == 4 || ms < best) {
      best = ms;
      best_g = G;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::lock_guard<std::mutex> lock(g_cn_mu);
  g_cn_groups.emplace(key, best_g);
}

void dense_tune_cn(int Kt, int L, int m, int n, int prec, const void* A, size_t sA, int lda, const void* B,
                   size_t sB, int ldb, double2* C, double2* work, cudaStream_t st) {
  if (Kt <= 0 || m <= 0 || n <= 0 || L <= 0) return;
  if (prec)
    tune_cn_t<float>(Kt, L, m, n, (const float2*)A, sA, lda, (const float2*)B, sB, ldb, C, work, st);
  else
    tune_cn_t<double>(Kt, L, m, n, (const double2*)A, sA, lda, (const double2*)B, sB, ldb, C, work, st);
}

int dense_cn_groups(int m, int n, int L, int prec) {
  return cn_groups_for(prec ? sizeof(float2) : sizeof(double2), m, n, L);
}

int dense_cn_force(int groups) {
  if (groups != 0 && groups != 1 && groups != 2 && groups != 4) return -1;
  std::lock_guard<std::mutex> lock(g_cn_mu);
  g_cn_force = groups;
  return 0;
}

void dense_gemm_cn(int K, int L, int m, int n, const double2* A, size_t sA, int lda, const double2* B, size_t sB,
                   int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta, double2* work,
                   const int* kactive, cudaStream_t st, int df) {
  if (df)
    gemm_cn_t<double, dfloat>(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, alpha, beta, work, kactive, st);
  else
    gemm_cn_t<double>(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, alpha, beta, work, kactive, st);
}
void dense_gemm_cn32(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const float2* B, size_t sB,
                     int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta, double2* work,
                     const int* kactive, cudaStream_t st) {
  gemm_cn_t<float>(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, alpha, beta, work, kactive, st);
}

// ----------------------------------------------------------------------------- A B (small B)
// C (L x n, VC) = alpha A (L x m, cplx<T>) B (m x n, FP64, staged in T) + beta C; the products
// accumulate in T and the result is formed in the precision of C (VC = cplx<T>, or double2
// for FP32 operands added into an FP64 block).
constexpr int NN_COLS = 8;
constexpr int NN_ROWS = 64;
template <typename T, typename TM, typename VC>
__global__ void k_gemm_nn(int L, int m, int n, const cplx<T>* __restrict__ A, size_t sA, int lda,
                          const double2* __restrict__ B, size_t sB, int ldb, VC* __restrict__ C, size_t sC,
                          int ldc, double2 alpha, double2 beta, const int* __restrict__ kactive) {
  using V = cplx<TM>;  // arithmetic type (the storage type T, or double-float for FP64 storage)
  using TC = decltype(C[0].x);
  const int k = blockIdx.y;
  if (kactive && !kactive[k]) return;
  __shared__ V sb[NN_ROWS][NN_COLS];
  // blockIdx.x = row block + rowblocks * column group; group gi takes the column groups of
  // NN_COLS columns j0 = NN_COLS (gi + ngroups i)
  const int rowblocks = (L + blockDim.x - 1) / blockDim.x;
  const int rb = blockIdx.x % rowblocks, gi = blockIdx.x / rowblocks;
  const int ngroups = gridDim.x / rowblocks;
  const int l = rb * blockDim.x + threadIdx.x;
  const cplx<T>* Ak = A + k * sA;
  const double2* Bk = B + k * sB;
  VC* Ck = C + k * sC;
  const bool bz = (beta.x == 0.0 && beta.y == 0.0);
  const VC al = to_c<TC>(alpha), be = to_c<TC>(beta);
  const V zero = czero<V>();
  for (int j0 = NN_COLS * gi; j0 < n; j0 += NN_COLS * ngroups) {
    V acc[NN_COLS];
#pragma unroll
    for (int jj = 0; jj < NN_COLS; ++jj) acc[jj] = zero;
    for (int i0 = 0; i0 < m; i0 += NN_ROWS) {
      __syncthreads();
      for (int e = threadIdx.x; e < NN_ROWS * NN_COLS; e += blockDim.x) {
        const int r = e / NN_COLS, c = e - r * NN_COLS;
        sb[r][c] = (i0 + r < m && j0 + c < n) ? cvt<V>(Bk[(size_t)(j0 + c) * ldb + i0 + r]) : zero;
      }
      __syncthreads();
      if (l < L) {
        const int iend = min(NN_ROWS, m - i0);
        for (int r = 0; r < iend; ++r) {
          const V a = cvt<V>(Ak[(size_t)(i0 + r) * lda + l]);
#pragma unroll
          for (int jj = 0; jj < NN_COLS; ++jj) acc[jj] = cfma(a, sb[r][jj], acc[jj]);
        }
      }
    }
    if (l < L) {
#pragma unroll
      for (int jj = 0; jj < NN_COLS; ++jj) {
        if (j0 + jj < n) {
          VC* cp = Ck + (size_t)(j0 + jj) * ldc + l;
          VC r = cmul(al, cvt<VC>(acc[jj]));
          if (!bz) r = r + cmul(be, *cp);
          *cp = r;
        }
      }
    }
  }
}

template <typename T, typename VC, typename TM = T>
static void gemm_nn_t(int K, int L, int m, int n, const cplx<T>* A, size_t sA, int lda, const double2* B, size_t sB,
                      int ldb, VC* C, size_t sC, int ldc, double2 alpha, double2 beta, const int* kactive,
                      cudaStream_t st) {
  if (K <= 0 || L <= 0 || n <= 0) return;
  // every output element is one thread's fixed-order sum whatever the split, so the column
  // groups only spread small problems over more SMs (GB300's FP64 units are 2 FMA per SM-clock)
  const int rowblocks = (L + 127) / 128;
  const int colgroups = (n + NN_COLS - 1) / NN_COLS;
  const int want = (GEMM_TARGET_CTAS + rowblocks * K - 1) / (rowblocks * K);
  const int groups = std::max(1, std::min(colgroups, want));
  dim3 g(rowblocks * groups, K);
  k_gemm_nn<T, TM, VC><<<g, 128, 0, st>>>(L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, alpha, beta, kactive);
  count_launch();
}

void dense_gemm_nn(int K, int L, int m, int n, const double2* A, size_t sA, int lda, const double2* B, size_t sB,
                   int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta, const int* kactive,
                   cudaStream_t st, int df) {
  if (df)
    gemm_nn_t<double, double2, dfloat>(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, alpha, beta, kactive, st);
  else
    gemm_nn_t<double, double2>(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, alpha, beta, kactive, st);
}
void dense_gemm_nn32(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const double2* B, size_t sB,
                     int ldb, float2* C, size_t sC, int ldc, double2 alpha, double2 beta, const int* kactive,
                     cudaStream_t st) {
  gemm_nn_t<float>(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, alpha, beta, kactive, st);
}
void dense_gemm_nn32_into64(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const double2* B,
                            size_t sB, int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta,
                            const int* kactive, cudaStream_t st) {
  gemm_nn_t<float>(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, alpha, beta, kactive, st);
}

// ----------------------------------------------------------------------------- FP32 block helpers
__global__ void k_to32(size_t n, const double2* __restrict__ x, double sc, float2* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = make_float2((float)(sc * x[i].x), (float)(sc * x[i].y));
}
__global__ void k_to64(size_t n, const float2* __restrict__ x, double2* __restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = make_double2((double)x[i].x, (double)x[i].y);
}
// out = a x + b y (y may be null), FP32 blocks with FP64 scalars
__global__ void k_axpby32(size_t n, double2 a, const float2* __restrict__ x, double2 b, const float2* __restrict__ y,
                          float2* __restrict__ out) {
  const float2 af = make_float2((float)a.x, (float)a.y), bf = make_float2((float)b.x, (float)b.y);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float2 r = cmul(af, x[i]);
    if (y) r = r + cmul(bf, y[i]);
    out[i] = r;
  }
}
__global__ void k_norms2_32(size_t len, const float2* __restrict__ V, double* __restrict__ out) {
  __shared__ double sh[256];
  const int k = blockIdx.x;
  const float2* v = V + (size_t)k * len;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < len; i += blockDim.x) s += (double)v[i].x * v[i].x + (double)v[i].y * v[i].y;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int q = blockDim.x / 2; q > 0; q >>= 1) {
    if (threadIdx.x < q) sh[threadIdx.x] += sh[threadIdx.x + q];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = sh[0];
}
__global__ void k_tpa32(int p, int n_max, const double* __restrict__ kin, const double* __restrict__ alpha,
                        const float2* __restrict__ in, float2* __restrict__ out) {
  const int k = blockIdx.y;
  const size_t tot = (size_t)p * n_max;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n_max), g = (int)(e % n_max);
    const float f = (float)(1.0 / (kin[(size_t)k * n_max + g] + alpha[(size_t)k * p + i]));
    const float2 v = in[(size_t)k * tot + e];
    out[(size_t)k * tot + e] = make_float2(v.x * f, v.y * f);
  }
}
void dense_to32(size_t n, const double2* x, double sc, float2* y, cudaStream_t st) {
  k_to32<<<(int)std::min((size_t)2048, (n + 255) / 256 + 1), 256, 0, st>>>(n, x, sc, y);
  count_launch();
}
void dense_to64(size_t n, const float2* x, double2* y, cudaStream_t st) {
  k_to64<<<(int)std::min((size_t)2048, (n + 255) / 256 + 1), 256, 0, st>>>(n, x, y);
  count_launch();
}
void dense_axpby32(size_t n, double2 a, const float2* x, double2 b, const float2* y, float2* out, cudaStream_t st) {
  k_axpby32<<<(int)std::min((size_t)2048, (n + 255) / 256 + 1), 256, 0, st>>>(n, a, x, b, y, out);
  count_launch();
}
void dense_norms2_32(int K, size_t len, const float2* V, double* out, cudaStream_t st) {
  k_norms2_32<<<K, 256, 0, st>>>(len, V, out);
  count_launch();
}
void dense_tpa32(int K, int p, int n_max, const double* kin, const double* alpha, const float2* in, float2* out,
                 cudaStream_t st) {
  dim3 g(64, K);
  k_tpa32<<<g, 256, 0, st>>>(p, n_max, kin, alpha, in, out);
  count_launch();
}

// ----------------------------------------------------------------------------- Hermitian eig
// Parallel cyclic Jacobi (round-robin pairs) on one p x p Hermitian matrix per CTA, FP64.
// The rotation parameters use multiply-add refinements of FP32 reciprocal / rsqrt seeds in
// FP64 (no FP64 divide or square root).  Converged when the off-diagonal norm is below
// 1e-14 of the matrix norm.
template <typename T>
struct JacobiMath;
template <>
struct JacobiMath<double> {
  static __device__ __forceinline__ double rsq(double x) { return rsqrt_nr(x); }
  static __device__ __forceinline__ double rcp(double x) { return rcp_nr(x); }
  static constexpr double tol2 = 1e-28, neg = 1e-16, tiny = 1e-280;
};
template <typename T>
__global__ void k_heig(int p, const double2* __restrict__ Ag, size_t sA, double* __restrict__ w,
                       double2* __restrict__ Vg, const int* __restrict__ kactive, unsigned char* gscr,
                       size_t gstride) {
  using V2 = cplx<T>;
  using M = JacobiMath<T>;
  const int k = blockIdx.x;
  if (kactive && !kactive[k]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int pe = p + (p & 1);  // even number of slots (a dummy index when p is odd)
  // A and V in shared memory, or (gscr set, large p) in this k's global scratch
  V2* A = reinterpret_cast<V2*>(gscr ? gscr + (size_t)k * gstride : smem_raw);
  V2* V = A + p * p;
  T* rot = reinterpret_cast<T*>(gscr ? smem_raw : reinterpret_cast<unsigned char*>(V + p * p));  // [pe/2][4]
  T* red = rot + 2 * pe;                     // [2 + 2 * warps]
  const double2* Ak = Ag + k * sA;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    // symmetrise exactly while loading: upper from (A_ij + conj A_ji) / 2
    const double2 a = Ak[(size_t)j * p + i], b = Ak[(size_t)i * p + j];
    double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    if (i == j) h.y = 0.0;
    A[e] = to_c<T>(h);
    V[e].x = (T)(i == j ? 1 : 0);
    V[e].y = (T)0;
  }
  __syncthreads();
  const int npair = pe / 2;
  // round-robin pairing (circle method): slot 0 fixed, slots 1..pe-1 rotate by one per round
  auto slot = [pe](int pos, int round) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (pe - 1); };
  for (int sweep = 0; sweep < 20; ++sweep) {
    {
      // off-diagonal and diagonal squared norms: fixed per-thread strides, then a fixed
      // shuffle tree per warp and a fixed warp order (deterministic)
      T off = 0, dia = 0;
      for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int j = e / p, i = e - j * p;
        const T a2 = A[e].x * A[e].x + A[e].y * A[e].y;
        if (i == j)
          dia += a2;
        else
          off += a2;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_down_sync(0xffffffffu, off, o);
        dia += __shfl_down_sync(0xffffffffu, dia, o);
      }
      if ((threadIdx.x & 31) == 0) {
        red[2 + 2 * (threadIdx.x >> 5)] = off;
        red[3 + 2 * (threadIdx.x >> 5)] = dia;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        T so = 0, sd = 0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) {
          so += red[2 + 2 * wi];
          sd += red[3 + 2 * wi];
        }
        red[0] = so;
        red[1] = sd;
      }
    }
    __syncthreads();
    const T fro2 = red[0] + red[1];
    const bool done = !(red[0] > M::tol2 * fro2);
    __syncthreads();
    if (done) break;
    const T negligible = M::neg * sqrt(fro2) / p;
    for (int round = 0; round < pe - 1; ++round) {
      // rotation parameters for each pair
      for (int t = threadIdx.x; t < npair; t += blockDim.x) {
        int i = slot(t, round), j = slot(pe - 1 - t, round);
        if (i > j) {
          const int q = i;
          i = j;
          j = q;
        }
        T c = 1, s = 0, cf = 1, sf = 0;
        if (j < p) {
          const V2 b = A[j * p + i];
          const T r2 = b.x * b.x + b.y * b.y;
          if (r2 > M::tiny && r2 > negligible * negligible) {
            const T a = A[i * p + i].x, d = A[j * p + j].x;
            const T ir = M::rsq(r2);                       // 1 / |b|
            const T zeta = (T)0.5 * (d - a) * ir;
            const T h = (T)1 + zeta * zeta;
            const T den = fabs(zeta) + h * M::rsq(h);      // |zeta| + sqrt(1 + zeta^2)
            const T tt = (zeta >= 0 ? (T)1 : (T)-1) * M::rcp(den);
            c = M::rsq((T)1 + tt * tt);
            s = tt * c;
            cf = b.x * ir;  // e^{i phi} = b / |b|
            sf = b.y * ir;
          }
        }
        rot[4 * t + 0] = c;
        rot[4 * t + 1] = s;
        rot[4 * t + 2] = cf;
        rot[4 * t + 3] = sf;
      }
      __syncthreads();
      // columns: (A_ki, A_kj) <- (c A_ki - s e^{-i phi} A_kj, s A_ki + c e^{-i phi} A_kj); same for V
      for (int e = threadIdx.x; e < npair * p; e += blockDim.x) {
        const int t = e / p, r = e - t * p;
        int i = slot(t, round), j = slot(pe - 1 - t, round);
        if (i > j) {
          const int q = i;
          i = j;
          j = q;
        }
        if (j >= p) continue;
        const T c = rot[4 * t], s = rot[4 * t + 1];
        V2 em;
        em.x = rot[4 * t + 2];
        em.y = -rot[4 * t + 3];  // e^{-i phi}
        {
          const V2 ai = A[i * p + r], aj = cmul(em, A[j * p + r]);
          A[i * p + r] = cscale(ai, c) - cscale(aj, s);
          A[j * p + r] = cscale(ai, s) + cscale(aj, c);
        }
        {
          const V2 vi = V[i * p + r], vj = cmul(em, V[j * p + r]);
          V[i * p + r] = cscale(vi, c) - cscale(vj, s);
          V[j * p + r] = cscale(vi, s) + cscale(vj, c);
        }
      }
      __syncthreads();
      // rows: (A_ik, A_jk) <- (c A_ik - s e^{i phi} A_jk, s A_ik + c e^{i phi} A_jk); the annihilated
      // pair is set to exactly zero and the diagonal kept real
      for (int e = threadIdx.x; e < npair * p; e += blockDim.x) {
        const int t = e / p, col = e - t * p;
        int i = slot(t, round), j = slot(pe - 1 - t, round);
        if (i > j) {
          const int q = i;
          i = j;
          j = q;
        }
        if (j >= p) continue;
        const T c = rot[4 * t], s = rot[4 * t + 1];
        V2 ep;
        ep.x = rot[4 * t + 2];
        ep.y = rot[4 * t + 3];
        const V2 ai = A[col * p + i], aj = cmul(ep, A[col * p + j]);
        V2 ni = cscale(ai, c) - cscale(aj, s);
        V2 nj = cscale(ai, s) + cscale(aj, c);
        if (s != (T)0 && col == j) ni.x = ni.y = (T)0;  // (i, j)
        if (s != (T)0 && col == i) nj.x = nj.y = (T)0;  // (j, i)
        if (col == i) ni.y = (T)0;
        if (col == j) nj.y = (T)0;
        A[col * p + i] = ni;
        A[col * p + j] = nj;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  // sort ascending by rank (ties by index) and write out
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const T wi = A[i * p + i].x;
    int rank = 0;
    for (int j = 0; j < p; ++j) {
      const T wj = A[j * p + j].x;
      if (wj < wi || (wj == wi && j < i)) ++rank;
    }
    w[(size_t)k * p + rank] = (double)wi;
    for (int r = 0; r < p; ++r) Vg[(size_t)k * p * p + (size_t)rank * p + r] = to_d(V[i * p + r]);
  }
}

// Matrices of the p x p kernels live in shared memory up to this size, else in global scratch.
constexpr size_t PP_SMEM_MAX = 200 * 1024;
constexpr int PP_GLOBAL_THREADS = 1024;  // threads of a p x p kernel working from global scratch

static size_t heig_big(int p) { return sizeof(double2) * 2 * (size_t)p * p; }
static size_t inverse_big(int p) { return sizeof(double2) * 2 * (size_t)p * p; }
static size_t lyap_big(int p) { return sizeof(double2) * 3 * (size_t)p * p; }
static size_t pivchol_big(int p) { return sizeof(double2) * 2 * (size_t)p * p + sizeof(int) * (size_t)p + 16; }
static size_t pp_stride(int p) {
  auto g = [](size_t b) { return b > PP_SMEM_MAX ? ((b + 255) & ~(size_t)255) : (size_t)0; };
  return std::max(std::max(g(heig_big(p)), g(inverse_big(p))), std::max(g(lyap_big(p)), g(pivchol_big(p))));
}
size_t dense_pp_scratch(int K, int p) { return (size_t)K * pp_stride(p); }

template <typename T>
static void heig_t(int K, int p, const double2* A, size_t sA, double* w, double2* V, const int* kactive,
                   void* scratch, cudaStream_t st) {
  const int pe = p + (p & 1);
  const bool big = heig_big(p) > PP_SMEM_MAX;
  if (big && !scratch) return;  // callers size the scratch with dense_pp_scratch
  const int threads = big ? PP_GLOBAL_THREADS : (p <= 16 ? 64 : 256);
  const size_t small = sizeof(T) * (2 * pe + 2 + 2 * (threads / 32)) + 16;
  const size_t sm = (big ? 0 : sizeof(cplx<T>) * 2 * p * p) + small;
  ensure_smem((const void*)k_heig<T>, sm);
  k_heig<T><<<K, threads, sm, st>>>(p, A, sA, w, V, kactive, big ? (unsigned char*)scratch : nullptr,
                                    pp_stride(p));
  count_launch();
}

void dense_heig(int K, int p, const double2* A, size_t sA, double* w, double2* V, const int* kactive,
                cudaStream_t st, void* scratch) {
  heig_t<double>(K, p, A, sA, w, V, kactive, scratch, st);
}
// out = V diag(f(w)) V^H, f(x) = x^expo for x > cut_rel * max(w, 0), else 0
__global__ void k_eig_func(int p, const double2* __restrict__ V, const double* __restrict__ w, double expo,
                           double cut_rel, double2* __restrict__ out, const int* __restrict__ kactive) {
  const int k = blockIdx.x;
  if (kactive && !kactive[k]) return;
  extern __shared__ double fsm[];
  const double* wk = w + (size_t)k * p;
  const double2* Vk = V + (size_t)k * p * p;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < p; ++i) mx = fmax(mx, wk[i]);
    fsm[p] = mx;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const double x = wk[i];
    fsm[i] = (x > cut_rel * fsm[p] && x > 0.0) ? pow(x, expo) : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    double2 s = make_double2(0.0, 0.0);
    for (int l = 0; l < p; ++l) {
      const double f = fsm[l];
      if (f != 0.0) s = s + cscale(cmul(Vk[l * p + i], cconj(Vk[l * p + j])), f);
    }
    out[(size_t)k * p * p + e] = s;
  }
}

void dense_eig_func(int K, int p, const double2* V, const double* w, double expo, double cut_rel, double2* out,
                    const int* kactive, cudaStream_t st) {
  k_eig_func<<<K, p > 64 ? 512 : 128, sizeof(double) * (p + 1), st>>>(p, V, w, expo, cut_rel, out, kactive);
  count_launch();
}

// Largest value over the warp with its index, the smallest index on ties (every lane gets it).
__device__ __forceinline__ void warp_argmax(double& v, int& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}

// Gauss-Jordan inverse with partial pivoting, one CTA per matrix; the augmented matrix in
// shared memory, or (gscr set, large p) in this k's global scratch.
__global__ void k_inverse(int p, const double2* __restrict__ A, double2* __restrict__ Ainv, int* __restrict__ info,
                          unsigned char* gscr, size_t gstride) {
  const int k = blockIdx.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* M = reinterpret_cast<double2*>(gscr ? gscr + (size_t)k * gstride : smem_raw);  // [2p][p] augmented
  __shared__ int piv;
  const double2* Ak = A + (size_t)k * p * p;
  for (int e = threadIdx.x; e < 2 * p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    M[e] = j < p ? Ak[e] : make_double2(i == j - p ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int c = 0; c < p; ++c) {
    if (threadIdx.x < 32) {  // pivot: the first row of largest modulus in column c
      double bv = -1.0;
      int best = p;
      for (int i = c + (int)threadIdx.x; i < p; i += 32) {
        const double v = cabs2(M[c * p + i]);
        if (v > bv) {
          bv = v;
          best = i;
        }
      }
      warp_argmax(bv, best);
      if (threadIdx.x == 0) {
        piv = best;
        if (bv == 0.0 && info) info[k] = c + 1;
      }
    }
    __syncthreads();
    const int r = piv;
    if (r != c) {
      for (int j = threadIdx.x; j < 2 * p; j += blockDim.x) {
        const double2 t = M[j * p + c];
        M[j * p + c] = M[j * p + r];
        M[j * p + r] = t;
      }
    }
    __syncthreads();
    const double2 d = M[c * p + c];
    const double dd = cabs2(d);
    const double2 dinv = dd > 0 ? make_double2(d.x / dd, -d.y / dd) : make_double2(0.0, 0.0);
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * p; j += blockDim.x) M[j * p + c] = cmul(M[j * p + c], dinv);
    __syncthreads();
    for (int e = threadIdx.x; e < p * 2 * p; e += blockDim.x) {
      const int j = e / p, i = e - j * p;
      if (i != c && j != c) {
        const double2 f = M[c * p + i];
        M[j * p + i] = M[j * p + i] - cmul(f, M[j * p + c]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p; i += blockDim.x)
      if (i != c) M[c * p + i] = make_double2(0.0, 0.0);
    __syncthreads();
    // column c of the left half now is e_c; its inverse part lives in column p + c
  }
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) Ainv[(size_t)k * p * p + e] = M[p * p + e];
}

void dense_inverse(int K, int p, const double2* A, double2* Ainv, int* info, cudaStream_t st, void* scratch) {
  const bool big = inverse_big(p) > PP_SMEM_MAX;
  if (big && !scratch) return;  // callers size the scratch with dense_pp_scratch
  const size_t sm = big ? 0 : inverse_big(p);
  ensure_smem((const void*)k_inverse, sm);
  k_inverse<<<K, big ? PP_GLOBAL_THREADS : 256, sm, st>>>(p, A, Ainv, info, big ? (unsigned char*)scratch : nullptr,
                                                           pp_stride(p));
  count_launch();
}

// Lyapunov by the eigenbasis of S; V and the two temporaries in shared memory, or (gscr set,
// large p) in this k's global scratch.
__global__ void k_lyap(int p, const double2* __restrict__ Vg, const double* __restrict__ s, const double2* __restrict__ Mg,
                       double2* __restrict__ X, unsigned char* gscr, size_t gstride) {
  const int k = blockIdx.x;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* V = reinterpret_cast<double2*>(gscr ? gscr + (size_t)k * gstride : smem_raw);
  double2* T1 = V + p * p;
  double2* T2 = T1 + p * p;
  const double2* Vk = Vg + (size_t)k * p * p;
  const double2* Mk = Mg + (size_t)k * p * p;
  const double* sk = s + (size_t)k * p;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) V[e] = Vk[e];
  __syncthreads();
  // T1 = M V
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    double2 a = make_double2(0.0, 0.0);
    for (int l = 0; l < p; ++l) a = cfma(Mk[l * p + i], V[j * p + l], a);
    T1[e] = a;
  }
  __syncthreads();
  // T2 = (V^H T1) ./ (s_i + s_j)
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    double2 a = make_double2(0.0, 0.0);
    for (int l = 0; l < p; ++l) a = cfmac(V[i * p + l], T1[j * p + l], a);
    T2[e] = cscale(a, 1.0 / (sk[i] + sk[j]));
  }
  __syncthreads();
  // T1 = T2 V^H ; X = V T1
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    double2 a = make_double2(0.0, 0.0);
    for (int l = 0; l < p; ++l) a = cfma(T2[l * p + i], cconj(V[l * p + j]), a);
    T1[e] = a;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    double2 a = make_double2(0.0, 0.0);
    for (int l = 0; l < p; ++l) a = cfma(V[l * p + i], T1[j * p + l], a);
    X[(size_t)k * p * p + e] = a;
  }
}

void dense_lyapunov(int K, int p, const double2* V, const double* s, const double2* M, double2* X, cudaStream_t st,
                    void* scratch) {
  const bool big = lyap_big(p) > PP_SMEM_MAX;
  if (big && !scratch) return;  // callers size the scratch with dense_pp_scratch
  const size_t sm = big ? 0 : lyap_big(p);
  ensure_smem((const void*)k_lyap, sm);
  k_lyap<<<K, big ? PP_GLOBAL_THREADS : 256, sm, st>>>(p, V, s, M, X, big ? (unsigned char*)scratch : nullptr,
                                                        pp_stride(p));
  count_launch();
}

// ----------------------------------------------------------------------------- elementwise
__global__ void k_axpby(size_t n, double2 a, const double2* __restrict__ x, double2 b, const double2* __restrict__ y,
                        double2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double2 r = cmul(a, x[i]);
    if (y) r = r + cmul(b, y[i]);
    out[i] = r;
  }
}
void dense_axpby(size_t n, double2 a, const double2* x, double2 b, const double2* y, double2* out, cudaStream_t st) {
  const int blocks = (int)min((size_t)2048, (n + 255) / 256);
  k_axpby<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(n, a, x, b, y, out);
  count_launch();
}

__global__ void k_herm(int p, double2* A) {
  const int k = blockIdx.x;
  double2* Ak = A + (size_t)k * p * p;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    if (i < j) {
      const double2 a = Ak[j * p + i], b = Ak[i * p + j];
      const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
      Ak[j * p + i] = h;
      Ak[i * p + j] = cconj(h);
    } else if (i == j) {
      Ak[e].y = 0.0;
    }
  }
}
void dense_herm(int K, int p, double2* A, cudaStream_t st) { k_herm<<<K, 256, 0, st>>>(p, A);
  count_launch(); }

__global__ void k_shift_diag(int p, const double2* __restrict__ A, double mu, double2* __restrict__ out) {
  const int k = blockIdx.x;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    double2 v = A[(size_t)k * p * p + e];
    if (i == j) v.x -= mu;
    out[(size_t)k * p * p + e] = v;
  }
}
void dense_shift_diag(int K, int p, const double2* A, double mu, double2* out, cudaStream_t st) {
  k_shift_diag<<<K, 256, 0, st>>>(p, A, mu, out);
  count_launch();
}

constexpr int DOT_BLOCKS_PER_K = 32;
__global__ void k_dot(int K, size_t len, const double2* __restrict__ V, const double2* __restrict__ W,
                      const double* __restrict__ wk, double* __restrict__ partials) {
  __shared__ double sh[256];
  const int k = blockIdx.y;
  const size_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const size_t b0 = blockIdx.x * chunk, b1 = min(len, b0 + chunk);
  double s = 0.0;
  const double2* v = V + (size_t)k * len;
  const double2* w = W + (size_t)k * len;
  for (size_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += v[i].x * w[i].x + v[i].y * w[i].y;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int q = blockDim.x / 2; q > 0; q >>= 1) {
    if (threadIdx.x < q) sh[threadIdx.x] += sh[threadIdx.x + q];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(size_t)k * gridDim.x + blockIdx.x] = sh[0] * (wk ? wk[k] : 1.0);
}
int dense_dot(int K, size_t len, const double2* V, const double2* W, const double* wk, double* partials,
              cudaStream_t st) {
  dim3 g(DOT_BLOCKS_PER_K, K);
  k_dot<<<g, 256, 0, st>>>(K, len, V, W, wk, partials);
  count_launch();
  return K * DOT_BLOCKS_PER_K;
}
// Sum of n partials by one CTA of 256 threads: thread t adds p[t], p[t + 256], ... in order,
// then a fixed shared-memory tree (deterministic).
__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ p, int n, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int q = blockDim.x / 2; q > 0; q >>= 1) {
    if (threadIdx.x < q) sh[threadIdx.x] += sh[threadIdx.x + q];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}
void dense_sum_partials(const double* partials, int n, double* out, cudaStream_t st) {
  k_sum_partials<<<1, 256, 0, st>>>(partials, n, out);
  count_launch();
}

__global__ void k_norms2(size_t len, const double2* __restrict__ V, double* __restrict__ out) {
  __shared__ double sh[256];
  const int k = blockIdx.x;
  const double2* v = V + (size_t)k * len;
  double s = 0.0;
  for (size_t i = threadIdx.x; i < len; i += blockDim.x) s += v[i].x * v[i].x + v[i].y * v[i].y;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int q = blockDim.x / 2; q > 0; q >>= 1) {
    if (threadIdx.x < q) sh[threadIdx.x] += sh[threadIdx.x + q];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[k] = sh[0];
}
void dense_norms2(int K, size_t len, const double2* V, double* out, cudaStream_t st) {
  k_norms2<<<K, 256, 0, st>>>(len, V, out);
  count_launch();
}

void dense_copy(double2* dst, const double2* src, size_t n, cudaStream_t st) {
  cudaMemcpyAsync(dst, src, n * sizeof(double2), cudaMemcpyDeviceToDevice, st);
}

__global__ void k_tpa(int p, int n_max, const double* __restrict__ kin, const double* __restrict__ alpha,
                      const double2* __restrict__ in, double2* __restrict__ out, bool unit_gain) {
  const int k = blockIdx.y;
  const size_t tot = (size_t)p * n_max;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n_max), g = (int)(e % n_max);
    const double a = alpha[(size_t)k * p + i];
    const double f = (unit_gain ? a : 1.0) / (kin[(size_t)k * n_max + g] + a);
    out[(size_t)k * tot + e] = cscale(in[(size_t)k * tot + e], f);
  }
}
void dense_tpa(int K, int p, int n_max, const double* kin, const double* alpha, const double2* in, double2* out,
               bool unit_gain, cudaStream_t st) {
  dim3 g(64, K);
  k_tpa<<<g, 256, 0, st>>>(p, n_max, kin, alpha, in, out, unit_gain);
  count_launch();
}

__global__ void k_kinetic_alpha(int p, int n_max, const double* __restrict__ kin, const double2* __restrict__ phi,
                                double* __restrict__ alpha) {
  __shared__ double sh[256];
  const int k = blockIdx.y, i = blockIdx.x;
  const double2* v = phi + ((size_t)k * p + i) * n_max;
  const double* kk = kin + (size_t)k * n_max;
  double s = 0.0;
  for (int g = threadIdx.x; g < n_max; g += blockDim.x) s += kk[g] * (v[g].x * v[g].x + v[g].y * v[g].y);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int q = blockDim.x / 2; q > 0; q >>= 1) {
    if (threadIdx.x < q) sh[threadIdx.x] += sh[threadIdx.x + q];
    __syncthreads();
  }
  if (threadIdx.x == 0) alpha[(size_t)k * p + i] = sh[0];
}
void dense_kinetic_alpha(int K, int p, int n_max, const double* kin, const double2* phi, double* alpha,
                         cudaStream_t st) {
  dim3 g(p, K);
  k_kinetic_alpha<<<g, 256, 0, st>>>(p, n_max, kin, phi, alpha);
  count_launch();
}

// E_kin partials: per (k, i) f w_k sum_g kin |c|^2
__global__ void k_kin_energy(int p, int n_max, const double* __restrict__ kin, const double2* __restrict__ phi,
                             const double* __restrict__ kw, double occ, double* __restrict__ partials) {
  __shared__ double sh[256];
  const int k = blockIdx.y, i = blockIdx.x;
  const double2* v = phi + ((size_t)k * p + i) * n_max;
  const double* kk = kin + (size_t)k * n_max;
  double s = 0.0;
  for (int g = threadIdx.x; g < n_max; g += blockDim.x) s += kk[g] * (v[g].x * v[g].x + v[g].y * v[g].y);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int q = blockDim.x / 2; q > 0; q >>= 1) {
    if (threadIdx.x < q) sh[threadIdx.x] += sh[threadIdx.x + q];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[(size_t)k * p + i] = occ * kw[k] * sh[0];
}
void dense_kin_energy(int K, int p, int n_max, const double* kin, const double2* phi, const double* kw, double occ,
                      double* partials, cudaStream_t st) {
  dim3 g(p, K);
  k_kin_energy<<<g, 256, 0, st>>>(p, n_max, kin, phi, kw, occ, partials);
  count_launch();
}

__global__ void k_scale_rows(int m, int n, double2* P, const double* __restrict__ d) {
  const int k = blockIdx.x;
  for (int e = threadIdx.x; e < m * n; e += blockDim.x) {
    const int j = e / m, i = e - j * m;
    P[(size_t)k * m * n + (size_t)j * m + i] = cscale(P[(size_t)k * m * n + (size_t)j * m + i], d[i]);
  }
}
void dense_scale_rows(int K, int m, int n, double2* P, const double* d, cudaStream_t st) {
  k_scale_rows<<<K, 256, 0, st>>>(m, n, P, d);
  count_launch();
}

// ----------------------------------------------------------------------------- FOM projected solves
// Shifted solves (A - s_m I) y_m = c_m, m < p, for one k per CTA; A is Hermitian q x q (FP64,
// column-major, ld lda), arithmetic in the working precision T.
//   1. Householder reduction A = Q T Q^*, Q = H_0 ... H_{q-2}, H_j = I - tau_j v_j v_j^* acting
//      on rows j+1.., chosen so that H_j^* maps column j below the diagonal onto beta_j e_1 with
//      beta_j real: T is real symmetric tridiagonal (diagonal d, off-diagonal e = beta).
//      Step j: x = tau A22 v, w = x - (tau/2) conj(v^* x) v, A22 <- A22 - v w^* - w v^*.
//   2. z_m = Q^* c_m (reflectors in order), (T - s_m I) z_m = Q^* c_m by Gaussian elimination
//      with partial pivoting (one thread per shift), y_m = Q z_m (reflectors in reverse order).
// One reduction of (16/3) q^3 flops replaces p dense factorisations of (8/3) q^3 each.  The
// packed lower triangle (column j holds rows j..q-1) stays in shared memory during the
// reduction when it fits, else in the global work area; the reflectors are kept in the work
// area for the two transforms.  Every reduction runs in a fixed order (deterministic).
constexpr int HS_THREADS = 1024;
constexpr int HG_MAX_CTAS = 1024;  // CTAs per k of the grid-wide variant (partial-sum slots)

__host__ __device__ __forceinline__ size_t poff(int j, int q) {  // start of packed column j
  return (size_t)j * q - (size_t)j * (j - 1) / 2;
}
// Offset and size of the large-q region of the shifted solve's work area (tau, d, e, v, w).
__host__ __device__ __forceinline__ size_t hs_extra_off(int p, int q, size_t es, size_t ts) {
  const size_t b = poff(q, q) * es + (size_t)q * p * es + (size_t)3 * p * q * ts;
  return (b + 255) & ~(size_t)255;
}
__host__ __device__ __forceinline__ size_t hs_extra_size(int q, size_t es, size_t ts) {
  return (size_t)q * es + (size_t)(2 * q + 2) * ts + 16 + (size_t)2 * q * es + HG_MAX_CTAS * es + 64;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Sum over the CTA of one value per thread in a fixed order (a shuffle tree per warp, then one
// over the warp sums); every thread gets the result.
template <typename V>
__device__ __forceinline__ V block_sum(V v, V* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    V t = threadIdx.x < nw ? red[threadIdx.x] : V{};
    t = warp_sum(t);
    if (threadIdx.x == 0) red[32] = t;
  }
  __syncthreads();
  const V r = red[32];
  __syncthreads();
  return r;
}

template <typename T>
__global__ void __launch_bounds__(HS_THREADS)
    k_hshift(int p, int q, const double2* __restrict__ A, int lda, size_t sA, const double* __restrict__ sh,
             const double2* __restrict__ C, int ldc, size_t sC, double2* __restrict__ Y, unsigned char* work,
             size_t work_stride, const int* __restrict__ kactive, int* __restrict__ info, int pack_in_smem,
             int z_in_smem, int small_in_smem) {
  using V = cplx<T>;
  const int k = blockIdx.x;
  if (kactive && !kactive[k]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* red = reinterpret_cast<V*>(smem_raw);  // [34]
  unsigned char* sbase = reinterpret_cast<unsigned char*>(red + 34);
  // work area of this k: packed reflectors, then z (q x p), then the bands (3 q per shift), then
  // (large q) tau, d, e, v and w
  unsigned char* wk = work + (size_t)k * work_stride;
  V* Pg = reinterpret_cast<V*>(wk);
  V* Zg = Pg + poff(q, q);
  T* Bg = reinterpret_cast<T*>(Zg + (size_t)q * p);
  unsigned char* xg = wk + hs_extra_off(p, q, sizeof(V), sizeof(T));
  // tau, the tridiagonal (d, e) and v, w in shared memory, or all in the work area for large q
  V* tau = reinterpret_cast<V*>(small_in_smem ? sbase : xg);
  T* dg = reinterpret_cast<T*>(tau + q);
  T* eg = dg + q;
  unsigned char* after = reinterpret_cast<unsigned char*>(eg + q + 2);
  after = reinterpret_cast<unsigned char*>(((uintptr_t)after + 15) & ~(uintptr_t)15);
  unsigned char* area = small_in_smem ? after : sbase;  // the rest of shared memory
  // phase-1 layout of the area: packed matrix (if in shared memory), v, w
  V* P = pack_in_smem ? reinterpret_cast<V*>(area) : Pg;
  V* vv = pack_in_smem ? P + poff(q, q) : reinterpret_cast<V*>(after);
  V* xv = vv + q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const double2* Ak = A + k * sA;
  for (int j = 0; j < q; ++j)
    for (int i = j + tid; i < q; i += blockDim.x) P[poff(j, q) + (i - j)] = to_c<T>(Ak[(size_t)j * lda + i]);
  __syncthreads();
  V zero;
  zero.x = 0;
  zero.y = 0;
  // ---- 1. reduction to tridiagonal form.  Four CTA barriers per column: every thread forms
  // the reflector from the same shared values; v^* x is summed per warp during the product
  // x = tau A22 v; w = x + a2 v is formed inside the rank-2 update; warp 0 updates the next
  // column first and sums its squared tail for the next reflector.
  __shared__ T s_ss;
  {
    V part = zero;
    for (int i = 2 + tid; i < q; i += blockDim.x) {
      const V x = P[i];  // column 0: P(i, 0) = P[i]
      part.x += x.x * x.x + x.y * x.y;
    }
    const T ss0 = block_sum(part, red).x;
    if (tid == 0) s_ss = ss0;
    __syncthreads();
  }
  for (int j = 0; j + 1 < q; ++j) {
    const size_t cj = poff(j, q) - j;  // P(i, j) = P[cj + i]
    const T ss = s_ss;
    const V alpha = P[cj + j + 1];
    V t = zero, scale = mk<V>((T)1, (T)0);
    T beta = alpha.x;
    if (ss > (T)0 || alpha.y != (T)0) {
      beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + ss), alpha.x);
      t.x = (beta - alpha.x) / beta;
      t.y = -alpha.y / beta;
      const V am = mk<V>(alpha.x - beta, alpha.y);  // scale = 1 / (alpha - beta)
      const T den = am.x * am.x + am.y * am.y;
      scale = mk<V>(am.x / den, -am.y / den);
    }
    if (tid == 0) {
      tau[j] = t;
      eg[j] = beta;
      dg[j] = P[cj + j].x;
    }
    for (int i = j + 1 + tid; i < q; i += blockDim.x) {
      const V v = (i == j + 1) ? mk<V>((T)1, (T)0) : cmul(P[cj + i], scale);
      vv[i] = v;
      P[cj + i] = v;
    }
    __syncthreads();
    if (t.x == (T)0 && t.y == (T)0) {
      // no reflection: the next column's tail norm by a CTA sum
      V part = zero;
      const size_t cn = poff(j + 1, q) - (j + 1);
      for (int i = j + 3 + tid; i < q; i += blockDim.x) {
        const V x = P[cn + i];
        part.x += x.x * x.x + x.y * x.y;
      }
      const T nss = block_sum(part, red).x;
      if (tid == 0) s_ss = nss;
      __syncthreads();
      continue;
    }
    // x = tau A22 v, warp per row i (lower part along the row, upper part down column i), and
    // the warp's share of v^* x
    V dpart = zero;
    for (int i = j + 1 + warp; i < q; i += nw) {
      const size_t ci = poff(i, q) - i;
      V acc = zero;
      for (int l = j + 1 + lane; l <= i; l += 32) acc = acc + cmul(P[poff(l, q) + (i - l)], vv[l]);
      for (int l = i + 1 + lane; l < q; l += 32) acc = acc + cmulc(P[ci + l], vv[l]);
      acc = warp_sum(acc);
      const V xi = cmul(t, acc);
      if (lane == 0) xv[i] = xi;
      dpart = dpart + cmulc(vv[i], xi);
    }
    if (lane == 0) red[warp] = dpart;
    __syncthreads();
    if (warp == 0) {
      V d = lane < nw ? red[lane] : zero;
      d = warp_sum(d);
      if (lane == 0) red[32] = d;
    }
    __syncthreads();
    // a2 = -(tau / 2) conj(v^* x); A22 -= v w^* + w v^* with w = x + a2 v, warp per column, lanes
    // down the rows; warp 0 takes column j + 1 first and sums the next reflector's tail norm
    const V a2 = cscale(cmul(t, cconj(red[32])), (T)-0.5);
    for (int l = j + 1 + warp; l < q; l += nw) {
      const size_t cl = poff(l, q) - l;
      const V vl = vv[l], wl = xv[l] + cmul(a2, vl);
      V tail = zero;
      for (int i = l + lane; i < q; i += 32) {
        const V vi = vv[i], wi = xv[i] + cmul(a2, vi);
        const V d = cmul(vi, cconj(wl)) + cmul(wi, cconj(vl));
        const V nv = P[cl + i] - d;
        P[cl + i] = nv;
        if (l == j + 1 && i >= j + 3) tail.x += nv.x * nv.x + nv.y * nv.y;
      }
      if (l == j + 1) {
        tail = warp_sum(tail);
        if (lane == 0) s_ss = tail.x;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    dg[q - 1] = P[poff(q - 1, q)].x;
    eg[q - 1] = 0;
  }
  if (pack_in_smem)
    for (size_t e = tid; e < poff(q, q); e += blockDim.x) Pg[e] = P[e];
  __syncthreads();
  // ---- 2. z = Q^* c per shift (warp per shift, reflectors from the work area)
  V* Z = z_in_smem ? reinterpret_cast<V*>(area) : Zg;
  T* Bd = z_in_smem ? reinterpret_cast<T*>(Z + (size_t)q * p) : Bg;
  for (int e = tid; e < q * p; e += blockDim.x) {
    const int m = e / q, i = e - m * q;
    Z[e] = to_c<T>(C[k * sC + (size_t)m * ldc + i]);
  }
  __syncthreads();
  for (int m = warp; m < p; m += nw) {
    V* z = Z + (size_t)m * q;
    for (int j = 0; j + 1 < q; ++j) {
      const V tj = tau[j];
      if (tj.x == (T)0 && tj.y == (T)0) continue;
      const V* v = Pg + poff(j, q) - j;
      V acc = zero;
      for (int i = j + 1 + lane; i < q; i += 32) acc = acc + cmulc(v[i], z[i]);
      const V f = cmul(cconj(tj), warp_sum(acc));
      __syncwarp();
      for (int i = j + 1 + lane; i < q; i += 32) z[i] = z[i] - cmul(v[i], f);
      __syncwarp();
    }
  }
  __syncthreads();
  // ---- 3. (T - s_m I) z = z by Gaussian elimination with partial pivoting, thread per shift
  for (int m = tid; m < p; m += blockDim.x) {
    V* b = Z + (size_t)m * q;
    T* dd = Bd + (size_t)m * 3 * q;
    T* du = dd + q;
    T* du2 = du + q;
    const T sm = (T)sh[(size_t)k * p + m];
    for (int i = 0; i < q; ++i) {
      dd[i] = dg[i] - sm;
      du[i] = eg[i];
      du2[i] = 0;
    }
    int bad = 0;
    for (int i = 0; i + 1 < q; ++i) {
      const T sub = eg[i];
      if (fabs(dd[i]) >= fabs(sub)) {
        if (dd[i] == (T)0) {
          bad = 1;
          continue;
        }
        const T f = sub / dd[i];
        dd[i + 1] -= f * du[i];
        b[i + 1] = b[i + 1] - cscale(b[i], f);
        du2[i] = 0;
      } else {
        const T f = dd[i] / sub;
        dd[i] = sub;
        const T tmp = dd[i + 1];
        dd[i + 1] = du[i] - f * tmp;
        if (i + 2 < q) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du2[i];
        }
        du[i] = tmp;
        const V bi = b[i];
        b[i] = b[i + 1];
        b[i + 1] = bi - cscale(b[i], f);
      }
    }
    if (dd[q - 1] == (T)0) bad = 1;
    if (bad) {
      if (info) info[k * p + m] = 1;
      for (int i = 0; i < q; ++i) b[i] = zero;
      continue;
    }
    b[q - 1] = cscale(b[q - 1], (T)1 / dd[q - 1]);
    if (q > 1) b[q - 2] = cscale(b[q - 2] - cscale(b[q - 1], du[q - 2]), (T)1 / dd[q - 2]);
    for (int i = q - 3; i >= 0; --i)
      b[i] = cscale(b[i] - cscale(b[i + 1], du[i]) - cscale(b[i + 2], du2[i]), (T)1 / dd[i]);
  }
  __syncthreads();
  // ---- 4. y = Q z (reflectors in reverse order), written in FP64
  for (int m = warp; m < p; m += nw) {
    V* z = Z + (size_t)m * q;
    for (int j = q - 2; j >= 0; --j) {
      const V tj = tau[j];
      if (tj.x == (T)0 && tj.y == (T)0) continue;
      const V* v = Pg + poff(j, q) - j;
      V acc = zero;
      for (int i = j + 1 + lane; i < q; i += 32) acc = acc + cmulc(v[i], z[i]);
      const V f = cmul(tj, warp_sum(acc));
      __syncwarp();
      for (int i = j + 1 + lane; i < q; i += 32) z[i] = z[i] - cmul(v[i], f);
      __syncwarp();
    }
    for (int i = lane; i < q; i += 32) Y[k * sC + (size_t)m * ldc + i] = to_d(z[i]);
  }
}

// ---- Grid-wide variant for large q: the same four steps with one cooperative launch of G CTAs
// per k (grid (G, K), 1024 threads each).  Step 1 keeps the packed matrix in the work area;
// per column every CTA forms the reflector v from the same values (its own shared copy), warps
// across all CTAs own rows of x = tau A22 v (each CTA's share of v^* x goes to a slot, summed
// in slot order after the barrier), then warps across all CTAs own columns of the rank-2 update;
// the warp owning column j + 1 writes the next tail norm.  Two grid barriers per column.  Steps
// 2-4 give each shift to one warp of the grid (step 3 on its lane 0), so they need no barrier.
// Every sum runs in a fixed order (deterministic for a given G).
template <typename T>
__global__ void __launch_bounds__(HS_THREADS)
    k_hshift_grid(int p, int q, const double2* __restrict__ A, int lda, size_t sA, const double* __restrict__ sh,
                  const double2* __restrict__ C, int ldc, size_t sC, double2* __restrict__ Y, unsigned char* work,
                  size_t work_stride, const int* __restrict__ kactive, int* __restrict__ info) {
  using V = cplx<T>;
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int k = blockIdx.y, cta = blockIdx.x, G = gridDim.x;
  const bool act = !kactive || kactive[k];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* vs = reinterpret_cast<V*>(smem_raw);  // [q] reflector of the current column
  V* xs = vs + q;                          // [q] x of the current column
  V* red = xs + q;                         // [34]
  unsigned char* wk = work + (size_t)k * work_stride;
  V* Pg = reinterpret_cast<V*>(wk);
  V* Zg = Pg + poff(q, q);
  T* Bg = reinterpret_cast<T*>(Zg + (size_t)q * p);
  unsigned char* xg = wk + hs_extra_off(p, q, sizeof(V), sizeof(T));
  V* tau = reinterpret_cast<V*>(xg);
  T* dg = reinterpret_cast<T*>(tau + q);
  T* eg = dg + q;
  unsigned char* after = reinterpret_cast<unsigned char*>(eg + q + 2);
  after = reinterpret_cast<unsigned char*>(((uintptr_t)after + 15) & ~(uintptr_t)15);
  V* xv = reinterpret_cast<V*>(after) + q;  // x of the current column, shared by the grid
  V* part = xv + q;                         // [HG_MAX_CTAS] per-CTA shares of v^* x
  T* ssg = reinterpret_cast<T*>(part + HG_MAX_CTAS);  // squared tail norm of the next column
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int gw = cta * nw + warp, GW = G * nw;  // this warp within the k's grid, and the count
  V zero;
  zero.x = 0;
  zero.y = 0;
  if (act) {
    const double2* Ak = A + k * sA;
    for (int j = cta; j < q; j += G)
      for (int i = j + tid; i < q; i += blockDim.x) Pg[poff(j, q) + (i - j)] = to_c<T>(Ak[(size_t)j * lda + i]);
    if (cta == G - 1) {  // tail norm of column 0 (rows 2..), read back after the barrier
      V prt = zero;
      for (int i = 2 + tid; i < q; i += blockDim.x) {
        const double2 a = Ak[i];
        const V x = to_c<T>(a);
        prt.x += x.x * x.x + x.y * x.y;
      }
      const T s0 = block_sum(prt, red).x;
      if (tid == 0) *ssg = s0;
    }
  }
  grid.sync();
  for (int j = 0; j + 1 < q; ++j) {
    const size_t cj = poff(j, q) - j;  // P(i, j) = Pg[cj + i]
    V t = zero;
    if (act) {
      const T ss = *ssg;
      const V alpha = Pg[cj + j + 1];
      V scale = mk<V>((T)1, (T)0);
      T beta = alpha.x;
      if (ss > (T)0 || alpha.y != (T)0) {
        beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + ss), alpha.x);
        t.x = (beta - alpha.x) / beta;
        t.y = -alpha.y / beta;
        const V am = mk<V>(alpha.x - beta, alpha.y);
        const T den = am.x * am.x + am.y * am.y;
        scale = mk<V>(am.x / den, -am.y / den);
      }
      if (cta == 0 && tid == 0) {
        tau[j] = t;
        eg[j] = beta;
        dg[j] = Pg[cj + j].x;
      }
      for (int i = j + 1 + tid; i < q; i += blockDim.x) vs[i] = (i == j + 1) ? mk<V>((T)1, (T)0) : cmul(Pg[cj + i], scale);
      __syncthreads();
      if (t.x != (T)0 || t.y != (T)0) {
        V dpart = zero;
        for (int i = j + 1 + gw; i < q; i += GW) {
          const size_t ci = poff(i, q) - i;
          V acc = zero;
          for (int l = j + 1 + lane; l <= i; l += 32) acc = acc + cmul(Pg[poff(l, q) + (i - l)], vs[l]);
          for (int l = i + 1 + lane; l < q; l += 32) acc = acc + cmulc(Pg[ci + l], vs[l]);
          acc = warp_sum(acc);
          const V xi = cmul(t, acc);
          if (lane == 0) xv[i] = xi;
          dpart = dpart + cmulc(vs[i], xi);
        }
        const V dsum = block_sum(dpart, red);  // lanes of a warp hold the same dpart: scale below
        if (tid == 0) part[cta] = cscale(dsum, (T)1 / (T)32);
      }
    }
    grid.sync();  // x and the shares of v^* x are complete; every CTA has read column j
    if (act) {
      if (t.x != (T)0 || t.y != (T)0) {
        if (warp == 0) {
          V d = zero;
          for (int c = lane; c < G; c += 32) d = d + part[c];
          d = warp_sum(d);
          if (lane == 0) red[32] = d;
        }
        for (int i = j + 1 + tid; i < q; i += blockDim.x) xs[i] = xv[i];
        __syncthreads();
        const V a2 = cscale(cmul(t, cconj(red[32])), (T)-0.5);
        for (int l = j + 1 + gw; l < q; l += GW) {
          const size_t cl = poff(l, q) - l;
          const V vl = vs[l], wl = xs[l] + cmul(a2, vl);
          V tail = zero;
          for (int i = l + lane; i < q; i += 32) {
            const V vi = vs[i], wi = xs[i] + cmul(a2, vi);
            const V d = cmul(vi, cconj(wl)) + cmul(wi, cconj(vl));
            const V nv = Pg[cl + i] - d;
            Pg[cl + i] = nv;
            if (l == j + 1 && i >= j + 3) tail.x += nv.x * nv.x + nv.y * nv.y;
          }
          if (l == j + 1) {
            tail = warp_sum(tail);
            if (lane == 0) *ssg = tail.x;
          }
        }
      } else if (cta == 0) {  // no reflection: the next column's tail norm
        V prt = zero;
        const size_t cn = poff(j + 1, q) - (j + 1);
        for (int i = j + 3 + tid; i < q; i += blockDim.x) {
          const V x = Pg[cn + i];
          prt.x += x.x * x.x + x.y * x.y;
        }
        const T nss = block_sum(prt, red).x;
        if (tid == 0) *ssg = nss;
      }
      if (cta == 0)  // the reflector replaces column j (all CTAs read it before the barrier)
        for (int i = j + 1 + tid; i < q; i += blockDim.x) Pg[cj + i] = vs[i];
    }
    grid.sync();  // the updated trailing matrix and the next tail norm are complete
  }
  if (act && cta == 0 && tid == 0) {
    dg[q - 1] = Pg[poff(q - 1, q)].x;
    eg[q - 1] = 0;
  }
  grid.sync();
  if (!act) return;
  // ---- 2.-4. one warp of the grid per shift: z = Q^* c, (T - s_m I) z = z, y = Q z
  for (int m = gw; m < p; m += GW) {
    V* z = Zg + (size_t)m * q;
    for (int i = lane; i < q; i += 32) z[i] = to_c<T>(C[k * sC + (size_t)m * ldc + i]);
    __syncwarp();
    for (int j = 0; j + 1 < q; ++j) {
      const V tj = tau[j];
      if (tj.x == (T)0 && tj.y == (T)0) continue;
      const V* v = Pg + poff(j, q) - j;
      V acc = zero;
      for (int i = j + 1 + lane; i < q; i += 32) acc = acc + cmulc(v[i], z[i]);
      const V f = cmul(cconj(tj), warp_sum(acc));
      __syncwarp();
      for (int i = j + 1 + lane; i < q; i += 32) z[i] = z[i] - cmul(v[i], f);
      __syncwarp();
    }
    if (lane == 0) {
      T* dd = Bg + (size_t)m * 3 * q;
      T* du = dd + q;
      T* du2 = du + q;
      const T smv = (T)sh[(size_t)k * p + m];
      for (int i = 0; i < q; ++i) {
        dd[i] = dg[i] - smv;
        du[i] = eg[i];
        du2[i] = 0;
      }
      int bad = 0;
      for (int i = 0; i + 1 < q; ++i) {
        const T sub = eg[i];
        if (fabs(dd[i]) >= fabs(sub)) {
          if (dd[i] == (T)0) {
            bad = 1;
            continue;
          }
          const T f = sub / dd[i];
          dd[i + 1] -= f * du[i];
          z[i + 1] = z[i + 1] - cscale(z[i], f);
          du2[i] = 0;
        } else {
          const T f = dd[i] / sub;
          dd[i] = sub;
          const T tmp = dd[i + 1];
          dd[i + 1] = du[i] - f * tmp;
          if (i + 2 < q) {
            du2[i] = du[i + 1];
            du[i + 1] = -f * du2[i];
          }
          du[i] = tmp;
          const V bi = z[i];
          z[i] = z[i + 1];
          z[i + 1] = bi - cscale(z[i], f);
        }
      }
      if (dd[q - 1] == (T)0) bad = 1;
      if (bad) {
        if (info) info[k * p + m] = 1;
        for (int i = 0; i < q; ++i) z[i] = zero;
      } else {
        z[q - 1] = cscale(z[q - 1], (T)1 / dd[q - 1]);
        if (q > 1) z[q - 2] = cscale(z[q - 2] - cscale(z[q - 1], du[q - 2]), (T)1 / dd[q - 2]);
        for (int i = q - 3; i >= 0; --i)
          z[i] = cscale(z[i] - cscale(z[i + 1], du[i]) - cscale(z[i + 2], du2[i]), (T)1 / dd[i]);
      }
    }
    __syncwarp();
    for (int j = q - 2; j >= 0; --j) {
      const V tj = tau[j];
      if (tj.x == (T)0 && tj.y == (T)0) continue;
      const V* v = Pg + poff(j, q) - j;
      V acc = zero;
      for (int i = j + 1 + lane; i < q; i += 32) acc = acc + cmulc(v[i], z[i]);
      const V f = cmul(tj, warp_sum(acc));
      __syncwarp();
      for (int i = j + 1 + lane; i < q; i += 32) z[i] = z[i] - cmul(v[i], f);
      __syncwarp();
    }
    for (int i = lane; i < q; i += 32) Y[k * sC + (size_t)m * ldc + i] = to_d(z[i]);
  }
}

// Work bytes per k of the shifted solve.
static size_t hs_work_stride(int p, int q, size_t es, size_t ts) {
  const size_t b = hs_extra_off(p, q, es, ts) + hs_extra_size(q, es, ts);
  return (b + 255) & ~(size_t)255;
}

size_t fom_shifted_work(int K, int p, int q, int prec) {
  const size_t es = prec ? sizeof(float2) : sizeof(double2), ts = prec ? sizeof(float) : sizeof(double);
  return (size_t)K * hs_work_stride(p, q, es, ts);
}

template <typename T>
static void hshift_launch(int K, int p, int q, const double2* A, int lda, size_t sA, const double* s,
                          const double2* C, int ldc, size_t sC, double2* Y, void* work, const int* kactive,
                          int* info, cudaStream_t st) {
  using V = cplx<T>;
  constexpr size_t LIMIT = 227 * 1024;
  constexpr int HG_MIN_Q = 1536;  // below this the one-CTA kernel is faster than grid barriers
  const size_t gsm = (2 * (size_t)q + 34) * sizeof(V);
  if (q >= HG_MIN_Q && gsm <= LIMIT) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    int dev = 0, sms = 0, coop = 0, per = 0;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess) {
      ensure_smem((const void*)k_hshift_grid<T>, gsm);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_hshift_grid<T>, HS_THREADS, gsm) != cudaSuccess) {
        cudaGetLastError();
        per = 0;
      }
      const int G = std::min(std::min(HG_MAX_CTAS, per * sms / std::max(K, 1)), std::max(1, q / 32));
      if (cs == cudaStreamCaptureStatusNone && coop && G >= 2) {
        int p_ = p, q_ = q, lda_ = lda, ldc_ = ldc;
        size_t sA_ = sA, sC_ = sC, stride = hs_work_stride(p, q, sizeof(V), sizeof(T));
        const double2* A_ = A;
        const double* s_ = s;
        const double2* C_ = C;
        double2* Y_ = Y;
        unsigned char* w_ = (unsigned char*)work;
        const int* ka_ = kactive;
        int* info_ = info;
        void* args[] = {&p_, &q_, &A_, &lda_, &sA_, &s_, &C_, &ldc_, &sC_, &Y_, &w_, &stride, &ka_, &info_};
        if (cudaLaunchCooperativeKernel((const void*)k_hshift_grid<T>, dim3(G, K), dim3(HS_THREADS), args, gsm, st) ==
            cudaSuccess) {
          count_launch();
          return;
        }
        cudaGetLastError();  // launch refused (e.g. too few resident CTAs): the one-CTA kernel below
      }
    }
  }
  const size_t red = 34 * sizeof(V);
  const size_t small = (size_t)q * sizeof(V) + (size_t)(2 * q + 2) * sizeof(T) + 16;  // tau, d, e
  const size_t pack = poff(q, q) * sizeof(V) + 2 * (size_t)q * sizeof(V);
  const size_t vecs = 2 * (size_t)q * sizeof(V);
  const size_t zb = (size_t)q * p * sizeof(V) + (size_t)3 * p * q * sizeof(T);
  const int small_in = red + small + vecs <= LIMIT;
  const size_t persist = red + (small_in ? small : 0);
  const int pack_in = small_in && persist + pack <= LIMIT;
  const int z_in = persist + zb <= LIMIT;
  const size_t sm = persist + std::max(pack_in ? pack : (small_in ? vecs : 0), z_in ? zb : (size_t)0);
  ensure_smem((const void*)k_hshift<T>, sm);
  k_hshift<T><<<K, HS_THREADS, sm, st>>>(p, q, A, lda, sA, s, C, ldc, sC, Y, (unsigned char*)work,
                                         hs_work_stride(p, q, sizeof(V), sizeof(T)), kactive, info, pack_in, z_in,
                                         small_in);
  count_launch();
}

void fom_shifted_solve(int K, int p, int q, const double2* A, int lda, size_t sA, const double* s, const double2* C,
                       int ldc, size_t sC, double2* Y, void* work, const int* kactive, int* info, int prec,
                       cudaStream_t st) {
  if (q <= 0) return;
  if (prec)
    hshift_launch<float>(K, p, q, A, lda, sA, s, C, ldc, sC, Y, work, kactive, info, st);
  else
    hshift_launch<double>(K, p, q, A, lda, sA, s, C, ldc, sC, Y, work, kactive, info, st);
}

__global__ void k_mirror(int q0, int p, double2* A, int lda, size_t sA, const int* __restrict__ kactive) {
  const int k = blockIdx.x;
  if (kactive && !kactive[k]) return;
  double2* Ak = A + k * sA;
  for (int e = threadIdx.x; e < q0 * p; e += blockDim.x) {
    const int jj = e / q0, i = e - jj * q0;  // element (i, q0 + jj) of the upper block
    Ak[(size_t)i * lda + q0 + jj] = cconj(Ak[(size_t)(q0 + jj) * lda + i]);
  }
}
void fom_mirror(int K, int q0, int p, double2* A, int lda, size_t sA, const int* kactive, cudaStream_t st) {
  if (q0 > 0) {
    k_mirror<<<K, 256, 0, st>>>(q0, p, A, lda, sA, kactive);
  count_launch();
  }
}

// Diagonal of the rows that belong to dropped (zero) Krylov columns: those rows and columns of
// A and of the projected right-hand side are zero, so any diagonal value d other than every
// shift gives them y = 0.  d = 1 + max_m |s_m| keeps A - s_m I nonsingular there and of the
// scale of the shifts (a huge d would overflow the FP32 Householder norms).
__global__ void k_pad_diag(int q0, int p, double2* A, int lda, size_t sA, const int* __restrict__ nzero,
                           const double* __restrict__ shifts) {
  const int k = blockIdx.x;
  double2* Ak = A + k * sA;
  const int nz = nzero[k];
  double d = 0.0;
  for (int m = 0; m < p; ++m) d = fmax(d, fabs(shifts[(size_t)k * p + m]));
  d += 1.0;
  for (int i = threadIdx.x; i < nz && i < p; i += blockDim.x) Ak[(size_t)(q0 + i) * lda + q0 + i] = make_double2(d, 0.0);
}
void fom_pad_diag(int K, int q0, int p, double2* A, int lda, size_t sA, const int* nzero, const double* shifts,
                  cudaStream_t st) {
  k_pad_diag<<<K, 64, 0, st>>>(q0, p, A, lda, sA, nzero, shifts);
  count_launch();
}

// ----------------------------------------------------------------------------- small helpers
// Rank-revealing orthonormalisation factor of a block from its Gram matrix G = R^* R (p x p,
// FP64, one CTA per k): Cholesky with diagonal pivoting, i.e. QR with column pivoting of R
// written on G.  Step j takes the largest remaining Schur-complement diagonal (first position
// on ties) and stops when it is not above tol * ref[k] (ref null: the largest diagonal of G).
// With r selected columns piv[0..r) and G[piv][:, piv] = L L^*, the factor M has zero columns
// 0..p-r-1 and column p-r+c = sum_a e_{piv[a]} (L^{-*})_{ac}, so R M is orthonormal on its
// last r columns; nzero[k] = p - r.
__global__ void k_pivchol(int p, const double2* __restrict__ G, const double* __restrict__ ref, double tol,
                          double2* __restrict__ M, int* __restrict__ nzero, const int* __restrict__ kactive,
                          unsigned char* gscr, size_t gstride) {
  const int k = blockIdx.x;
  if (kactive && !kactive[k]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // S, L and piv in shared memory, or (gscr set, large p) in this k's global scratch
  double2* S = reinterpret_cast<double2*>(gscr ? gscr + (size_t)k * gstride : smem_raw);  // S(i, j) = S[j * p + i]
  double2* L = S + p * p;                             // factor, then its inverse
  int* piv = reinterpret_cast<int*>(L + p * p);
  __shared__ int mstep, rsel;
  __shared__ double thr;
  const double2* Gk = G + (size_t)k * p * p;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    const double2 a = Gk[(size_t)j * p + i], b = Gk[(size_t)i * p + j];
    S[e] = make_double2(0.5 * (a.x + b.x), i == j ? 0.0 : 0.5 * (a.y - b.y));
    L[e] = make_double2(0.0, 0.0);
  }
  for (int i = threadIdx.x; i < p; i += blockDim.x) piv[i] = i;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r0 = ref ? ref[k] : 0.0;
    if (!ref)
      for (int i = 0; i < p; ++i) r0 = fmax(r0, S[i * p + i].x);
    thr = tol * r0;
    rsel = 0;
  }
  for (int j = 0; j < p; ++j) {
    if (threadIdx.x < 32) {  // the first position of the largest remaining diagonal
      double bv = -INFINITY;
      int m = p;
      for (int i = j + (int)threadIdx.x; i < p; i += 32) {
        const double v = S[i * p + i].x;
        if (v > bv) {
          bv = v;
          m = i;
        }
      }
      warp_argmax(bv, m);
      if (threadIdx.x == 0) mstep = (m < p && bv > thr) ? m : -1;
    }
    __syncthreads();
    const int m = mstep;
    if (m < 0) break;
    if (m != j) {  // symmetric swap of positions j and m in S, rows of L, piv
      for (int c = threadIdx.x; c < p; c += blockDim.x) {
        const double2 t = S[c * p + j];
        S[c * p + j] = S[c * p + m];
        S[c * p + m] = t;
      }
      __syncthreads();
      for (int c = threadIdx.x; c < p; c += blockDim.x) {
        const double2 t = S[j * p + c];
        S[j * p + c] = S[m * p + c];
        S[m * p + c] = t;
      }
      for (int c = threadIdx.x; c < j; c += blockDim.x) {
        const double2 t = L[c * p + j];
        L[c * p + j] = L[c * p + m];
        L[c * p + m] = t;
      }
      if (threadIdx.x == 0) {
        const int t = piv[j];
        piv[j] = piv[m];
        piv[m] = t;
      }
      __syncthreads();
    }
    const double ljj = sqrt(S[j * p + j].x);
    const double inv = 1.0 / ljj;
    for (int i = j + threadIdx.x; i < p; i += blockDim.x)
      L[j * p + i] = i == j ? make_double2(ljj, 0.0) : cscale(S[j * p + i], inv);
    __syncthreads();
    const int t = p - j - 1;
    for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
      const int b = j + 1 + e / t, a = j + 1 + e % t;
      S[b * p + a] = S[b * p + a] - cmul(L[j * p + a], cconj(L[j * p + b]));
    }
    if (threadIdx.x == 0) rsel = j + 1;
    __syncthreads();
  }
  __syncthreads();
  const int r = rsel;
  // X = L^{-1} (lower), column c by forward substitution, one thread per column
  double2* X = S;
  for (int c = threadIdx.x; c < r; c += blockDim.x) {
    for (int i = 0; i < r; ++i) X[c * p + i] = make_double2(0.0, 0.0);
    X[c * p + c] = make_double2(1.0 / L[c * p + c].x, 0.0);
    for (int i = c + 1; i < r; ++i) {
      double2 acc = make_double2(0.0, 0.0);
      for (int a = c; a < i; ++a) acc = acc + cmul(L[a * p + i], X[c * p + a]);
      X[c * p + i] = cscale(acc, -1.0 / L[i * p + i].x);
    }
  }
  __syncthreads();
  double2* Mk = M + (size_t)k * p * p;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) Mk[e] = make_double2(0.0, 0.0);
  __syncthreads();
  // M[piv[a]][p - r + c] = conj(X[c][a]) for a <= c
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int c = e / r, a = e - c * r;
    if (a <= c) Mk[(size_t)(p - r + c) * p + piv[a]] = cconj(X[a * p + c]);
  }
  if (threadIdx.x == 0 && nzero) nzero[k] = p - r;
}
void small_pivchol(int K, int p, const double2* G, const double* ref, double tol, double2* M, int* nzero,
                   const int* kactive, cudaStream_t st, void* scratch) {
  const bool big = pivchol_big(p) > PP_SMEM_MAX;
  if (big && !scratch) return;  // callers size the scratch with dense_pp_scratch
  const size_t sm = big ? 0 : sizeof(double2) * 2 * p * p + sizeof(int) * p;
  ensure_smem((const void*)k_pivchol, sm);
  k_pivchol<<<K, big ? PP_GLOBAL_THREADS : 128, sm, st>>>(p, G, ref, tol, M, nzero, kactive,
                                                          big ? (unsigned char*)scratch : nullptr, pp_stride(p));
  count_launch();
}

// Largest diagonal entry (real part) of K p x p matrices: the largest squared column norm
// when G is a Gram matrix.
__global__ void k_max_diag(int K, int p, const double2* __restrict__ G, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double2* Gk = G + (size_t)k * p * p;
  double m = Gk[0].x;
  for (int i = 1; i < p; ++i) m = fmax(m, Gk[(size_t)i * p + i].x);
  out[k] = m;
}
void small_max_diag(int K, int p, const double2* G, double* out, cudaStream_t st) {
  k_max_diag<<<(K + 127) / 128, 128, 0, st>>>(K, p, G, out);
  count_launch();
}

__global__ void k_put_herm_block(int p, const double2* __restrict__ src, double2* A, int lda, size_t sA, int q0) {
  const int k = blockIdx.x;
  const double2* S = src + (size_t)k * p * p;
  double2* Ak = A + k * sA;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    const double2 a = S[j * p + i], b = S[i * p + j];
    Ak[(size_t)(q0 + j) * lda + q0 + i] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  }
}
void small_put_herm_block(int K, int p, const double2* src, double2* A, int lda, size_t sA, int q0, cudaStream_t st) {
  k_put_herm_block<<<K, 256, 0, st>>>(p, src, A, lda, sA, q0);
  count_launch();
}

__global__ void k_take_y(int q, int qcap, int p, const double2* __restrict__ Y, double2* __restrict__ Yf,
                         const int* __restrict__ take) {
  const int k = blockIdx.x;
  if (!take[k]) return;
  for (int e = threadIdx.x; e < qcap * p; e += blockDim.x) {
    const int j = e / qcap, i = e - j * qcap;
    const size_t o = (size_t)k * qcap * p + (size_t)j * qcap + i;
    Yf[o] = i < q ? Y[o] : make_double2(0.0, 0.0);
  }
}
void small_take_y(int K, int q, int qcap, int p, const double2* Y, double2* Yf, const int* take, cudaStream_t st) {
  k_take_y<<<K, 256, 0, st>>>(q, qcap, p, Y, Yf, take);
  count_launch();
}


__global__ void k_conj_transpose(int p, const double2* __restrict__ A, double2* __restrict__ out) {
  const int k = blockIdx.x;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    out[(size_t)k * p * p + e] = cconj(A[(size_t)k * p * p + (size_t)i * p + j]);
  }
}
void small_conj_transpose(int K, int p, const double2* A, double2* out, cudaStream_t st) {
  k_conj_transpose<<<K, 256, 0, st>>>(p, A, out);
  count_launch();
}

__global__ void k_add_herm(int p, const double2* __restrict__ A, double sc, double2* __restrict__ out) {
  const int k = blockIdx.x;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int j = e / p, i = e - j * p;
    const double2 a = A[(size_t)k * p * p + e], b = A[(size_t)k * p * p + (size_t)i * p + j];
    out[(size_t)k * p * p + e] = make_double2(sc * (a.x + b.x), sc * (a.y - b.y));
  }
}
void small_add_herm(int K, int p, const double2* A, double s, double2* out, cudaStream_t st) {
  k_add_herm<<<K, 256, 0, st>>>(p, A, s, out);
  count_launch();
}

__global__ void k_sqrt_vals(int n, const double* __restrict__ w, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = sqrt(w[i]);
}
void small_sqrt_vals(int K, int p, const double* w, double* out, cudaStream_t st) {
  k_sqrt_vals<<<(K * p + 127) / 128, 128, 0, st>>>(K * p, w, out);
  count_launch();
}

}  // namespace eacg
