// Kernels of the pruned 3D FFT pair of the Hamiltonian and of the density, and of the
// full 3D FFT of the potential build, for one compile-time grid size N (sm_103a).
//
// The transform of one band runs as
//   x pass  over the disk columns (my, mz) of the cutoff sphere          k_xpass_inv
//   plane   per x-plane jx: z over the rows that hold columns, y over
//           every jz, potential multiply, y back, z back onto the columns k_plane_h
//   x pass  back, gathered onto the sphere (+ kinetic term)               k_xpass_fwd
// and the density replaces the last three by k_plane_rho.  Every line transform is the
// two-step register FFT of fft.cuh; lines are read from and written to their final place
// by the phase functors, so no kernel zeroes, scatters or gathers a plane separately.
//
// Layouts: psi[K][p][n_max]; tbuf[band][jx][col]; xmap[k][fx][col] (sphere index or -1);
// cmapy[l][N + 1] (column of (ylist[l], fz) or -1); rowmask[fy] (1 if row fy holds columns);
// real-space grids [jx][jy][jz].
#pragma once
#include "common.cuh"
#include "fft.cuh"
#include "kernels.h"

namespace eacg {

constexpr int XPASS_THREADS = 256;  // x-pass CTA: 256 / N2 columns of one band

// The segment (system) that grid row y of a multi-system launch belongs to.
__device__ __forceinline__ int seg_of(const GridSegs& t, int y) {
  int i = 0;
  while (i + 1 < t.n && y >= t.s[i + 1].y0) ++i;
  return i;
}

// Inverse x pass: sphere coefficients gathered straight into the step-1 registers; the
// transformed columns are written to tbuf[band][jx][col] (coalesced over columns).
template <typename T, int N, int PV, typename TIO>
__global__ void __launch_bounds__(XPASS_THREADS) k_xpass_inv(const __grid_constant__ GridSegs tab) {
  using V = cplx<T>;
  constexpr int N2 = LinePlan<N, PV>::N2;
  __shared__ V tw[N];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* A = reinterpret_cast<V*>(smem_raw);
  const GridSeg& S = tab.s[seg_of(tab, blockIdx.y)];
  const int band = blockIdx.y - S.y0, k = band / S.p;
  const int ncols = S.ncols;
  const int cpc = blockDim.x / N2;
  const int c0 = blockIdx.x * cpc;
  if (c0 >= ncols || (S.kactive && !S.kactive[k])) return;
  const int nc = min(cpc, ncols - c0);
  const V* tw_g = static_cast<const V*>(S.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  __syncthreads();
  const int* xm = S.xmap + (size_t)k * N * ncols + c0;
  const TIO* src = static_cast<const TIO*>(S.in) + (size_t)band * S.n_max;
  V* dst = static_cast<V*>(S.tbuf) + (size_t)band * N * ncols + c0;
  fft_phase<N, PV, true, false>(
      nc, tw, PitchedScratch<V>{A, N + 1},
      [&](int l, int fx) {
        const int id = xm[(size_t)fx * ncols + l];
        return id >= 0 ? cvt<V>(src[id]) : czero<V>();
      },
      [&](int l, int jx, V x, int) { dst[(size_t)jx * ncols + l] = x; });
}

// Forward x pass and gather: out = scale * FFT + kin * in (kin may be null); the padding
// beyond n_k is zeroed.
template <typename T, int N, int PV, typename TIO>
__global__ void __launch_bounds__(XPASS_THREADS) k_xpass_fwd(const __grid_constant__ GridSegs tab) {
  using V = cplx<T>;
  constexpr int N2 = LinePlan<N, PV>::N2;
  __shared__ V tw[N];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* A = reinterpret_cast<V*>(smem_raw);
  const GridSeg& S = tab.s[seg_of(tab, blockIdx.y)];
  const int band = blockIdx.y - S.y0, k = band / S.p;
  const int ncols = S.ncols, n_max = S.n_max;
  const int cpc = blockDim.x / N2;
  const int c0 = blockIdx.x * cpc;
  if (c0 >= ncols || (S.kactive && !S.kactive[k])) return;
  const int nc = min(cpc, ncols - c0);
  const V* tw_g = static_cast<const V*>(S.tw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  __syncthreads();
  const int* xm = S.xmap + (size_t)k * N * ncols + c0;
  const V* src = static_cast<const V*>(S.tbuf) + (size_t)band * N * ncols + c0;
  TIO* o = static_cast<TIO*>(S.out) + (size_t)band * n_max;
  const TIO* pin = static_cast<const TIO*>(S.in) + (size_t)band * n_max;
  const double* kk = S.kin ? S.kin + (size_t)k * n_max : nullptr;
  const double scale = S.scale;
  fft_phase<N, PV, false, false>(
      nc, tw, PitchedScratch<V>{A, N + 1}, [&](int l, int jx) { return src[(size_t)jx * ncols + l]; },
      [&](int l, int fx, V x, int) {
        const int id = xm[(size_t)fx * ncols + l];
        if (id >= 0) {
          double2 v = cscale(to_d(x), scale);
          if (kk) {
            const double2 s = to_d(pin[id]);
            v.x += kk[id] * s.x;
            v.y += kk[id] * s.y;
          }
          o[id] = cvt<TIO>(v);
        }
      });
  if (blockIdx.x == 0) {
    for (int i = S.nk[k] + threadIdx.x; i < n_max; i += blockDim.x) o[i] = cvt<TIO>(make_double2(0.0, 0.0));
  }
}

// Shared set-up of the plane kernels: twiddles, row mask, row list and the column map of
// the rows with columns, copied once per CTA.
template <typename V, int N>
__device__ __forceinline__ void plane_setup(V* tw, int* rows, int* yl, int* cm, const V* tw_g,
                                            const int* rowmask, const int* ylist, const int* cmapy, int ny) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = tw_g[i];
    rows[i] = rowmask[i];
  }
  for (int i = threadIdx.x; i < ny; i += blockDim.x) yl[i] = ylist[i];
  for (int i = threadIdx.x; i < ny * (N + 1); i += blockDim.x) cm[i] = cmapy[i];
  __syncthreads();
}

// Plane buffers: B = the plane [jy][jz] (pitch N + 1) and, where two planes fit in shared
// memory, A = step-1 scratch (ping-pong: one barrier per step).  Otherwise the step-1
// values stay in B in place and the phases that store into B add a barrier.
// Double-float transforms are latency-bound (long dependent chains of error-free operations):
// they keep two planes only where four CTAs still fit an SM (N <= 41), and otherwise work in
// place with twice the CTAs per SM.
template <typename T, int N>
struct PlaneCfg {
  static constexpr bool pingpong = std::is_same<T, dfloat>::value
                                       ? 2 * sizeof(cplx<T>) * N * (N + 1) <= 56 * 1024
                                       : 2 * sizeof(cplx<T>) * N * (N + 1) <= 200 * 1024;
  static size_t smem_bytes(int ny) {
    return (pingpong ? 2 : 1) * sizeof(cplx<T>) * (size_t)N * (N + 1) + sizeof(int) * (size_t)ny * (N + 1);
  }
};

// Step-1 scratch of the z phases (line l = row ylist[l]) and of the y phases (line = jz).
template <typename V, int N, bool PING>
struct ZScratch {
  V* A;
  V* B;
  const int* yl;
  __device__ __forceinline__ V* operator()(int l, int pos) const {
    return PING ? A + (size_t)l * (N + 1) + pos : B + (size_t)yl[l] * (N + 1) + pos;
  }
};
template <typename V, int N, bool PING>
struct YScratch {
  V* A;
  V* B;
  __device__ __forceinline__ V* operator()(int jz, int pos) const {
    return PING ? A + (size_t)jz * (N + 1) + pos : B + (size_t)pos * (N + 1) + jz;
  }
};

// Apply the local potential to one x-plane of one band.  Only rows that hold columns are
// read before the y pass, so nothing is zeroed.
template <typename T, int N, int PV>
__global__ void __launch_bounds__(N * LinePlan<N, PV>::N2) k_plane_h(const __grid_constant__ GridSegs tab) {
  using V = cplx<T>;
  constexpr int PP = N + 1;
  constexpr bool PING = PlaneCfg<T, N>::pingpong;
  __shared__ V tw[N];
  __shared__ int rows[N], yl[N];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* B = reinterpret_cast<V*>(smem_raw);
  V* A = PING ? B + (size_t)N * PP : B;
  int* cm = reinterpret_cast<int*>(B + (size_t)(PING ? 2 : 1) * N * PP);
  const GridSeg& S = tab.s[seg_of(tab, blockIdx.y)];
  const int jx = blockIdx.x, band = blockIdx.y - S.y0;
  if (S.kactive && !S.kactive[band / S.p]) return;
  const int ny = S.ny;
  plane_setup<V, N>(tw, rows, yl, cm, static_cast<const V*>(S.tw), S.rowmask, S.ylist, S.cmapy, ny);
  V* tb = static_cast<V*>(S.tbuf) + ((size_t)band * N + jx) * S.ncols;
  const T* vv = static_cast<const T*>(S.v) + (size_t)jx * N * N;
  const ZScratch<V, N, PING> zs{A, B, yl};
  const YScratch<V, N, PING> ys{A, B};
  // z inverse over the rows with columns, straight from the column buffer
  fft_phase<N, PV, true, !PING>(
      ny, tw, zs,
      [&](int l, int fz) {
        const int c = cm[l * PP + fz];
        return c >= 0 ? tb[c] : czero<V>();
      },
      [&](int l, int jz, V x, int) { B[yl[l] * PP + jz] = x; });
  // y inverse over every jz (rows without columns are zero), times the potential
  fft_phase<N, PV, true, !PING>(
      N, tw, ys, [&](int jz, int fy) { return rows[fy] ? B[fy * PP + jz] : czero<V>(); },
      [&](int jz, int jy, V x, int) { B[jy * PP + jz] = cscale(x, vv[jy * N + jz]); });
  // y forward, keeping the rows with columns
  fft_phase<N, PV, false, !PING>(
      N, tw, ys, [&](int jz, int jy) { return B[jy * PP + jz]; },
      [&](int jz, int fy, V x, int) {
        if (rows[fy]) B[fy * PP + jz] = x;
      });
  // z forward, back onto the columns
  fft_phase<N, PV, false, false>(
      ny, tw, zs, [&](int l, int jz) { return B[yl[l] * PP + jz]; },
      [&](int l, int fz, V x, int) {
        const int c = cm[l * PP + fz];
        if (c >= 0) tb[c] = x;
      });
}

// Accumulator of the density: FP64 for FP32 and FP64 transforms, double-float for
// double-float transforms (FP64-accurate without the FP64 pipe).
template <typename T>
struct RhoAcc {
  using type = double;
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double weight(double w) { return w; }
  template <typename V>
  static __device__ __forceinline__ double add(double acc, double w, V x) {
    const double2 u = to_d(x);
    return acc + w * (u.x * u.x + u.y * u.y);
  }
  static __device__ __forceinline__ double out(double a) { return a; }
};
template <>
struct RhoAcc<dfloat> {
  using type = dfloat;
  static __device__ __forceinline__ dfloat zero() { return dfloat(0.0f, 0.0f); }
  static __device__ __forceinline__ dfloat weight(double w) { return df_from(w); }
  static __device__ __forceinline__ dfloat add(dfloat acc, dfloat w, dcomplex x) {
    return acc + w * (x.x * x.x + x.y * x.y);
  }
  static __device__ __forceinline__ double out(dfloat a) { return df_to(a); }
};

// Density of a group of bands on one x-plane: sum_b w_b |u_b|^2 accumulated per grid point
// (each point owned by one thread of the y pass, bands in a fixed order), written as FP64
// partial[g][jx][jy][jz].  Grid rows are the band groups of the segments.
template <typename T, int N, int PV>
__global__ void __launch_bounds__(N * LinePlan<N, PV>::N2) k_plane_rho(const __grid_constant__ GridSegs tab) {
  using V = cplx<T>;
  constexpr int PP = N + 1, N1 = LinePlan<N, PV>::N1, N2 = LinePlan<N, PV>::N2;
  constexpr bool PING = PlaneCfg<T, N>::pingpong;
  __shared__ V tw[N];
  __shared__ int rows[N], yl[N];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* B = reinterpret_cast<V*>(smem_raw);
  V* A = PING ? B + (size_t)N * PP : B;
  int* cm = reinterpret_cast<int*>(B + (size_t)(PING ? 2 : 1) * N * PP);
  const GridSeg& S = tab.s[seg_of(tab, blockIdx.y)];
  const int jx = blockIdx.x, g = blockIdx.y - S.y0;
  const int ny = S.ny, ncols = S.ncols, nbands = S.nbands;
  plane_setup<V, N>(tw, rows, yl, cm, static_cast<const V*>(S.tw), S.rowmask, S.ylist, S.cmapy, ny);
  const ZScratch<V, N, PING> zs{A, B, yl};
  const YScratch<V, N, PING> ys{A, B};
  using Acc = RhoAcc<T>;
  typename Acc::type acc[N1];
#pragma unroll
  for (int q = 0; q < N1; ++q) acc[q] = Acc::zero();
  const int bpg = (nbands + S.groups - 1) / S.groups;
  const int b0 = g * bpg, b1 = min(nbands, b0 + bpg);
  const V* tbuf = static_cast<const V*>(S.tbuf);
  for (int band = b0; band < b1; ++band) {
    const V* tb = tbuf + ((size_t)band * N + jx) * ncols;
    fft_phase<N, PV, true, !PING>(
        ny, tw, zs,
        [&](int l, int fz) {
          const int c = cm[l * PP + fz];
          return c >= 0 ? tb[c] : czero<V>();
        },
        [&](int l, int jz, V x, int) { B[yl[l] * PP + jz] = x; });
    const auto w = Acc::weight(S.bw[band]);
    fft_phase<N, PV, true, false>(
        N, tw, ys, [&](int jz, int fy) { return rows[fy] ? B[fy * PP + jz] : czero<V>(); },
        [&](int, int, V x, int q) { acc[q] = Acc::add(acc[q], w, x); });
  }
  // thread (jz, t) of the y pass owns jy = (t + N2 j) + N1 k2 at q = j N2 + k2
  const int L = blockDim.x / N2;
  const int jz = threadIdx.x % L, t = threadIdx.x / L;
  if (t < N2 && jz < N) {
    double* out = S.partial + ((size_t)g * N + jx) * N * N;
#pragma unroll
    for (int q = 0; q < N1; ++q) {
      const int jy = (t + N2 * (q / N2)) + N1 * (q % N2);
      out[(size_t)jy * N + jz] = Acc::out(acc[q]);
    }
  }
}

// Lines along one axis of a complex N^3 array a[x][y][z] (axis 2 = z, 1 = y, 0 = x),
// transformed in place, 256 / N2 lines per CTA.
template <int N, int PV, bool INV>
__global__ void __launch_bounds__(XPASS_THREADS)
    k_fft3_axis(double2* __restrict__ a, int axis, const double2* __restrict__ tw_g) {
  constexpr int N2 = LinePlan<N, PV>::N2;
  __shared__ double2 tw[N];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* A = reinterpret_cast<double2*>(smem_raw);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  __syncthreads();
  const int lpc = blockDim.x / N2;
  const int l0 = blockIdx.x * lpc;
  const int nl = min(lpc, N * N - l0);
  auto addr = [&](int l, int j) -> size_t {
    const int L = l0 + l, u = L / N, w = L - (L / N) * N;
    if (axis == 2) return ((size_t)u * N + w) * N + j;
    if (axis == 1) return ((size_t)u * N + j) * N + w;
    return ((size_t)j * N + u) * N + w;
  };
  fft_phase<N, PV, INV, false>(
      nl, tw, PitchedScratch<double2>{A, N + 1}, [&](int l, int j) { return a[addr(l, j)]; },
      [&](int l, int o, double2 x, int) { a[addr(l, o)] = x; });
}

template <typename T>
struct TwKind {
  static constexpr int value = std::is_same<T, float>::value ? 1 : std::is_same<T, dfloat>::value ? 2 : 0;
};

// Launchers of one grid size and line-plan variant; instantiated per supported (N, variant)
// in the grid_fft_*.cu units.  Each launch covers the requests r[0..n) (n <= GRID_MAX_SEGS).
template <int N, int PV>
struct GridFft {
  static constexpr int N2 = LinePlan<N, PV>::N2;

  // segment table of the requests; rows(i) = grid rows of request i; returns the total
  // tw_kind: 0 FP64 twiddles, 1 FP32, 2 double-float
  static int table(GridSegs& t, const GridReq* r, int n, int tw_kind, bool groups_as_rows) {
    int y = 0;
    t.n = n;
    for (int i = 0; i < n; ++i) {
      const GridCtx& g = *r[i].g;
      GridSeg& S = t.s[i];
      S.in = r[i].in;
      S.tbuf = r[i].tbuf;
      S.out = r[i].out;
      S.kin = r[i].kin;
      S.v = r[i].v;
      S.kactive = r[i].kactive;
      S.nk = g.nk;
      S.xmap = g.xmap;
      S.cmapy = g.cmapy;
      S.ylist = g.ylist;
      S.rowmask = g.rowmask;
      S.tw = tw_kind == 1 ? g.tw32 : tw_kind == 2 ? g.twdf : g.tw64;
      S.bw = r[i].bw;
      S.partial = r[i].partial;
      S.scale = r[i].scale;
      S.n_max = g.n_max;
      S.p = g.p;
      S.ncols = g.ncols;
      S.ny = g.ny;
      S.nbands = r[i].nbands;
      S.groups = r[i].groups;
      S.y0 = y;
      y += groups_as_rows ? r[i].groups : r[i].nbands;
    }
    return y;
  }
  static int max_cols(const GridReq* r, int n) {
    int c = 0;
    for (int i = 0; i < n; ++i) c = c > r[i].g->ncols ? c : r[i].g->ncols;
    return c;
  }
  static int max_ny(const GridReq* r, int n) {
    int c = 0;
    for (int i = 0; i < n; ++i) c = c > r[i].g->ny ? c : r[i].g->ny;
    return c;
  }

  template <typename T, typename TIO>
  static void xinv(const GridReq* r, int n, cudaStream_t st) {
    GridSegs t;
    const int rows = table(t, r, n, TwKind<T>::value, false);
    const int cpc = XPASS_THREADS / N2;
    dim3 grid((max_cols(r, n) + cpc - 1) / cpc, rows);
    const size_t sm = sizeof(cplx<T>) * (size_t)cpc * (N + 1);
    ensure_smem((const void*)k_xpass_inv<T, N, PV, TIO>, sm);
    k_xpass_inv<T, N, PV, TIO><<<grid, cpc * N2, sm, st>>>(t);
    count_launch();
  }

  template <typename T, typename TIO>
  static void xfwd(const GridReq* r, int n, cudaStream_t st) {
    GridSegs t;
    const int rows = table(t, r, n, TwKind<T>::value, false);
    const int cpc = XPASS_THREADS / N2;
    dim3 grid((max_cols(r, n) + cpc - 1) / cpc, rows);
    const size_t sm = sizeof(cplx<T>) * (size_t)cpc * (N + 1);
    ensure_smem((const void*)k_xpass_fwd<T, N, PV, TIO>, sm);
    k_xpass_fwd<T, N, PV, TIO><<<grid, cpc * N2, sm, st>>>(t);
    count_launch();
  }

  // mode 0: FP64 transforms of FP64 blocks; 1: FP32 transforms of FP64 blocks;
  // 2: FP32 transforms of FP32 blocks
  // mode 3: double-float transforms of FP64 blocks
  static void xpass_inv(int mode, const GridReq* r, int n, cudaStream_t st);

  static void xpass_fwd(int mode, const GridReq* r, int n, cudaStream_t st);

  template <typename T>
  static void plane_h_t(const GridReq* r, int n, cudaStream_t st) {
    GridSegs t;
    const int rows = table(t, r, n, TwKind<T>::value, false);
    const size_t sm = PlaneCfg<T, N>::smem_bytes(max_ny(r, n));
    ensure_smem((const void*)k_plane_h<T, N, PV>, sm);
    k_plane_h<T, N, PV><<<dim3(N, rows), N * N2, sm, st>>>(t);
    count_launch();
  }

  // prec 0: FP64, 1: FP32, 2: double-float
  static void plane_h(int prec, const GridReq* r, int n, cudaStream_t st);

  template <typename T>
  static void plane_rho_t(const GridReq* r, int n, cudaStream_t st) {
    GridSegs t;
    const int rows = table(t, r, n, TwKind<T>::value, true);
    const size_t sm = PlaneCfg<T, N>::smem_bytes(max_ny(r, n));
    ensure_smem((const void*)k_plane_rho<T, N, PV>, sm);
    k_plane_rho<T, N, PV><<<dim3(N, rows), N * N2, sm, st>>>(t);
    count_launch();
  }

  static void plane_rho(int prec, const GridReq* r, int n, cudaStream_t st);

  template <bool INV>
  static void fft3_axis(const GridCtx& g, double2* a, int axis, cudaStream_t st) {
    const int lpc = XPASS_THREADS / N2;
    const size_t sm = sizeof(double2) * (size_t)lpc * (N + 1);
    ensure_smem((const void*)k_fft3_axis<N, PV, INV>, sm);
    k_fft3_axis<N, PV, INV><<<(N * N + lpc - 1) / lpc, lpc * N2, sm, st>>>(a, axis, (const double2*)g.tw64);
    count_launch();
  }

  static void fft3(const GridCtx& g, double2* a, bool inverse, cudaStream_t st);
};

// Dispatchers defined outside the class, so that they are not inline: the explicit
// instantiations in the grid_fft_*.cu units are then the only ones, and other translation
// units see only their declarations (extern template).
// The FP64-accurate plane kernels hold a plane of 16-byte values in shared memory, which fits
// up to N = 96; larger grids have the FP32 transforms only (the driver refuses the others
// before any launch, so those branches are not instantiated).
template <int N>
struct Fp64Planes {
  static constexpr bool value = N <= 96;
};

template <int N, int PV>
void GridFft<N, PV>::xpass_inv(int mode, const GridReq* r, int n, cudaStream_t st) {
  if (mode == 1)
    xinv<float, double2>(r, n, st);
  else if (mode == 2)
    xinv<float, float2>(r, n, st);
  else if constexpr (Fp64Planes<N>::value) {
    if (mode == 0)
      xinv<double, double2>(r, n, st);
    else
      xinv<dfloat, double2>(r, n, st);
  }
}

template <int N, int PV>
void GridFft<N, PV>::xpass_fwd(int mode, const GridReq* r, int n, cudaStream_t st) {
  if (mode == 1)
    xfwd<float, double2>(r, n, st);
  else if (mode == 2)
    xfwd<float, float2>(r, n, st);
  else if constexpr (Fp64Planes<N>::value) {
    if (mode == 0)
      xfwd<double, double2>(r, n, st);
    else
      xfwd<dfloat, double2>(r, n, st);
  }
}

template <int N, int PV>
void GridFft<N, PV>::plane_h(int prec, const GridReq* r, int n, cudaStream_t st) {
  if (prec == 1)
    plane_h_t<float>(r, n, st);
  else if constexpr (Fp64Planes<N>::value) {
    if (prec == 0)
      plane_h_t<double>(r, n, st);
    else
      plane_h_t<dfloat>(r, n, st);
  }
}

template <int N, int PV>
void GridFft<N, PV>::plane_rho(int prec, const GridReq* r, int n, cudaStream_t st) {
  if (prec == 1)
    plane_rho_t<float>(r, n, st);
  else if constexpr (Fp64Planes<N>::value) {
    if (prec == 0)
      plane_rho_t<double>(r, n, st);
    else
      plane_rho_t<dfloat>(r, n, st);
  }
}

template <int N, int PV>
void GridFft<N, PV>::fft3(const GridCtx& g, double2* a, bool inverse, cudaStream_t st) {
  for (int axis = 2; axis >= 0; --axis) {
    if (inverse)
      fft3_axis<true>(g, a, axis, st);
    else
      fft3_axis<false>(g, a, axis, st);
  }
}

}  // namespace eacg
