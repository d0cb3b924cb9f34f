// Plane-wave grid kernels of libeacg (sm_103a): G-sphere index maps, the potential build
// (Hartree by FFT, Slater exchange, Gaussian local part), the fixed-order reduction of the
// density partials, and the dispatch of the per-grid-size FFT kernels (grid_fft.cuh, one
// instantiation unit per group of sizes).
//
// Layouts (all row-major, last index fastest):
//   coefficient blocks  psi[K][p][n_max]        complex double, zero beyond n_k
//   real-space grids    v[jx][jy][jz]            N^3
//   FFT intermediate    tbuf[band][jx][col]      band = k * p + i, col = (my, mz) disk column
#include <math.h>

#include "common.cuh"
#include "grid_fft.cuh"
#include "kernels.h"

namespace eacg {

// ----------------------------------------------------------------------------- basis
// Sphere test of one integer triple at fractional k: s = (m+k)^2 summed x, y, z in
// order with rounded products and sums (no contraction), compared with thr.
__device__ __forceinline__ bool in_sphere(int mx, int my, int mz, const double* kf, double thr) {
  double qx = __dadd_rn((double)mx, kf[0]);
  double qy = __dadd_rn((double)my, kf[1]);
  double qz = __dadd_rn((double)mz, kf[2]);
  double s = __dadd_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(qz, qz));
  return s <= thr;
}

// One CTA per k: count sphere points per (mx, my) row (canonical order), exclusive scan,
// then write the integer triples, 1/2 |k+G|^2 and the union-column marks.
__global__ void k_sphere_build(int N, const double* __restrict__ kfrac, double thr, double b, int n_max_cap,
                               int* __restrict__ nk_out, int* __restrict__ row_off /*[K][N*N+1]*/,
                               int* __restrict__ m_out /*[K][n_max_cap][3]*/, double* __restrict__ kin /*[K][n_max_cap]*/,
                               int* __restrict__ colmark /*[N*N] (my,mz) signed-index grid*/) {
  const int k = blockIdx.x;
  const double* kf = kfrac + 3 * k;
  int* off = row_off + (size_t)k * (N * N + 1);
  const int h = N / 2;
  // counts per row (mx, my) with mx slowest: row r = (mx + h) * N + (my + h)
  for (int r = threadIdx.x; r < N * N; r += blockDim.x) {
    const int mx = r / N - h, my = r % N - h;
    int c = 0;
    for (int mz = -h; mz < N - h; ++mz) c += in_sphere(mx, my, mz, kf, thr) ? 1 : 0;
    off[r + 1] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    off[0] = 0;
    for (int r = 0; r < N * N; ++r) off[r + 1] += off[r];
    nk_out[k] = off[N * N];
  }
  __syncthreads();
  const int nk = off[N * N];
  if (m_out == nullptr || nk > n_max_cap) return;  // count-only call, or the host rejects nk
  for (int r = threadIdx.x; r < N * N; r += blockDim.x) {
    const int mx = r / N - h, my = r % N - h;
    int o = off[r];
    for (int mz = -h; mz < N - h; ++mz) {
      if (in_sphere(mx, my, mz, kf, thr)) {
        int* mm = m_out + ((size_t)k * n_max_cap + o) * 3;
        mm[0] = mx;
        mm[1] = my;
        mm[2] = mz;
        const double qx = mx + kf[0], qy = my + kf[1], qz = mz + kf[2];
        kin[(size_t)k * n_max_cap + o] = 0.5 * b * b * (qx * qx + qy * qy + qz * qz);
        atomicOr(&colmark[(my + h) * N + (mz + h)], 1);
        ++o;
      }
    }
  }
}

// Single CTA: list of union columns in canonical (my, mz) order, the list of distinct fy
// rows, the row mask and the per-row column map cmapy[l][fz] (pitch N + 1).
// colidx[(my+h)*N + (mz+h)] = column number or -1.
__global__ void k_columns(int N, const int* __restrict__ colmark, int* __restrict__ colidx, int* __restrict__ cmapy,
                          int* __restrict__ rowmask, int* __restrict__ ncols_out, int* __restrict__ ylist,
                          int* __restrict__ ny_out) {
  if (threadIdx.x != 0) return;
  const int h = N / 2;
  for (int i = 0; i < N * (N + 1); ++i) cmapy[i] = -1;
  for (int i = 0; i < N; ++i) rowmask[i] = 0;
  int c = 0, ny = 0;
  for (int a = 0; a < N; ++a) {
    const int fy = ((a - h) % N + N) % N;
    bool rowhas = false;
    for (int z = 0; z < N; ++z) {
      const int r = a * N + z;
      if (colmark[r]) {
        colidx[r] = c;
        cmapy[ny * (N + 1) + ((z - h) % N + N) % N] = c;
        ++c;
        rowhas = true;
      } else {
        colidx[r] = -1;
      }
    }
    if (rowhas) {
      ylist[ny++] = fy;
      rowmask[fy] = 1;
    }
  }
  *ncols_out = c;
  *ny_out = ny;
}

// xmap[k][fx][col] = sphere index of (mx = fx signed, my, mz) at k, or -1.
__global__ void k_xmap(int N, int K, int n_max, const int* __restrict__ nk, const int* __restrict__ m,
                       const int* __restrict__ colidx, int ncols, int* __restrict__ xmap) {
  const int k = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk[k]) return;
  const int* mm = m + ((size_t)k * n_max + i) * 3;
  const int h = N / 2;
  const int c = colidx[(mm[1] + h) * N + (mm[2] + h)];
  const int fx = (mm[0] % N + N) % N;
  xmap[((size_t)k * N + fx) * ncols + c] = i;
}

__global__ void k_fill_int(int* p, size_t n, int v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void k_reduce_groups(const double* __restrict__ partial, int G, size_t n, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += partial[(size_t)g * n + i];
    out[i] = s;
  }
}

// ----------------------------------------------------------------------------- potential
// Signed frequency of FFT index f; Nyquist (-N/2) flagged.
__device__ __forceinline__ int sfreq(int f, int N, bool* nyq) {
  const int s = f < (N + 1) / 2 ? f : f - N;
  if ((N % 2 == 0) && s == -(N / 2)) *nyq = true;
  return s;
}

// Gaussian-screened local potential in reciprocal space (complex N^3, G = 0 and Nyquist zero).
__global__ void k_vloc_g(int N, double b, double omega, int natoms, const double* __restrict__ pos,
                         const double* __restrict__ Z, const double* __restrict__ rc, double2* __restrict__ out) {
  const size_t n3 = (size_t)N * N * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const int fx = (int)(i / ((size_t)N * N)), fy = (int)((i / N) % N), fz = (int)(i % N);
    bool nyq = false;
    const int mx = sfreq(fx, N, &nyq), my = sfreq(fy, N, &nyq), mz = sfreq(fz, N, &nyq);
    const double gx = b * mx, gy = b * my, gz = b * mz;
    const double g2 = gx * gx + gy * gy + gz * gz;
    double2 acc = make_double2(0.0, 0.0);
    if (!nyq && g2 > 0.0) {
      for (int a = 0; a < natoms; ++a) {
        const double amp = -4.0 * M_PI * Z[a] / (omega * g2) * exp(-g2 * rc[a] * rc[a] / 4.0);
        double s, c;
        sincos(gx * pos[3 * a] + gy * pos[3 * a + 1] + gz * pos[3 * a + 2], &s, &c);
        acc.x += amp * c;
        acc.y -= amp * s;
      }
    }
    out[i] = acc;
  }
}

// a(G) *= 4 pi / (|G|^2 N^3) (zero at G = 0 and on Nyquist planes): Poisson in reciprocal space.
__global__ void k_hartree_scale(double2* __restrict__ a, int N, double b) {
  const size_t n3 = (size_t)N * N * N;
  const double inv = 1.0 / (double)n3;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const int fx = (int)(i / ((size_t)N * N)), fy = (int)((i / N) % N), fz = (int)(i % N);
    bool nyq = false;
    const int mx = sfreq(fx, N, &nyq), my = sfreq(fy, N, &nyq), mz = sfreq(fz, N, &nyq);
    const double g2 = b * b * (double)(mx * mx + my * my + mz * mz);
    if (nyq || g2 == 0.0) {
      a[i] = make_double2(0.0, 0.0);
    } else {
      a[i] = cscale(a[i], 4.0 * M_PI / g2 * inv);
    }
  }
}

__global__ void k_real_to_complex(const double* __restrict__ r, double2* __restrict__ c, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    c[i] = make_double2(r[i], 0.0);
}
__global__ void k_complex_real_part(const double2* __restrict__ c, double* __restrict__ r, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) r[i] = c[i].x;
}

// LDA correlation of the spin-unpolarised homogeneous gas, Perdew-Wang 1992 fit (Phys. Rev. B
// 45, 13244, Eq. (10), zeta = 0 parameters of Table I): with r_s = (3 / (4 pi rho))^{1/3},
//   eps_c = -2 A (1 + alpha1 r_s) ln(1 + 1 / Q),  Q = 2 A (beta1 r_s^1/2 + beta2 r_s + beta3 r_s^3/2
//   + beta4 r_s^2);  V_c = eps_c - (r_s / 3) d eps_c / d r_s.  rho > 0; returns rho eps_c.
__device__ __forceinline__ double pw92_correlation(double rho, double* vc) {
  const double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
  const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
  const double sq = sqrt(rs);
  const double pre = -2.0 * A * (1.0 + a1 * rs);
  const double q = 2.0 * A * (sq * (b1 + b3 * rs) + rs * (b2 + b4 * rs));
  const double dq = A * (b1 / sq + 2.0 * b2 + 3.0 * b3 * sq + 4.0 * b4 * rs);
  const double lg = log1p(1.0 / q);
  const double eps = pre * lg;
  const double deps = -2.0 * A * a1 * lg - pre * dq / (q * (q + 1.0));
  *vc = eps - rs * deps / 3.0;
  return rho * eps;
}

// V_tot = V_loc + V_H + V_xc(rho) and the energy integrands (loc, hartree, xc) reduced per
// block; xc: 0 none, 1 Slater exchange, 2 Slater exchange + PW92 correlation.
__global__ void k_vtot_energy(size_t n, const double* __restrict__ vloc, const double* __restrict__ vh,
                              const double* __restrict__ rho, int hartree, int xc, double* __restrict__ vtot,
                              float* __restrict__ vtot32, float2* __restrict__ vtotdf,
                              double* __restrict__ blocksums /*[gridDim][3]*/) {
  __shared__ double sh[3][256];
  double el = 0.0, eh = 0.0, ex = 0.0;
  const double cx = -0.75 * cbrt(3.0 / M_PI);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double r = rho[i];
    const double rp = r > 0.0 ? r : 0.0;
    double v = vloc[i];
    el += vloc[i] * r;
    if (hartree) {
      v += vh[i];
      eh += 0.5 * vh[i] * r;
    }
    if (xc) {
      const double c3 = cbrt(rp);
      v -= cbrt(3.0 * rp / M_PI);
      ex += cx * rp * c3;
      if (xc == 2 && rp > 0.0) {
        double vc;
        ex += pw92_correlation(rp, &vc);
        v += vc;
      }
    }
    vtot[i] = v;
    if (vtot32) vtot32[i] = (float)v;
    if (vtotdf) {
      const dfloat d = df_from(v);  // double-float copy for the double-float transforms
      vtotdf[i] = make_float2(d.hi, d.lo);
    }
  }
  sh[0][threadIdx.x] = el;
  sh[1][threadIdx.x] = eh;
  sh[2][threadIdx.x] = ex;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) blocksums[blockIdx.x * 3 + q] = sh[q][0];
}

// Gaussian s/p projector coefficients B[k][j][n_max] (j = atom * npa + l; l = s, px, py, pz).
__global__ void k_projectors(int K, int n_max, const int* __restrict__ nk, const int* __restrict__ m,
                             const double* __restrict__ kfrac, double b, double omega, int natoms,
                             const double* __restrict__ pos, int npa, double w, double2* __restrict__ B) {
  const int k = blockIdx.y;
  const int nproj = natoms * npa;
  const size_t tot = (size_t)nproj * n_max;
  const double invs = 1.0 / sqrt(omega);
  const double fs0 = pow(2.0, 1.5) * pow(M_PI, 0.75) * pow(w, 1.5);
  const double fp0 = w * w * pow(2.0 * M_PI * w * w, 1.5) * sqrt(2.0 / (w * w)) * pow(M_PI * w * w, -0.75);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n_max), i = (int)(e % n_max);
    double2 val = make_double2(0.0, 0.0);
    if (i < nk[k]) {
      const int* mm = m + ((size_t)k * n_max + i) * 3;
      const double qx = b * (mm[0] + kfrac[3 * k]), qy = b * (mm[1] + kfrac[3 * k + 1]),
                   qz = b * (mm[2] + kfrac[3 * k + 2]);
      const double q2 = qx * qx + qy * qy + qz * qz;
      const double gsn = exp(-q2 * w * w / 2.0);
      const int a = j / npa, l = j - (j / npa) * npa;
      const double* R = pos + 3 * a;
      double s, c;
      sincos(qx * R[0] + qy * R[1] + qz * R[2], &s, &c);
      // phase e^{-i q.R} / sqrt(Omega)
      const double2 ph = make_double2(c * invs, -s * invs);
      if (l == 0) {
        val = cscale(ph, fs0 * gsn);
      } else {
        const double qa = l == 1 ? qx : (l == 2 ? qy : qz);
        // F_p = -i q_a fp0 g
        const double2 f = make_double2(0.0, -qa * fp0 * gsn);
        val = cmul(f, ph);
      }
    }
    B[((size_t)k * nproj + j) * n_max + i] = val;
  }
}

// ----------------------------------------------------------------------------- launchers
#define EACG_EXTERN_N(N_) extern template struct GridFft<N_, 0>;
EACG_FOR_EACH_N(EACG_EXTERN_N)
#undef EACG_EXTERN_N
#define EACG_EXTERN_N1(N_) extern template struct GridFft<N_, 1>;
EACG_FOR_EACH_N_PLAN1(EACG_EXTERN_N1)
#undef EACG_EXTERN_N1

#define EACG_CASE_N(N_) \
  case N_:              \
    return true;
bool grid_supported(int N) {
  switch (N) {
    EACG_FOR_EACH_N(EACG_CASE_N)
    default:
      return false;
  }
}
bool grid_has_plan1(int N) {
  switch (N) {
    EACG_FOR_EACH_N_PLAN1(EACG_CASE_N)
    default:
      return false;
  }
}
#undef EACG_CASE_N

// Calls f(GridFft<N, plan>()) for the grid size N (grid_supported(N) is checked at set-up);
// plan 1 falls back to 0 where N has no second plan.
template <typename F>
static void dispatch_n(int N, int plan, const F& f) {
  if (plan == 1) {
    switch (N) {
#define EACG_CASE_N1(N_)  \
  case N_:                \
    f(GridFft<N_, 1>());  \
    return;
      EACG_FOR_EACH_N_PLAN1(EACG_CASE_N1)
#undef EACG_CASE_N1
      default:
        break;
    }
  }
  switch (N) {
#define EACG_CASE_N(N_)   \
  case N_:                \
    f(GridFft<N_, 0>());  \
    break;
    EACG_FOR_EACH_N(EACG_CASE_N)
#undef EACG_CASE_N
    default:
      break;
  }
}

// line-plan variant of the transforms in this precision (0: FP64-accurate, else FP32)
static int plan_of(const GridCtx& g, int prec) { return prec == 0 ? g.plan64 : g.plan32; }
// launch mode of the x passes of FP64 blocks and precision of the plane kernels: the
// FP64-accurate transforms run on the FP64 pipe (mode 0 / prec 0) or in double-float
// arithmetic (mode 3 / prec 2)
static int xmode_of(const GridCtx& g, int prec) { return prec != 0 ? 1 : g.df64 ? 3 : 0; }
static int pprec_of(const GridCtx& g, int prec) { return prec != 0 ? 1 : g.df64 ? 2 : 0; }

// Launches f over chunks of at most GRID_MAX_SEGS requests.
template <typename F>
static void in_chunks(const GridReq* r, int n, const F& f) {
  for (int i = 0; i < n; i += GRID_MAX_SEGS) f(r + i, n - i < GRID_MAX_SEGS ? n - i : GRID_MAX_SEGS);
}

void grid_xpass_inv_multi(int N, int plan, int mode, const GridReq* r, int n, cudaStream_t st) {
  dispatch_n(N, plan, [&](auto G) {
    in_chunks(r, n, [&](const GridReq* c, int m) { decltype(G)::xpass_inv(mode, c, m, st); });
  });
}
void grid_xpass_fwd_multi(int N, int plan, int mode, const GridReq* r, int n, cudaStream_t st) {
  dispatch_n(N, plan, [&](auto G) {
    in_chunks(r, n, [&](const GridReq* c, int m) { decltype(G)::xpass_fwd(mode, c, m, st); });
  });
}
void grid_plane_h_multi(int N, int plan, int prec, const GridReq* r, int n, cudaStream_t st) {
  dispatch_n(N, plan, [&](auto G) {
    in_chunks(r, n, [&](const GridReq* c, int m) { decltype(G)::plane_h(prec, c, m, st); });
  });
}
void grid_plane_rho_multi(int N, int plan, int prec, const GridReq* r, int n, cudaStream_t st) {
  dispatch_n(N, plan, [&](auto G) {
    in_chunks(r, n, [&](const GridReq* c, int m) { decltype(G)::plane_rho(prec, c, m, st); });
  });
}

// Single-system launches: a one-segment table.
static GridReq req_of(const GridCtx& g, int nbands, const int* kactive) {
  GridReq r{};
  r.g = &g;
  r.nbands = nbands;
  r.kactive = kactive;
  r.scale = 1.0;
  r.groups = 1;
  return r;
}

void grid_xpass_inv(const GridCtx& g, int prec, const double2* psi, void* tbuf, int nbands, const int* kactive,
                    cudaStream_t st) {
  GridReq r = req_of(g, nbands, kactive);
  r.in = psi;
  r.tbuf = tbuf;
  grid_xpass_inv_multi(g.N, plan_of(g, prec), xmode_of(g, prec), &r, 1, st);
}

void grid_xpass_fwd(const GridCtx& g, int prec, const void* tbuf, const double2* psi_in, const double* kin,
                    double scale, double2* out, int nbands, const int* kactive, cudaStream_t st) {
  GridReq r = req_of(g, nbands, kactive);
  r.in = psi_in;
  r.tbuf = const_cast<void*>(tbuf);
  r.out = out;
  r.kin = kin;
  r.scale = scale;
  grid_xpass_fwd_multi(g.N, plan_of(g, prec), xmode_of(g, prec), &r, 1, st);
}

void grid_xpass_inv32(const GridCtx& g, const float2* psi, void* tbuf, int nbands, const int* kactive,
                      cudaStream_t st) {
  GridReq r = req_of(g, nbands, kactive);
  r.in = psi;
  r.tbuf = tbuf;
  grid_xpass_inv_multi(g.N, g.plan32, 2, &r, 1, st);
}

void grid_xpass_fwd32(const GridCtx& g, const void* tbuf, const float2* psi_in, const double* kin, double scale,
                      float2* out, int nbands, const int* kactive, cudaStream_t st) {
  GridReq r = req_of(g, nbands, kactive);
  r.in = psi_in;
  r.tbuf = const_cast<void*>(tbuf);
  r.out = out;
  r.kin = kin;
  r.scale = scale;
  grid_xpass_fwd_multi(g.N, g.plan32, 2, &r, 1, st);
}

void grid_plane_h(const GridCtx& g, int prec, void* tbuf, const void* v, int nbands, const int* kactive,
                  cudaStream_t st) {
  GridReq r = req_of(g, nbands, kactive);
  r.tbuf = tbuf;
  r.v = v;
  grid_plane_h_multi(g.N, plan_of(g, prec), pprec_of(g, prec), &r, 1, st);
}

void grid_plane_rho(const GridCtx& g, int prec, const void* tbuf, int nbands, int groups, const double* bw,
                    double* partial, cudaStream_t st) {
  GridReq r = req_of(g, nbands, nullptr);
  r.tbuf = const_cast<void*>(tbuf);
  r.bw = bw;
  r.partial = partial;
  r.groups = groups;
  grid_plane_rho_multi(g.N, plan_of(g, prec), pprec_of(g, prec), &r, 1, st);
}

void grid_fft3(const GridCtx& g, double2* a, bool inverse, cudaStream_t st) {
  dispatch_n(g.N, g.plan64, [&](auto G) { decltype(G)::fft3(g, a, inverse, st); });
}

void grid_reduce_groups(const double* partial, int G, size_t n, double* out, cudaStream_t st) {
  k_reduce_groups<<<(int)min((size_t)1024, (n + 255) / 256), 256, 0, st>>>(partial, G, n, out);
  count_launch();
}

void grid_build_sphere(int N, int K, const double* kfrac_d, double thr, double b, int n_max_cap, int* nk, int* row_off,
                       int* m, double* kin, int* colmark, cudaStream_t st) {
  k_sphere_build<<<K, 256, 0, st>>>(N, kfrac_d, thr, b, n_max_cap, nk, row_off, m, kin, colmark);
  count_launch();
}
void grid_columns(int N, const int* colmark, int* colidx, int* cmapy, int* rowmask, int* ncols, int* ylist, int* ny,
                  cudaStream_t st) {
  k_columns<<<1, 32, 0, st>>>(N, colmark, colidx, cmapy, rowmask, ncols, ylist, ny);
  count_launch();
}
void grid_xmap(int N, int K, int n_max, const int* nk, const int* m, const int* colidx, int ncols, int* xmap,
               cudaStream_t st) {
  k_fill_int<<<256, 256, 0, st>>>(xmap, (size_t)K * ncols * N, -1);
  count_launch();
  dim3 grid((n_max + 255) / 256, K);
  k_xmap<<<grid, 256, 0, st>>>(N, K, n_max, nk, m, colidx, ncols, xmap);
  count_launch();
}
void grid_vloc_g(int N, double b, double omega, int natoms, const double* pos, const double* Z, const double* rc,
                 double2* out, cudaStream_t st) {
  k_vloc_g<<<1024, 256, 0, st>>>(N, b, omega, natoms, pos, Z, rc, out);
  count_launch();
}
void grid_hartree_scale(double2* a, int N, double b, cudaStream_t st) { k_hartree_scale<<<1024, 256, 0, st>>>(a, N, b);
  count_launch(); }
void grid_real_to_complex(const double* r, double2* c, size_t n, cudaStream_t st) {
  k_real_to_complex<<<1024, 256, 0, st>>>(r, c, n);
  count_launch();
}
void grid_complex_real_part(const double2* c, double* r, size_t n, cudaStream_t st) {
  k_complex_real_part<<<1024, 256, 0, st>>>(c, r, n);
  count_launch();
}
int grid_vtot_energy(size_t n, const double* vloc, const double* vh, const double* rho, int hartree, int xc,
                     double* vtot, float* vtot32, float2* vtotdf, double* blocksums, cudaStream_t st) {
  const int blocks = 256;
  k_vtot_energy<<<blocks, 256, 0, st>>>(n, vloc, vh, rho, hartree, xc, vtot, vtot32, vtotdf, blocksums);
  count_launch();
  return blocks;
}
void grid_projectors(int K, int n_max, const int* nk, const int* m, const double* kfrac, double b, double omega,
                     int natoms, const double* pos, int npa, double w, double2* B, cudaStream_t st) {
  dim3 grid(256, K);
  k_projectors<<<grid, 256, 0, st>>>(K, n_max, nk, m, kfrac, b, omega, natoms, pos, npa, w, B);
  count_launch();
}

}  // namespace eacg
