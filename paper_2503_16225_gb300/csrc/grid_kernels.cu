// Plane-wave grid kernels of libeacg (sm_103a): G-sphere index maps, the pruned
// 3D FFT pair of the Hamiltonian application, the density accumulation, and
// the potential build (Hartree by FFT, Slater exchange, Gaussian local part).
//
// Layouts (all row-major, last index fastest):
//   coefficient blocks  psi[K][p][n_max]        complex double, zero beyond n_k
//   real-space grids    v[jx][jy][jz]            N^3
//   FFT intermediate    tbuf[band][jx][col]      band = k * p + i, col = (my, mz) disk column
// The transform of one band runs as
//   x-pass  (columns (my, mz) of the cutoff sphere, along x)           k_xpass_inv
//   plane   (fixed jx: z along the columns' rows, then y; V multiply)  k_plane_h / k_plane_rho
//   x-pass  (forward, gather back onto the sphere)                      k_xpass_fwd
#include <math.h>

#include "common.cuh"
#include "fft.cuh"
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

// Single CTA: list of union columns in canonical (my, mz) order, their FFT indices and
// the list of distinct fy rows.  colidx[(my+h)*N + (mz+h)] = column number or -1.
__global__ void k_columns(int N, const int* __restrict__ colmark, int* __restrict__ colidx, int* __restrict__ colfy,
                          int* __restrict__ colfz, int* __restrict__ ncols_out, int* __restrict__ ylist,
                          int* __restrict__ ny_out) {
  if (threadIdx.x != 0) return;
  const int h = N / 2;
  int c = 0, ny = 0;
  for (int a = 0; a < N; ++a) {
    bool rowhas = false;
    for (int z = 0; z < N; ++z) {
      const int r = a * N + z;
      if (colmark[r]) {
        colidx[r] = c;
        const int my = a - h, mz = z - h;
        colfy[c] = (my % N + N) % N;
        colfz[c] = (mz % N + N) % N;
        ++c;
        rowhas = true;
      } else {
        colidx[r] = -1;
      }
    }
    if (rowhas) ylist[ny++] = ((a - h) % N + N) % N;
  }
  *ncols_out = c;
  *ny_out = ny;
}

// xmap[k][col][fx] = sphere index of (mx = fx signed, my, mz) at k, or -1.
__global__ void k_xmap(int N, int K, int n_max, const int* __restrict__ nk, const int* __restrict__ m,
                       const int* __restrict__ colidx, int ncols, int* __restrict__ xmap) {
  const int k = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nk[k]) return;
  const int* mm = m + ((size_t)k * n_max + i) * 3;
  const int h = N / 2;
  const int c = colidx[(mm[1] + h) * N + (mm[2] + h)];
  const int fx = (mm[0] % N + N) % N;
  xmap[((size_t)k * ncols + c) * N + fx] = i;
}

__global__ void k_fill_int(int* p, size_t n, int v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// ----------------------------------------------------------------------------- x passes
// Inverse x pass: per CTA, cols_per_cta columns of one band.  Shared: twiddles, lines
// with pitch N + 1.  Output tbuf[band][jx][col].
template <typename T, int E, typename TIO>
__global__ void k_xpass_inv(const TIO* __restrict__ psi, int n_max, int p, const int* __restrict__ xmap,
                            int ncols, cplx<T>* __restrict__ tbuf, FftPlan pl, const cplx<T>* __restrict__ tw_g,
                            int cols_per_cta, const int* __restrict__ kactive) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* lines = tw + pl.N;
  const int N = pl.N, LP = N + 1;
  const int band = blockIdx.y;
  const int k = band / p;
  if (kactive && !kactive[k]) return;
  const int c0 = blockIdx.x * cols_per_cta;
  const int nc = min(cols_per_cta, ncols - c0);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  const int* xm = xmap + ((size_t)k * ncols + c0) * N;
  const TIO* src = psi + (size_t)band * n_max;
  for (int e = threadIdx.x; e < nc * N; e += blockDim.x) {
    const int c = e / N, fx = e - c * N;
    const int id = xm[e];
    V v;
    if (id >= 0) {
      v = cvt<V>(src[id]);
    } else {
      v.x = 0;
      v.y = 0;
    }
    lines[c * LP + fx] = v;
  }
  __syncthreads();
  fft_lines<V, E, true>(lines, nc, LP, 1, pl, tw);
  V* dst = tbuf + (size_t)band * N * ncols + c0;
  for (int e = threadIdx.x; e < nc * N; e += blockDim.x) {
    const int jx = e / nc, c = e - jx * nc;
    dst[(size_t)jx * ncols + c] = lines[c * LP + jx];
  }
}

// Forward x pass and gather: out = scale * FFT + kin * psi_in (kin may be null).
template <typename T, int E, typename TIO>
__global__ void k_xpass_fwd(const cplx<T>* __restrict__ tbuf, const int* __restrict__ xmap, int ncols, FftPlan pl,
                            const cplx<T>* __restrict__ tw_g, int cols_per_cta, int n_max, int p,
                            const int* __restrict__ nk, const TIO* __restrict__ psi_in,
                            const double* __restrict__ kin, double scale, TIO* __restrict__ out,
                            const int* __restrict__ kactive) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* lines = tw + pl.N;
  const int N = pl.N, LP = N + 1;
  const int band = blockIdx.y;
  const int k = band / p;
  if (kactive && !kactive[k]) return;
  const int c0 = blockIdx.x * cols_per_cta;
  const int nc = min(cols_per_cta, ncols - c0);
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  const V* src = tbuf + (size_t)band * N * ncols + c0;
  for (int e = threadIdx.x; e < nc * N; e += blockDim.x) {
    const int jx = e / nc, c = e - jx * nc;
    lines[c * LP + jx] = src[(size_t)jx * ncols + c];
  }
  __syncthreads();
  fft_lines<V, E, false>(lines, nc, LP, 1, pl, tw);
  const int* xm = xmap + ((size_t)k * ncols + c0) * N;
  TIO* o = out + (size_t)band * n_max;
  const TIO* pin = psi_in + (size_t)band * n_max;
  const double* kk = kin ? kin + (size_t)k * n_max : nullptr;
  for (int e = threadIdx.x; e < nc * N; e += blockDim.x) {
    const int c = e / N, fx = e - c * N;
    const int id = xm[e];
    if (id >= 0) {
      double2 v = cscale(to_d(lines[c * LP + fx]), scale);
      if (kk) {
        const double2 s = to_d(pin[id]);
        v.x += kk[id] * s.x;
        v.y += kk[id] * s.y;
      }
      o[id] = cvt<TIO>(v);
    }
  }
  if (blockIdx.x == 0) {
    for (int i = nk[k] + threadIdx.x; i < n_max; i += blockDim.x) o[i] = cvt<TIO>(make_double2(0.0, 0.0));
  }
}

// ----------------------------------------------------------------------------- plane kernels
// Apply the local potential to one x-plane of one band: z inverse (rows with columns),
// y inverse (all jz), multiply by v, y forward, z forward, write the disk columns back.
template <typename T, int E>
__global__ void k_plane_h(cplx<T>* __restrict__ tbuf, int ncols, const int* __restrict__ colfy,
                          const int* __restrict__ colfz, const int* __restrict__ ylist, int ny,
                          const T* __restrict__ v, FftPlan pl, const cplx<T>* __restrict__ tw_g, int p,
                          const int* __restrict__ kactive) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = pl.N, PP = N + 1;
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* plane = tw + N;
  int* yoff = reinterpret_cast<int*>(plane + (size_t)N * PP);
  const int jx = blockIdx.x, band = blockIdx.y;
  if (kactive && !kactive[band / p]) return;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = threadIdx.x; i < ny; i += blockDim.x) yoff[i] = ylist[i] * PP;
  for (int i = threadIdx.x; i < N * PP; i += blockDim.x) {
    plane[i].x = 0;
    plane[i].y = 0;
  }
  __syncthreads();
  V* tb = tbuf + ((size_t)band * N + jx) * ncols;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) plane[colfy[c] * PP + colfz[c]] = tb[c];
  __syncthreads();
  fft_lines_list<V, E, true>(plane, yoff, ny, 1, pl, tw);   // along z, rows fy with data
  fft_lines<V, E, true>(plane, N, 1, PP, pl, tw);            // along y, every jz
  const T* vv = v + (size_t)jx * N * N;
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int jy = e / N, jz = e - jy * N;
    plane[jy * PP + jz] = cscale(plane[jy * PP + jz], vv[e]);
  }
  __syncthreads();
  fft_lines<V, E, false>(plane, N, 1, PP, pl, tw);
  fft_lines_list<V, E, false>(plane, yoff, ny, 1, pl, tw);
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) tb[c] = plane[colfy[c] * PP + colfz[c]];
}

// Density of a group of bands on one x-plane: sum_b w_b |u_b|^2 accumulated in FP64
// registers in a fixed band order, written as partial[g][jx][jy][jz].
constexpr int RHO_NPT = 16;
template <typename T, int E>
__global__ void k_plane_rho(const cplx<T>* __restrict__ tbuf, int ncols, const int* __restrict__ colfy,
                            const int* __restrict__ colfz, const int* __restrict__ ylist, int ny, FftPlan pl,
                            const cplx<T>* __restrict__ tw_g, int nbands, int bands_per_group,
                            const double* __restrict__ bw, double* __restrict__ partial) {
  using V = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = pl.N, PP = N + 1;
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* plane = tw + N;
  int* yoff = reinterpret_cast<int*>(plane + (size_t)N * PP);
  const int jx = blockIdx.x, g = blockIdx.y;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  for (int i = threadIdx.x; i < ny; i += blockDim.x) yoff[i] = ylist[i] * PP;
  double acc[RHO_NPT];
#pragma unroll
  for (int i = 0; i < RHO_NPT; ++i) acc[i] = 0.0;
  const int b0 = g * bands_per_group, b1 = min(nbands, b0 + bands_per_group);
  for (int band = b0; band < b1; ++band) {
    for (int i = threadIdx.x; i < N * PP; i += blockDim.x) {
      plane[i].x = 0;
      plane[i].y = 0;
    }
    __syncthreads();
    const V* tb = tbuf + ((size_t)band * N + jx) * ncols;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) plane[colfy[c] * PP + colfz[c]] = tb[c];
    __syncthreads();
    fft_lines_list<V, E, true>(plane, yoff, ny, 1, pl, tw);
    fft_lines<V, E, true>(plane, N, 1, PP, pl, tw);
    const double w = bw[band];
#pragma unroll
    for (int i = 0; i < RHO_NPT; ++i) {
      const int e = threadIdx.x + i * blockDim.x;
      if (e < N * N) {
        const int jy = e / N, jz = e - jy * N;
        const double2 u = to_d(plane[jy * PP + jz]);
        acc[i] += w * (u.x * u.x + u.y * u.y);
      }
    }
    __syncthreads();
  }
  double* out = partial + ((size_t)g * N + jx) * N * N;
#pragma unroll
  for (int i = 0; i < RHO_NPT; ++i) {
    const int e = threadIdx.x + i * blockDim.x;
    if (e < N * N) out[e] = acc[i];
  }
}

__global__ void k_reduce_groups(const double* __restrict__ partial, int G, size_t n, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += partial[(size_t)g * n + i];
    out[i] = s;
  }
}

// ----------------------------------------------------------------------------- full 3D FFT
// Lines along one axis of a complex N^3 array a[x][y][z]; axis 2 = z, 1 = y, 0 = x.
template <int E, bool INV>
__global__ void k_fft3_axis(double2* __restrict__ a, int axis, FftPlan pl, const double2* __restrict__ tw_g,
                            int lines_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = pl.N, LP = N + 1;
  double2* tw = reinterpret_cast<double2*>(smem_raw);
  double2* lines = tw + N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = tw_g[i];
  const int l0 = blockIdx.x * lines_per_cta;
  const int nl = min(lines_per_cta, N * N - l0);
  // line l (0..N^2): axis z: (x, y) = (l / N, l % N); axis y: (x, z); axis x: (y, z)
  auto addr = [&](int l, int j) -> size_t {
    const int u = l / N, w = l - (l / N) * N;
    if (axis == 2) return ((size_t)u * N + w) * N + j;
    if (axis == 1) return ((size_t)u * N + j) * N + w;
    return ((size_t)j * N + u) * N + w;
  };
  for (int e = threadIdx.x; e < nl * N; e += blockDim.x) {
    int l, j;
    if (axis == 2) {
      l = e / N;
      j = e - l * N;
    } else {
      j = e / nl;
      l = e - j * nl;
    }
    lines[l * LP + j] = a[addr(l0 + l, j)];
  }
  __syncthreads();
  fft_lines<double2, E, INV>(lines, nl, LP, 1, pl, tw);
  for (int e = threadIdx.x; e < nl * N; e += blockDim.x) {
    int l, j;
    if (axis == 2) {
      l = e / N;
      j = e - l * N;
    } else {
      j = e / nl;
      l = e - j * nl;
    }
    a[addr(l0 + l, j)] = lines[l * LP + j];
  }
}

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

// V_tot = V_loc + V_H + V_x(rho) and the energy integrands (loc, hartree, xc) reduced per block.
__global__ void k_vtot_energy(size_t n, const double* __restrict__ vloc, const double* __restrict__ vh,
                              const double* __restrict__ rho, int hartree, int xc, double* __restrict__ vtot,
                              float* __restrict__ vtot32, double* __restrict__ blocksums /*[gridDim][3]*/) {
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
    }
    vtot[i] = v;
    if (vtot32) vtot32[i] = (float)v;
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
template <typename T, int E, typename TIO>
static void launch_xinv(const GridCtx& g, const TIO* psi, void* tbuf, const void* tw, int nbands,
                        const int* kactive, cudaStream_t st) {
  const int cpc = g.cols_per_cta;
  dim3 grid((g.ncols + cpc - 1) / cpc, nbands);
  const int threads = min(1024, max(32, cpc * g.plan.TPL));
  const size_t sm = sizeof(cplx<T>) * (g.plan.N + (size_t)cpc * (g.plan.N + 1));
  ensure_smem((const void*)k_xpass_inv<T, E, TIO>, sm);
  k_xpass_inv<T, E, TIO><<<grid, threads, sm, st>>>(psi, g.n_max, g.p, g.xmap, g.ncols, (cplx<T>*)tbuf, g.plan,
                                                    (const cplx<T>*)tw, cpc, kactive);
  count_launch();
}

template <typename T, int E, typename TIO>
static void launch_xfwd(const GridCtx& g, const void* tbuf, const void* tw, const TIO* psi_in, const double* kin,
                        double scale, TIO* out, int nbands, const int* kactive, cudaStream_t st) {
  const int cpc = g.cols_per_cta;
  dim3 grid((g.ncols + cpc - 1) / cpc, nbands);
  const int threads = min(1024, max(32, cpc * g.plan.TPL));
  const size_t sm = sizeof(cplx<T>) * (g.plan.N + (size_t)cpc * (g.plan.N + 1));
  ensure_smem((const void*)k_xpass_fwd<T, E, TIO>, sm);
  k_xpass_fwd<T, E, TIO><<<grid, threads, sm, st>>>((const cplx<T>*)tbuf, g.xmap, g.ncols, g.plan,
                                                    (const cplx<T>*)tw, cpc, g.n_max, g.p, g.nk, psi_in, kin, scale,
                                                    out, kactive);
  count_launch();
}

template <typename T>
static size_t plane_smem(int N, int ny) {
  return sizeof(cplx<T>) * ((size_t)N + (size_t)N * (N + 1)) + sizeof(int) * (size_t)ny;
}

static int plane_threads(const FftPlan& pl) {
  int t = pl.N * pl.TPL;
  if (t > 1024) t = (1024 / pl.TPL) * pl.TPL;
  if (t < 64) t = 64;
  return t;
}

template <typename T, int E>
static void launch_plane_h(const GridCtx& g, void* tbuf, const void* tw, const void* v, int nbands,
                           const int* kactive, cudaStream_t st) {
  const size_t sm = plane_smem<T>(g.plan.N, g.ny);
  ensure_smem((const void*)k_plane_h<T, E>, sm);
  dim3 grid(g.plan.N, nbands);
  k_plane_h<T, E><<<grid, plane_threads(g.plan), sm, st>>>((cplx<T>*)tbuf, g.ncols, g.colfy, g.colfz, g.ylist, g.ny,
                                                           (const T*)v, g.plan, (const cplx<T>*)tw, g.p, kactive);
  count_launch();
}

template <typename T, int E>
static void launch_plane_rho(const GridCtx& g, const void* tbuf, const void* tw, int nbands, int groups,
                             const double* bw, double* partial, cudaStream_t st) {
  const size_t sm = plane_smem<T>(g.plan.N, g.ny);
  ensure_smem((const void*)k_plane_rho<T, E>, sm);
  int threads = plane_threads(g.plan);
  const int need = (g.plan.N * g.plan.N + RHO_NPT - 1) / RHO_NPT;
  while (threads < need) threads += g.plan.TPL;
  const int bpg = (nbands + groups - 1) / groups;
  dim3 grid(g.plan.N, groups);
  k_plane_rho<T, E><<<grid, threads, sm, st>>>((const cplx<T>*)tbuf, g.ncols, g.colfy, g.colfz, g.ylist, g.ny,
                                               g.plan, (const cplx<T>*)tw, nbands, bpg, bw, partial);
  count_launch();
}

#define EACG_DISPATCH_E(E_, CALL)                              \
  switch (E_) {                                                \
    case 4: { constexpr int EE = 4; CALL; } break;             \
    case 8: { constexpr int EE = 8; CALL; } break;             \
    case 12: { constexpr int EE = 12; CALL; } break;           \
    case 20: { constexpr int EE = 20; CALL; } break;           \
    default: break;                                            \
  }

void grid_xpass_inv(const GridCtx& g, int prec, const double2* psi, void* tbuf, int nbands, const int* kactive,
                    cudaStream_t st) {
  if (prec == 0) {
    EACG_DISPATCH_E(g.plan.E, (launch_xinv<double, EE, double2>(g, psi, tbuf, g.tw64, nbands, kactive, st)));
  } else {
    EACG_DISPATCH_E(g.plan.E, (launch_xinv<float, EE, double2>(g, psi, tbuf, g.tw32, nbands, kactive, st)));
  }
}

void grid_xpass_fwd(const GridCtx& g, int prec, const void* tbuf, const double2* psi_in, const double* kin,
                    double scale, double2* out, int nbands, const int* kactive, cudaStream_t st) {
  if (prec == 0) {
    EACG_DISPATCH_E(g.plan.E, (launch_xfwd<double, EE, double2>(g, tbuf, g.tw64, psi_in, kin, scale, out, nbands,
                                                                kactive, st)));
  } else {
    EACG_DISPATCH_E(g.plan.E, (launch_xfwd<float, EE, double2>(g, tbuf, g.tw32, psi_in, kin, scale, out, nbands,
                                                               kactive, st)));
  }
}

void grid_xpass_inv32(const GridCtx& g, const float2* psi, void* tbuf, int nbands, const int* kactive,
                      cudaStream_t st) {
  EACG_DISPATCH_E(g.plan.E, (launch_xinv<float, EE, float2>(g, psi, tbuf, g.tw32, nbands, kactive, st)));
}

void grid_xpass_fwd32(const GridCtx& g, const void* tbuf, const float2* psi_in, const double* kin, double scale,
                      float2* out, int nbands, const int* kactive, cudaStream_t st) {
  EACG_DISPATCH_E(g.plan.E,
                  (launch_xfwd<float, EE, float2>(g, tbuf, g.tw32, psi_in, kin, scale, out, nbands, kactive, st)));
}

void grid_plane_h(const GridCtx& g, int prec, void* tbuf, const void* v, int nbands, const int* kactive,
                  cudaStream_t st) {
  if (prec == 0) {
    EACG_DISPATCH_E(g.plan.E, (launch_plane_h<double, EE>(g, tbuf, g.tw64, v, nbands, kactive, st)));
  } else {
    EACG_DISPATCH_E(g.plan.E, (launch_plane_h<float, EE>(g, tbuf, g.tw32, v, nbands, kactive, st)));
  }
}

void grid_plane_rho(const GridCtx& g, int prec, const void* tbuf, int nbands, int groups, const double* bw,
                    double* partial, cudaStream_t st) {
  if (prec == 0) {
    EACG_DISPATCH_E(g.plan.E, (launch_plane_rho<double, EE>(g, tbuf, g.tw64, nbands, groups, bw, partial, st)));
  } else {
    EACG_DISPATCH_E(g.plan.E, (launch_plane_rho<float, EE>(g, tbuf, g.tw32, nbands, groups, bw, partial, st)));
  }
}

void grid_reduce_groups(const double* partial, int G, size_t n, double* out, cudaStream_t st) {
  k_reduce_groups<<<(int)min((size_t)1024, (n + 255) / 256), 256, 0, st>>>(partial, G, n, out);
  count_launch();
}

template <int E, bool INV>
static void launch_fft3(const GridCtx& g, double2* a, int axis, cudaStream_t st) {
  const int N = g.plan.N;
  int lpc = 32;
  const size_t sm = sizeof(double2) * ((size_t)N + (size_t)lpc * (N + 1));
  const int threads = min(1024, lpc * g.plan.TPL);
  const int blocks = (N * N + lpc - 1) / lpc;
  ensure_smem((const void*)k_fft3_axis<E, INV>, sm);
  k_fft3_axis<E, INV><<<blocks, threads, sm, st>>>(a, axis, g.plan, (const double2*)g.tw64, lpc);
  count_launch();
}

void grid_fft3(const GridCtx& g, double2* a, bool inverse, cudaStream_t st) {
  for (int axis = 2; axis >= 0; --axis) {
    if (inverse) {
      EACG_DISPATCH_E(g.plan.E, (launch_fft3<EE, true>(g, a, axis, st)));
    } else {
      EACG_DISPATCH_E(g.plan.E, (launch_fft3<EE, false>(g, a, axis, st)));
    }
  }
}

void grid_build_sphere(int N, int K, const double* kfrac_d, double thr, double b, int n_max_cap, int* nk, int* row_off,
                       int* m, double* kin, int* colmark, cudaStream_t st) {
  k_sphere_build<<<K, 256, 0, st>>>(N, kfrac_d, thr, b, n_max_cap, nk, row_off, m, kin, colmark);
  count_launch();
}
void grid_columns(int N, const int* colmark, int* colidx, int* colfy, int* colfz, int* ncols, int* ylist, int* ny,
                  cudaStream_t st) {
  k_columns<<<1, 32, 0, st>>>(N, colmark, colidx, colfy, colfz, ncols, ylist, ny);
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
void grid_fill_int(int* p, size_t n, int v, cudaStream_t st) { k_fill_int<<<256, 256, 0, st>>>(p, n, v);
  count_launch(); }
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
                     double* vtot, float* vtot32, double* blocksums, cudaStream_t st) {
  const int blocks = 256;
  k_vtot_energy<<<blocks, 256, 0, st>>>(n, vloc, vh, rho, hartree, xc, vtot, vtot32, blocksums);
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
