// Internal launch interface between the C-ABI driver (eacg.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"


namespace eacg {

// Counts one kernel launch of this library (defined in eacg.cu).
void count_launch();
// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the current device.
// The limit is a process-wide property of the kernel, so it only ever grows: systems of
// different sizes running concurrently in several host threads never lower it under each
// other's launches (defined in eacg.cu).
void ensure_smem(const void* func, size_t bytes);

// Device-side description of the plane-wave grid of one system.
struct GridCtx {
  int N, K, p, n_max, ncols, ny;
  int plan64, plan32;  // line-plan variant of the FP64 and the FP32 transforms (0 or 1)
  const int* nk;       // [K]
  const int* xmap;     // [K][N][ncols]: sphere index of (fx, column) at k, or -1
  const int* cmapy;    // [ny][N + 1]: column of (ylist[l], fz), or -1
  const int* rowmask;  // [N]: 1 if row fy holds columns
  const int* ylist;    // [ny]: the rows fy that hold columns
  const void* tw64;    // double2[N]
  const void* tw32;    // float2[N]
  const void* twdf;    // dcomplex[N]
  int df64;            // 1: the FP64-accurate transforms run in double-float arithmetic
};

// One system's share of a transform launch.  A launch covers the bands of up to
// GRID_MAX_SEGS systems of the same grid size, line plan and precision: grid row y of the
// launch belongs to the segment with the largest y0 <= y (bands for the x passes and the
// potential multiply, band groups for the density).  The table travels as a kernel parameter.
struct GridSeg {
  const void* in;        // coefficient blocks [bands][n_max] (block precision)
  void* tbuf;            // x-pass intermediate [bands][N][ncols] (transform precision)
  void* out;             // forward x pass: result blocks [bands][n_max]
  const double* kin;     // forward x pass: kinetic factors [K][n_max] (may be null)
  const void* v;         // plane kernel: potential [N^3] (transform precision)
  const int* kactive;    // [K] or null
  const int* nk;         // [K]
  const int* xmap;       // [K][N][ncols]
  const int* cmapy;      // [ny][N + 1]
  const int* ylist;      // [ny]
  const int* rowmask;    // [N]
  const void* tw;        // twiddles [N] (transform precision)
  const double* bw;      // density: weight of every band
  double* partial;       // density: [groups][N^3]
  double scale;          // forward x pass: factor of the transform
  int n_max, p, ncols, ny, nbands, groups;
  int y0;                // first grid row of the segment
};
constexpr int GRID_MAX_SEGS = 16;
struct GridSegs {
  int n;
  GridSeg s[GRID_MAX_SEGS];
};

// A transform request of one system, the unit a multi-system launch is built from.
struct GridReq {
  const GridCtx* g;
  const void* in;
  void* tbuf;
  void* out;
  const double* kin;
  double scale;
  const void* v;
  const int* kactive;
  int nbands;
  const double* bw;
  double* partial;
  int groups;
};

// ---- grid_kernels.cu
// Multi-system transform launches (one kernel launch per call for up to GRID_MAX_SEGS requests
// of the same N, line plan and mode; longer lists are split).  mode 0: FP64 transforms of FP64
// blocks; 1: FP32 transforms of FP64 blocks; 2: FP32 transforms of FP32 blocks.  plane_h and
// plane_rho take prec (0 FP64, 1 FP32).
void grid_xpass_inv_multi(int N, int plan, int mode, const GridReq* r, int n, cudaStream_t st);
void grid_xpass_fwd_multi(int N, int plan, int mode, const GridReq* r, int n, cudaStream_t st);
void grid_plane_h_multi(int N, int plan, int prec, const GridReq* r, int n, cudaStream_t st);
void grid_plane_rho_multi(int N, int plan, int prec, const GridReq* r, int n, cudaStream_t st);
void grid_build_sphere(int N, int K, const double* kfrac_d, double thr, double b, int n_max_cap, int* nk, int* row_off,
                       int* m, double* kin, int* colmark, cudaStream_t st);
// True if N has a compile-time line plan (the grid sizes this library transforms), and if it
// has a second plan variant for the autotuner to try.
bool grid_supported(int N);
bool grid_has_plan1(int N);
void grid_columns(int N, const int* colmark, int* colidx, int* cmapy, int* rowmask, int* ncols, int* ylist, int* ny,
                  cudaStream_t st);
void grid_xmap(int N, int K, int n_max, const int* nk, const int* m, const int* colidx, int ncols, int* xmap,
               cudaStream_t st);
void grid_xpass_inv(const GridCtx& g, int prec, const double2* psi, void* tbuf, int nbands, const int* kactive,
                    cudaStream_t st);
void grid_xpass_fwd(const GridCtx& g, int prec, const void* tbuf, const double2* psi_in, const double* kin,
                    double scale, double2* out, int nbands, const int* kactive, cudaStream_t st);
// FP32 blocks in and out (FP32 transforms): used by the FOM of the mixed-precision mode.
void grid_xpass_inv32(const GridCtx& g, const float2* psi, void* tbuf, int nbands, const int* kactive,
                      cudaStream_t st);
void grid_xpass_fwd32(const GridCtx& g, const void* tbuf, const float2* psi_in, const double* kin, double scale,
                      float2* out, int nbands, const int* kactive, cudaStream_t st);
void grid_plane_h(const GridCtx& g, int prec, void* tbuf, const void* v, int nbands, const int* kactive,
                  cudaStream_t st);
void grid_plane_rho(const GridCtx& g, int prec, const void* tbuf, int nbands, int groups, const double* bw,
                    double* partial, cudaStream_t st);
void grid_reduce_groups(const double* partial, int G, size_t n, double* out, cudaStream_t st);
void grid_fft3(const GridCtx& g, double2* a, bool inverse, cudaStream_t st);
void grid_vloc_g(int N, double b, double omega, int natoms, const double* pos, const double* Z, const double* rc,
                 double2* out, cudaStream_t st);
void grid_hartree_scale(double2* a, int N, double b, cudaStream_t st);
void grid_real_to_complex(const double* r, double2* c, size_t n, cudaStream_t st);
void grid_complex_real_part(const double2* c, double* r, size_t n, cudaStream_t st);
int grid_vtot_energy(size_t n, const double* vloc, const double* vh, const double* rho, int hartree, int xc,
                     double* vtot, float* vtot32, float2* vtotdf, double* blocksums, cudaStream_t st);
void grid_projectors(int K, int n_max, const int* nk, const int* m, const double* kfrac, double b, double omega,
                     int natoms, const double* pos, int npa, double w, double2* B, cudaStream_t st);

// ---- dense_kernels.cu  (complex double blocks, batched over k with per-k strides)
// C[k](m x n, ldc) = alpha * A[k]^H B[k] + beta * C[k]; A: L x m (lda), B: L x n (ldb).
// Deterministic: fixed row chunks reduced in a fixed order.  work must hold
// K * nchunks * m * n double2 (see dense_cn_work).
size_t dense_cn_work(int K, int L, int m, int n);
// C_k = alpha sum_ch part[k][ch] + beta C_k (fixed chunk order), part[k][ch][n][m]
void dense_cn_reduce(int K, int m, int n, int nch, const double2* work, double2* C, size_t sC, int ldc,
                     double2 alpha, double2 beta, const int* kactive, cudaStream_t st);
// Block overlaps of complex64 blocks on the tensor cores (tcgen05, 3 x TF32 split, FP32
// accumulation per chunk of 1024 rows, FP64 chunk sums); C_k = alpha A_k^* B_k + beta C_k.
// Eligible shapes: m >= 128 and n a multiple of 16.  work: dense_overlap_tc_work elements.
bool dense_overlap_tc_eligible(int m, int n);
size_t dense_overlap_tc_work(int K, int L, int m, int n);
void dense_overlap_tf32x3(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const float2* B,
                          size_t sB, int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta,
                          double2* work, const int* kactive, cudaStream_t st);
// Back-projection C_k += A_k Q_k on the tensor cores (same split and accumulation): A_k L x m
// complex64 ([m][lda]), Q_k m x n complex double ([n][ldq]), C_k L x n complex double
// ([n][ldc]).  Eligible: 16 <= n <= 256, n a multiple of 16.
bool dense_backproject_tc_eligible(int m, int n);
void dense_backproject_tf32x3(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const double2* Q,
                              size_t sQ, int ldq, double2* C, size_t sC, int ldc, const int* kactive,
                              cudaStream_t st);
// Number of tensor-core CTAs on the current device whose bounded mbarrier waits gave up (their
// outputs hold NaN) since the library was loaded; read on st after synchronising it (~0u when
// the read fails).  A change across a call marks that call, or one running beside it, failed.
unsigned int dense_tc_gaveup_count(cudaStream_t st);
// df = 1: the products and sums in double-float arithmetic (FP64-accurate, on the FP32 pipe).
void dense_gemm_cn(int K, int L, int m, int n, const double2* A, size_t sA, int lda, const double2* B, size_t sB,
                   int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta, double2* work,
                   const int* kactive, cudaStream_t st, int df = 0);
// C[k](L x n, ldc) = alpha * A[k](L x m, lda) * B[k](m x n, ldb) + beta * C[k].
void dense_gemm_nn(int K, int L, int m, int n, const double2* A, size_t sA, int lda, const double2* B, size_t sB,
                   int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta, const int* kactive,
                   cudaStream_t st, int df = 0);
// Tile autotune of the A^H B kernel: times its row-group variants on these operands (Kt
// k-points, prec 0 complex128 / 1 complex64 A and B) and records the fastest for the shape bucket
// of (m, n, L) for the whole process (kept if already tuned).  C: Kt * m * n, work:
// dense_cn_work(Kt, L, m, n).  dense_cn_groups: the variant in use for a shape (4 if untuned).
void dense_tune_cn(int Kt, int L, int m, int n, int prec, const void* A, size_t sA, int lda, const void* B,
                   size_t sB, int ldb, double2* C, double2* work, cudaStream_t st);
int dense_cn_groups(int m, int n, int L, int prec);
int dense_cn_force(int groups);  // 1, 2, 4 forces that variant for every shape; 0 back to tuned
// FP32-block variants: A, B (cn) / A, C (nn) complex64, FP32 accumulation; small factors and
// the cn result stay FP64.
void dense_gemm_cn32(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const float2* B, size_t sB,
                     int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta, double2* work,
                     const int* kactive, cudaStream_t st);
void dense_gemm_nn32(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const double2* B, size_t sB,
                     int ldb, float2* C, size_t sC, int ldc, double2 alpha, double2 beta, const int* kactive,
                     cudaStream_t st);
// complex64 A times FP64 B (staged in FP32, FP32 accumulation) formed and added into an FP64 C
void dense_gemm_nn32_into64(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const double2* B,
                            size_t sB, int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta,
                            const int* kactive, cudaStream_t st);
void dense_to32(size_t n, const double2* x, double sc, float2* y, cudaStream_t st);
void dense_to64(size_t n, const float2* x, double2* y, cudaStream_t st);
void dense_axpby32(size_t n, double2 a, const float2* x, double2 b, const float2* y, float2* out, cudaStream_t st);
void dense_norms2_32(int K, size_t len, const float2* V, double* out, cudaStream_t st);
void dense_tpa32(int K, int p, int n_max, const double* kin, const double* alpha, const float2* in, float2* out,
                 cudaStream_t st);
// The p x p kernels (eigen-decomposition, inverse, Lyapunov, pivoted Cholesky) run one CTA per
// k with the matrices in shared memory while they fit (up to p = 64 to 80 by kernel), else in a
// global scratch of dense_pp_scratch(K, p) bytes (0 when none is needed) passed as `scratch`.
size_t dense_pp_scratch(int K, int p);
// Hermitian eigen-decomposition of K matrices p x p (ld p): ascending eigenvalues and
// unit eigenvectors (columns).
void dense_heig(int K, int p, const double2* A, size_t sA, double* w, double2* V, const int* kactive, cudaStream_t st,
                void* scratch = nullptr);
// out[k] = V diag(f(w)) V^H with f(x) = x^e (e = -0.5, 0.5) restricted to w > cut; else 0.
void dense_eig_func(int K, int p, const double2* V, const double* w, double expo, double cut_rel, double2* out,
                    const int* kactive, cudaStream_t st);
// Inverse of K general p x p complex matrices (Gauss-Jordan, partial pivoting).
void dense_inverse(int K, int p, const double2* A, double2* Ainv, int* info, cudaStream_t st, void* scratch = nullptr);
// Lyapunov S X + X S = M with S = V diag(s) V^H: X = V [(V^H M V)_ij / (s_i + s_j)] V^H.
void dense_lyapunov(int K, int p, const double2* V, const double* s, const double2* M, double2* X, cudaStream_t st,
                    void* scratch = nullptr);
// Elementwise helpers on blocks of length n per k (K blocks, stride s).
void dense_axpby(size_t n, double2 a, const double2* x, double2 b, const double2* y, double2* out, cudaStream_t st);
void dense_herm(int K, int p, double2* A, cudaStream_t st);
void dense_shift_diag(int K, int p, const double2* A, double mu, double2* out, cudaStream_t st);
// partial sums of sum_k wk Re <V_k, W_k> over blocks [K][len]: returns number of partials
int dense_dot(int K, size_t len, const double2* V, const double2* W, const double* wk, double* partials,
              cudaStream_t st);
void dense_sum_partials(const double* partials, int n, double* out, cudaStream_t st);
// Per-k Frobenius norm squared of blocks [K][len] -> out[K] (deterministic).
void dense_norms2(int K, size_t len, const double2* V, double* out, cudaStream_t st);
// Copy helper
void dense_copy(double2* dst, const double2* src, size_t n, cudaStream_t st);
// Column-wise TPA preconditioner: out[k][i][g] = in * scale_i / (kin[k][g] + alpha[k][i]).
void dense_tpa(int K, int p, int n_max, const double* kin, const double* alpha, const double2* in, double2* out,
               bool unit_gain, cudaStream_t st);
// alpha[k][i] = sum_g kin[k][g] |phi[k][i][g]|^2
void dense_kinetic_alpha(int K, int p, int n_max, const double* kin, const double2* phi, double* alpha,
                         cudaStream_t st);
// Diagonal scaling of projections: P[k][j][i] *= d[j]
void dense_scale_rows(int K, int m, int n, double2* P, const double* d, cudaStream_t st);
// Per-column norms of a p x p matrix block etc.
void dense_kin_energy(int K, int p, int n_max, const double* kin, const double2* phi, const double* kw, double occ,
                      double* partials, cudaStream_t st);

// ---- FOM projected solves (dense_kernels.cu)
// Solve (A[k] - s[k][m] I) y = c for every (k, m): A Hermitian q x q (lda), c/y columns of q x p
// (ldc), by one Householder tridiagonalisation per k and p tridiagonal solves.
// prec 0: FP64 arithmetic, 1: FP32 arithmetic (FP64 in and out).  work: fom_shifted_work bytes
// (reflectors, right-hand sides and tridiagonal factors of every k).  info[k * p + m] = 1 when a
// shifted tridiagonal matrix is exactly singular (that y is set to zero); may be null.
size_t fom_shifted_work(int K, int p, int q, int prec);
void fom_shifted_solve(int K, int p, int q, const double2* A, int lda, size_t sA, const double* s,
                       const double2* C, int ldc, size_t sC, double2* Y, void* work, const int* kactive,
                       int* info, int prec, cudaStream_t st);
// A[k][i][j] for i in [q0, q0 + p) and j < q0: conj of A[k][j][i] (Hermitian mirror).
void fom_mirror(int K, int q0, int p, double2* A, int lda, size_t sA, const int* kactive, cudaStream_t st);
// Rows of A with zero new columns: A[k][q0 + i][q0 + i] = 1 + max_m |shifts[k][m]| for i < nzero[k].
void fom_pad_diag(int K, int q0, int p, double2* A, int lda, size_t sA, const int* nzero, const double* shifts,
                  cudaStream_t st);

}  // namespace eacg
