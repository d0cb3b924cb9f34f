/*
 * libeacg: energy-adaptive Riemannian conjugate gradient (eARCG) minimisation of the
 * Kohn-Sham energy on the Stiefel manifold in a periodic plane-wave basis, on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Peterseim, Pueschel, Stykel, "Energy-Adaptive Riemannian Conjugate Gradient
 * Method for Density Functional Theory", arXiv 2503.16225.  Problem statement
 * min_{Phi in St} E(Phi): Sec. 2.1, Eq. (2.2); discrete form on the product of
 * Stiefel manifolds over k-points: Sec. 5.1, Eq. (5.1).
 *
 * Conventions shared by every entry point
 *   - Coefficient blocks ("psi" buffers) are complex double (interleaved re, im),
 *     laid out [K][p][n_max]: k-point major, then band, then plane-wave index in the
 *     canonical basis order of eacg_get_basis; entries n_k .. n_max-1 of every band are
 *     zero on input and are written as zero on output.  Column i of block k is orbital
 *     i of Phi_k in C^{n_k x p} (Sec. 5.1).
 *   - Real-space grids are double [jx][jy][jz] (z fastest), r_j = a j / N.
 *   - Small matrices (Lambda) are complex double [K][p][p], column-major.
 *   - Pointers named *_dev are device pointers (caller-owned, valid for the call);
 *     *_host are host pointers.  Calls are ordered on the system's CUDA stream and
 *     return after the stream has been synchronised.
 *   - Every call returns eacg_status; no call aborts or throws.  eacg_last_error gives
 *     a message for the last failing call of a system.  After a failure other than
 *     EACG_ENOTCONV or EACG_ELINESEARCH the system keeps its state from before the call.
 *   - One system is not thread-safe; distinct systems are independent.
 */
#ifndef EACG_H
#define EACG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eacg_system eacg_system;

/* Band limits.  The transforms, the density, the potential, H application and the energy
 * evaluation take up to EACG_MAX_BANDS bands per k-point.  The calls that decompose p x p
 * matrices (eacg_set_psi, eacg_step, eacg_solve, eacg_solve_host, eacg_ea_gradient,
 * eacg_retract, eacg_scf_guess: polar factor, inverse, Lyapunov solve, rank-revealing QR,
 * projected FOM solves) run one CTA per k-point; up to 64 bands (80 for some of them) the p x p
 * blocks sit in shared memory, above that in a global scratch owned by the system.  They
 * return EACG_EUNSUPPORTED for p > EACG_MAX_BANDS_DENSE. */
#define EACG_MAX_BANDS 1024
#define EACG_MAX_BANDS_DENSE 512

typedef enum {
  EACG_OK = 0,
  EACG_EINVAL = 1,        /* invalid argument or model                          */
  EACG_ENOMEM = 2,        /* device allocation failed                           */
  EACG_ECUDA = 3,         /* a CUDA runtime call or launch failed               */
  EACG_EBREAKDOWN = 4,    /* singular projected system in the block FOM         */
  EACG_ENONCOERCIVE = 5,  /* reserved: shifted Hamiltonian not coercive         */
  EACG_ELINESEARCH = 6,   /* step-size search hit its trial cap (Algorithm 2)   */
  EACG_ENAN = 7,          /* non-finite energy or residual                      */
  EACG_ENOTCONV = 8,      /* outer iteration cap reached before the tolerance   */
  EACG_EUNSUPPORTED = 9   /* size outside what this build supports              */
} eacg_status;

/* Synthetic crystal (cubic cell) and its discretisation (Sec. 1, Eq. (1.1); Sec. 5.1).
 * Local part: V(G) = sum_a -4 pi Z_a / (Omega |G|^2) exp(-|G|^2 rc_a^2 / 4) e^{-i G.R_a}.
 * Nonlocal part: nproj_per_atom in {0, 1, 4} L2-normalised Gaussian projectors
 * (s, px, py, pz) of width proj_width with couplings D[a][0] (s) and D[a][1] (p). */
typedef struct {
  double a;                /* cubic cell edge (bohr)                           */
  int natoms;
  const double* pos;       /* host, natoms x 3 cartesian (bohr)                */
  const int* Z;            /* host, natoms                                     */
  const double* rc;        /* host, natoms (bohr)                              */
  int nproj_per_atom;      /* 0, 1 or 4                                        */
  double proj_width;       /* bohr                                             */
  const double* D;         /* host, natoms x 2 (Ha)                            */
  double ecut;             /* basis: 1/2 |k+G|^2 <= ecut (Ha)                  */
  int N;                   /* FFT grid edge: 8, 12, 16, 20, 24, 32, 36, 40, 48, 64, 72, 80, 96 or
                            * 128; at N = 128 only FP32 transforms exist (precision 1 of
                            * eacg_density, eacg_apply_H, eacg_energy); FP64-accurate ones return
                            * EACG_EUNSUPPORTED */
  int nbands;              /* p: occupied orbitals per k-point, <= EACG_MAX_BANDS */
  int nk;                  /* K: number of k-points                            */
  const double* kfrac;     /* host, K x 3 fractional coordinates (units of 2 pi / a) */
  const double* kweight;   /* host, K weights (sum 1)                          */
  int hartree;             /* 1: Hartree term on                               */
  int xc;                  /* 0: none; 1: Slater exchange; 2: LDA = Slater exchange
                            * + spin-unpolarised Perdew-Wang 1992 correlation
                            * (DFTK's LDA model of the experiments, Sec. 5.3)     */
  double occ;              /* occupation f of every orbital (2: spin paired)   */
} eacg_model;

/* Iteration constants (defaults: Sec. 5.2).  precision: 0 = FP64 throughout,
 * 1 = mixed (FP32 transforms while ||R||_F > switch_res, FP64 afterwards). */
typedef struct {
  double mu;          /* shift correction, Sigma = Lambda - mu I (Sec. 4.3): 0.01  */
  double res_tol;     /* stop when ||R||_F <= res_tol: 1e-8                        */
  double fom_rtol;    /* relative Sylvester residual of the block FOM: 2.5e-2      */
  double delta, sigma, gamma, eps;  /* Algorithm 2: 0.05, 0.1, 0.5, 1e-12          */
  double warm_res;    /* warm-up phase ends at ||R||_F <= warm_res: 1e-2          */
  double switch_res;  /* mixed precision: FP64 from ||R||_F <= switch_res: 1e-3    */
  int max_outer;      /* 300 */
  int max_warm;       /* 100 */
  int max_fom;        /* 50  */
  int max_ls;         /* 30  */
  int precision;      /* 0 FP64, 1 mixed */
  int graphs;         /* 1: the FOM's block H application is replayed as a CUDA graph per system
                       * (captured on its second call with the same buffers; needs a stream of
                       * the system's own, not the legacy default stream); 0: direct launches.
                       * Results are identical either way.  Default 1 */
  int fft_plan;       /* line-FFT plan of the transforms: -1 picks the faster of the compiled
                       * plans for this grid by timing both on the system at set-up (autotune);
                       * 0 or 1 forces a plan (one that does not exist for N falls back to 0).
                       * Default -1 */
  int method;         /* 0: EARCG (Algorithm 3); 1: EARGD, the paper's gradient-descent comparator
                       * (same warm-up; then eta = -G with an alternating Barzilai-Borwein step
                       * and Zhang-Hager non-monotone backtracking, rho 0.85, delta 1e-4).
                       * Default 0 */
  int tensor_cores;   /* 1: where nproj >= 128 and nbands is a multiple of 16, the projector
                       * overlaps of complex64 blocks (FP32 phase, FP32 FOM; eacg_overlap_c64,
                       * method 1) and the back-projection of FP32-phase evaluations (in column
                       * blocks of at most 256 bands; eacg_backproject_c64, method 1) on the
                       * tensor cores; 0: SIMT FP32.
                       * Default 1 */
  int df_transforms;  /* 1: the FP64-accurate transforms (FP64 mode, the FP64 phase of the mixed
                       * mode and the density) run in double-float arithmetic, each value an
                       * unevaluated sum of two FP32 numbers (about 48 significant bits, 1e-14
                       * relative error on a transform), on GB300's FP32 pipe, which is 64 times
                       * wider than its FP64 pipe; 0: plain FP64 arithmetic.  Default 1 */
} eacg_params;

typedef struct {
  double E;            /* energy after the step (Ha, without ion-ion term)        */
  double rnorm;        /* ||R||_F = (sum_k ||H Phi_k - Phi_k Lambda_k||_F^2)^1/2   */
  double tau;          /* accepted step size                                       */
  double beta;         /* CG parameter used for the next direction                 */
  int fom_iters_max;   /* largest per-k FOM iteration count at the new point       */
  int ls_trials;       /* trial points of Algorithm 2 in this step                 */
  int phase;           /* 0 warm-up, 1 energy-adaptive                             */
  int precision;       /* precision used for this step's transforms                */
  int converged;       /* 1 when rnorm <= res_tol                                  */
  long long h_band_apps; /* cumulative band applications of H (one band at one k = 1) */
} eacg_step_info;

typedef struct {
  double E;
  double rnorm;
  int iterations;
  int warm_iterations;
  int status;          /* eacg_status of the solve */
  int ls_trials;       /* total trial points */
  long long h_band_apps;
} eacg_result;

/* Defaults of Sec. 5.2 and the readings documented with the library. */
void eacg_default_params(eacg_params* prm);

/* Device bytes a system of this model needs (HBM admission), excluding the Krylov
 * blocks of the FOM, which grow with its iteration count (returned in *fom_bytes_per_iter
 * when not NULL).  Returns 0 for an invalid model. */
size_t eacg_bytes_required(const eacg_model* model, const eacg_params* prm, size_t* fom_bytes_per_iter);

/* Builds the basis (Sec. 5.1), local potential and projectors on the device.
 * stream: a cudaStream_t (NULL = legacy default stream).  *out owns all device state.
 * While a call on the system runs, nothing else may be enqueued on its stream: the FOM's
 * block H application is captured from that stream into a CUDA graph, and work of another
 * system on the same stream would be captured with it.  Concurrent systems therefore need
 * streams of their own (eacg_stream_create gives such streams). */
eacg_status eacg_create_system(const eacg_model* model, const eacg_params* prm, void* stream, eacg_system** out);
/* Synchronises the system's stream and frees every device and pinned host buffer the system
 * owns; NULL is ignored.  Resource management only, the paper has no counterpart. */
void eacg_destroy(eacg_system* sys);
/* Message of the last failing call on sys ("null system" for NULL); owned by the system and
 * valid until its next call.  Error reporting only, the paper has no counterpart. */
const char* eacg_last_error(const eacg_system* sys);

/* n_k per k-point (nk_host: K ints, may be NULL), n_max = max n_k, union column count. */
eacg_status eacg_get_dims(const eacg_system* sys, int* nk_host, int* n_max, int* ncols);
/* Line-FFT plan variant (0 or 1) the system uses for its FP64 and its FP32 transforms: the
 * one eacg_params.fft_plan forced, else the one the set-up timing found faster (variant 0
 * where the grid size has a single plan).  Implementation detail of the transforms; the
 * paper has no counterpart. */
eacg_status eacg_get_plans(const eacg_system* sys, int* plan64, int* plan32);
/* Number of CUDA-graph replays of the FOM's block H application on this system so far (see
 * eacg_params.graphs).  Graphs need a stream of the system's own: on the legacy default stream
 * (stream NULL) capture is impossible and the system launches directly.  The paper has no
 * counterpart. */
long long eacg_graph_launches(const eacg_system* sys);
/* Tile variant (row groups per CTA: 1, 2 or 4) of the block-overlap kernel A^H B for an m x n
 * result over L rows in the given block precision (0 complex128, 1 complex64): the fastest one
 * timed when a system using that shape was set up, 4 for shapes never tuned.  Process-wide;
 * the paper has no counterpart. */
int eacg_gemm_tile(int m, int n, int L, int precision);
/* Forces tile variant 1, 2 or 4 for every shape of every system in the process (results change
 * only by rounding order); 0 returns to the tuned choices.  EACG_EINVAL for other values.  For
 * tests and tuning experiments; the paper has no counterpart. */
eacg_status eacg_force_gemm_tile(int groups);
/* Integer triples m (G = 2 pi m / a) of the basis: m_dev int32 [K][n_max][3]
 * (rows >= n_k unspecified).  Canonical order: (mx, my, mz) lexicographic, mz fastest. */
eacg_status eacg_get_basis(const eacg_system* sys, int* m_dev);

/* Sets the iterate to pf(psi) (polar factor, Eq. (3.1)) of a raw block and resets the
 * CG state; the next eacg_step starts Algorithm 3 from it. */
eacg_status eacg_set_psi(eacg_system* sys, const double* psi_dev);
/* Copies the current iterate Phi = (Phi_k) of the product of Stiefel manifolds (Sec. 5.1,
 * Eq. (5.1)) into psi_dev_out, a caller-owned device buffer [K][p][n_max] in the block
 * layout above (orthonormal columns per k; entries n_k .. n_max-1 zero).  EACG_EINVAL before
 * the first eacg_set_psi. */
eacg_status eacg_get_psi(eacg_system* sys, double* psi_dev_out);

/* Density rho(r_j) = sum_k w_k f sum_i |u_ik(r_j)|^2 of an orthonormal block (Sec. 1),
 * written to rho_dev (N^3, may be NULL); updates the system's potential
 * V = V_loc + V_H(rho) + V_x(rho) used by eacg_apply_H.  precision as in eacg_params. */
eacg_status eacg_density(eacg_system* sys, const double* psi_dev, double* rho_dev, int precision);
/* Current total potential (N^3). */
eacg_status eacg_get_potential(eacg_system* sys, double* vtot_dev);

/* hpsi = H psi with the current potential: 1/2 |k+G|^2 psi + local part by the FFT pair
 * + B D B^* psi (Eq. (1.4) in the DFTK form of Sec. 5.2).  psi and hpsi must not overlap. */
eacg_status eacg_apply_H(eacg_system* sys, const double* psi_dev, double* hpsi_dev, int precision);

/* Full evaluation at an orthonormal block: density, potential, H Phi, Lambda =
 * herm(Phi^* H Phi) (Eq. (2.6)), residual R = H Phi - Phi Lambda, energy terms.
 * terms_host[6] = {kinetic, local, Hartree, exchange-correlation, nonlocal, total}.  lam_dev and
 * res_dev may be NULL.  *rnorm = ||R||_F. */
eacg_status eacg_energy(eacg_system* sys, const double* psi_dev, double* terms_host, double* lam_dev,
                        double* res_dev, double* rnorm, int precision);

/* Energy-adaptive gradient G = Phi - X (Phi^* X)^{-1}, H X - X (Lambda - mu I) = Phi solved
 * per k by the preconditioned block FOM (Sec. 5.2, Algorithm 4).  fom_iters_host: K ints
 * (may be NULL). */
eacg_status eacg_ea_gradient(eacg_system* sys, const double* psi_dev, double* g_dev, int* fom_iters_host,
                             int precision);

/* Polar retraction Phi+ = pf(Phi + tau eta) (Eq. (3.2)) and the transport
 * T_{tau eta}(eta) = eta S^{-1} - tau Phi+ [[eta S^{-1}, eta S^{-1}]] (Sec. 3.2). */
eacg_status eacg_retract(eacg_system* sys, const double* phi_dev, const double* eta_dev, double tau,
                         double* phi_out_dev, double* teta_out_dev);

/* Live kernel timing (no counterpart in the paper; used for roofline reports).
 * eacg_profile_enable(sys, 1) clears and starts recording CUDA events around the main
 * kernels of the Hamiltonian application, density, potential and FOM solves on the
 * system's stream; eacg_profile_read writes up to max entries (name with the precision of
 * the variant, launches, summed device milliseconds, summed algorithmic bytes, summed
 * algorithmic FLOPs (5 N log2 N per N-point transform), summed work units = band
 * applications) and returns their number (negative eacg_status on error).  Reading clears
 * the records. */
typedef struct {
  char name[24];
  long long launches;
  double ms;
  double bytes;
  double flops;
  double units;
} eacg_kernel_stat;
eacg_status eacg_profile_enable(eacg_system* sys, int on);
int eacg_profile_read(eacg_system* sys, eacg_kernel_stat* out, int max);
/* Number of kernels this library has launched in the process so far. */
long long eacg_launch_count(void);
/* A new non-blocking CUDA stream on the current device (*stream, a cudaStream_t), for a system
 * of its own; eacg_stream_destroy synchronises and destroys it.  Stream management for
 * concurrent systems; the paper has no counterpart.  EACG_ECUDA if the runtime refuses. */
eacg_status eacg_stream_create(void** stream);
eacg_status eacg_stream_destroy(void* stream);

/* Allocation-free block overlaps (the paper has no counterpart; this serves callers that
 * cannot allocate device memory, e.g. code running inside a memory pool or framework that
 * owns all device allocations and forbids cudaMalloc).  Computes c_k = a_k^* b_k for k < K, where
 * a_k, b_k are n x p complex double blocks (column-major, ld n, laid out [K][p][n]) and c_k
 * is p x p column-major ([K][p][p]); all three are caller-owned device buffers.  Needs no
 * system and calls no allocator: its scratch is a fixed device array of
 * EACG_NOALLOC_MAX_PARTIALS complex doubles (8 MiB), held by every GPU that loads the library
 * until the process exits, and shared by all calls.  Returns EACG_EINVAL when
 * K * ceil(n / 1024) * p * p exceeds EACG_NOALLOC_MAX_PARTIALS, K exceeds 65535 (one grid row
 * per k-point) or an argument is invalid.
 * The first call on a device looks up the scratch address for that device (make it before
 * any stream capture).  stream: cudaStream_t or NULL; the call returns after synchronising
 * it.  Calls that overlap on the GPU (other host threads or streams) race on the scratch. */
#define EACG_NOALLOC_MAX_PARTIALS 524288
eacg_status eacg_overlap_noalloc(int K, int n, int p, const double* a_dev, const double* b_dev, double* c_dev,
                                 void* stream);

/* Block overlaps of complex64 blocks, the contraction of the projector overlaps P = B^* Psi
 * of the nonlocal term (Sec. 5.1) in the FP32 phase: c_k = a_k^* b_k for k < K, where a_k is
 * L x m and b_k is L x n complex64 (column-major, ld L, laid out [K][m][L] and [K][n][L]) and
 * c_k is m x n complex double (column-major, [K][n][m]); caller-owned device buffers.
 * method 0: SIMT FP32 products; 1: tensor cores (tcgen05, each FP32 operand split into two
 * TF32 parts, three TF32 products per product), for m >= 128 and n a multiple of 16, else
 * EACG_EUNSUPPORTED.  Both accumulate in FP32 within chunks of 1024 rows and sum the chunks in
 * FP64 in a fixed order.  Allocates and frees its own scratch; stream: cudaStream_t or NULL;
 * returns after synchronising it.  EACG_EINVAL for negative sizes or null buffers.
 * The tensor-core kernel waits on its MMAs with bounded polls; a CTA whose wait gives up
 * writes NaN for its tile and counts itself in a per-device counter, and the call then returns
 * EACG_ECUDA (also when a tensor-core call running beside it on the same device gave up). */
eacg_status eacg_overlap_c64(int K, int L, int m, int n, const float* a_dev, const float* b_dev, double* c_dev,
                             int method, void* stream);

/* Back-projection of the nonlocal term (Sec. 5.1: H Psi += B (D P)) for complex64 projector
 * blocks: c_k += a_k q_k for k < K, a_k L x m complex64 ([K][m][L], column-major, ld L),
 * q_k m x n complex double ([K][n][m]), c_k L x n complex double ([K][n][L]); caller-owned
 * device buffers.  method 0: SIMT FP32 products (FP32 accumulation), result added in FP64;
 * 1: tensor cores (tcgen05, 3 x TF32 split, accumulation runs of 48 MMAs summed with
 * round-to-nearest FP32 adds) for 16 <= n <= 256 with n a multiple of 16, else
 * EACG_EUNSUPPORTED.  stream: cudaStream_t or NULL; returns after synchronising it.
 * EACG_EINVAL for negative sizes or null buffers.
 * A tensor-core wait that gives up is reported as in eacg_overlap_c64 (NaN added to the
 * CTA's rows, EACG_ECUDA). */
eacg_status eacg_backproject_c64(int K, int L, int m, int n, const float* a_dev, const double* q_dev, double* c_dev,
                                 int method, void* stream);

/* Initial guess of the experiments (Sec. 5.2): self-consistent field iterations until the
 * density difference of two successive iterates is below drho_tol (0.1 in the paper).  The
 * first input density is that of polar(psi0) (psi0: caller's device buffer [K][p][n_max]);
 * each step minimises the band energy f sum_k w_k tr(Phi_k^* H[rho_in] Phi_k) with the
 * potential of the input density held fixed (the same warm-up and energy-adaptive iterations
 * as eacg_step, params.precision applies) until ||H Phi - Phi Lambda||_F <= eig_tol, takes
 * rho_out = rho(Phi) and d = ||rho_out - rho_in||_2 = (integral over the cell of
 * (rho_out - rho_in)^2)^{1/2}; d < drho_tol ends it with Phi as the system's iterate, else
 * rho_in <- rho_in + alpha (rho_out - rho_in) (simple mixing, 0 < alpha <= 1).  *steps_out
 * (may be NULL) = steps taken; history_host (may be NULL, max_scf doubles) receives d per step.
 * Afterwards eacg_step / eacg_solve continue from Phi with its own density and potential.
 * EACG_ENOTCONV when max_scf steps do not reach drho_tol (Phi is the last step's); errors of
 * an inner step are returned as they are; EACG_EINVAL for invalid arguments. */
eacg_status eacg_scf_guess(eacg_system* sys, const double* psi0_dev, double drho_tol, double alpha, int max_scf,
                           double eig_tol, int* steps_out, double* history_host);

/* One outer iteration of Algorithm 3 (warm-up iterations first, see eacg_params). */
eacg_status eacg_step(eacg_system* sys, eacg_step_info* info);
/* One outer iteration of Algorithm 3 on each of nsys distinct systems, taken together (the
 * serving form of eacg_step; Algorithm 3 itself is per system and unchanged).  Every system
 * steps in a host thread of its own on its own stream; the plane-wave transforms of the H
 * applications and densities that several systems reach at the same time are launched
 * together, one launch per transform kernel over a table of (system, band) work items, for the
 * systems that share the grid size, line plan and transform precision.  A system that reaches
 * a transform waits at most window_us microseconds for the others to reach one.  Each band's
 * arithmetic is that of an unbatched launch, so every result equals the one of eacg_step bit
 * for bit.  infos (nsys entries) and statuses (nsys entries, each system's own eacg_status) may
 * be NULL.  Returns EACG_OK when every step succeeded, else the first failing system's status;
 * EACG_EINVAL for a NULL or repeated system or a negative window, EACG_EUNSUPPORTED for
 * p > EACG_MAX_BANDS_DENSE.  The FOM's graph replay is not used inside batched steps. */
eacg_status eacg_step_many(eacg_system* const* sys, int nsys, eacg_step_info* infos, int* statuses, int window_us);
/* Process-wide batching of eacg_step: with window_us >= 0, concurrent eacg_step calls from
 * different host threads (e.g. a serving loop with one thread per resident system) batch their
 * transforms as eacg_step_many does, each waiting at most window_us microseconds; window_us = -1
 * turns it off (the default).  Steps already running keep the setting they started with.
 * EACG_EINVAL for window_us < -1.  Serving utility; the paper has no counterpart. */
eacg_status eacg_batching(int window_us);
/* Process-wide counts since start: batched transform groups launched by eacg_step_many and
 * batched eacg_step calls (*groups) and the system requests they covered (*members; a group of
 * one is a system that found no partner within the window).  Either pointer may be NULL. */
eacg_status eacg_batch_counts(long long* groups, long long* members);
/* Algorithm 3 to convergence: iterates eacg_step from the current iterate until the
 * residual ||R||_F of Sec. 5.3 is <= res_tol (status EACG_OK) or max_outer iterations
 * (EACG_ENOTCONV); E, ||R||_F and the counts in *out (out may not be NULL).  Errors of a step
 * end the solve with that step's status. */
eacg_status eacg_solve(eacg_system* sys, eacg_result* out);
/* eacg_set_psi + eacg_solve + eacg_get_psi (Algorithm 3 from pf(psi0)) through host buffers
 * (copies on the system's stream; psi0_host and psi_out_host are [K][p][n_max] complex
 * double, may alias). */
eacg_status eacg_solve_host(eacg_system* sys, const double* psi0_host, double* psi_out_host, eacg_result* out);

#ifdef __cplusplus
}
#endif
#endif
