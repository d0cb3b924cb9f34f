// libeacg C ABI and host-side driver of the eARCG iteration (arXiv 2503.16225).
//
// The driver only sequences kernels and takes the scalar decisions of the step-size
// search (Algorithm 2), the CG parameter (Sec. 3.4) and the per-k stopping of the block
// FOM (Algorithm 4); every vector and matrix operation runs in the kernels of
// grid_kernels.cu and dense_kernels.cu on the system's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "../../include/eacg.h"
#include "kernels.h"

using namespace eacg;

namespace {

const double2 ONE = {1.0, 0.0};
const double2 ZERO = {0.0, 0.0};
const double2 MONE = {-1.0, 0.0};
inline double2 cr(double x) { return make_double2(x, 0.0); }

struct Status {
  eacg_status code = EACG_OK;
};

}  // namespace

namespace eacg {
void small_pivchol(int K, int p, const double2* G, const double* ref, double tol, double2* M, int* nzero,
                   const int* kactive, cudaStream_t st, void* scratch);
void small_max_diag(int K, int p, const double2* G, double* out, cudaStream_t st);
void small_put_herm_block(int K, int p, const double2* src, double2* A, int lda, size_t sA, int q0, cudaStream_t st);
void small_take_y(int K, int q, int qcap, int p, const double2* Y, double2* Yf, const int* take, cudaStream_t st);
void small_conj_transpose(int K, int p, const double2* A, double2* out, cudaStream_t st);
void small_add_herm(int K, int p, const double2* A, double s, double2* out, cudaStream_t st);
void small_sqrt_vals(int K, int p, const double* w, double* out, cudaStream_t st);
}  // namespace eacg

struct eacg_system {
  // ---- model
  int N = 0, K = 0, p = 0, natoms = 0, npa = 0, nproj = 0, hartree = 1, xc = 1;
  double a = 0, omega = 0, b = 0, ecut = 0, occ = 2, width = 0.7, thr = 0;
  std::vector<double> kfrac, kw, pos, Z, rc, D, dvec;
  eacg_params prm{};
  cudaStream_t st = nullptr;
  std::string err;
  // ---- basis
  std::vector<int> nk;
  int n_max = 0, ncols = 0, ny = 0;
  GridCtx g{};
  size_t blk = 0;  // elements of one [K][p][n_max] block
  // ---- device allocations (freed in destroy)
  std::vector<void*> allocs;
  int *d_nk = nullptr, *d_m = nullptr, *d_xmap = nullptr, *d_cmapy = nullptr, *d_rowmask = nullptr, *d_ylist = nullptr;
  double *d_kfrac = nullptr, *d_kin = nullptr, *d_kw = nullptr, *d_pos = nullptr, *d_Z = nullptr, *d_rc = nullptr;
  double *d_dvec = nullptr, *d_bw = nullptr;
  double2* d_tw64 = nullptr;
  float2* d_tw32 = nullptr;
  double *d_vloc = nullptr, *d_vtot = nullptr, *d_rho = nullptr, *d_vh = nullptr, *d_partial = nullptr;
  float* d_vtot32 = nullptr;
  float2* d_vtotdf = nullptr;         // double-float copy of V_tot (hi, lo)
  void* d_twdf = nullptr;             // double-float twiddles
  double2* d_fft3 = nullptr;
  double2 *d_B = nullptr, *d_P = nullptr, *d_P2 = nullptr;
  float2* d_B32 = nullptr;
  void* d_tbuf = nullptr;
  int rho_groups = 1;
  // blocks
  double2 *phi = nullptr, *hphi = nullptr, *res = nullptr, *eta = nullptr, *gv = nullptr, *teta = nullptr,
          *tg = nullptr, *psi_t = nullptr, *phi_t = nullptr, *hphi_t = nullptr, *res_t = nullptr, *teta_t = nullptr,
          *tmp1 = nullptr, *tmp2 = nullptr, *tmp3 = nullptr, *Xb = nullptr, *Cb = nullptr, *fvt = nullptr,
          *fwt = nullptr, *c32 = nullptr;
  // small [K][p][p]
  double2 *lam = nullptr, *lam_t = nullptr, *sm1 = nullptr, *sm2 = nullptr, *sm3 = nullptr, *evec = nullptr,
          *evec_t = nullptr, *sinv_t = nullptr, *sig = nullptr, *sigv = nullptr, *sigvh = nullptr;
  double *eval = nullptr, *eval_t = nullptr, *alpha = nullptr, *sqd = nullptr, *lref = nullptr;
  unsigned char* ppscr = nullptr;  // global scratch of the p x p kernels (large p only)
  double2* cn_work = nullptr;
  size_t cn_elems = 0;
  double* d_red = nullptr;    // reduction scratch
  double* d_esum = nullptr;   // block sums of the grid energy terms
  double* d_out = nullptr;    // scalars copied to the host
  double* h_out = nullptr;    // pinned
  int *d_kactive = nullptr, *d_nzero = nullptr, *d_info = nullptr, *d_take = nullptr;
  int* h_int = nullptr;       // pinned
  // FOM Krylov storage (grown on demand)
  int qcap = 0;
  double2 *fV = nullptr, *fW = nullptr, *fA = nullptr, *fC = nullptr, *fY = nullptr, *fYt = nullptr, *fYf = nullptr,
          *fwork = nullptr;
  size_t fwork_elems = 0;
  size_t fom_es = sizeof(double2);  // element bytes of the Krylov blocks V, W
  // ---- iteration state
  int fresh = 1, have_psi = 0, phase = 0, iter = 0, warm_iter = 0, cur_prec = 0;
  int eval_prec = 0;  // transform precision of the evaluation of the current point
  double E = 0, rnorm = 0, tau = 1, rg = 0;
  double nm_C = 0, nm_Q = 1;  // EARGD: non-monotone reference value and its weight
  int ea_steps = 0;           // EARGD: energy-adaptive steps taken (alternates the BB formula)
  double eterms[5] = {0, 0, 0, 0, 0};
  long long h_apps = 0;
  int last_fom_max = 0;
  int ls_total = 0;
  // ---- live kernel timing
  struct ProfRec {
    int slot;
    cudaEvent_t a, b;
    double bytes, flops, units;
  };
  bool prof_on = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  struct ProfMs {  // profile records already read back (graph replays)
    int slot;
    double ms, bytes, flops, units;
  };
  std::vector<ProfMs> prof_ms;
  // ---- CUDA graph of the FOM's block H application, one per block precision
  struct HGraph {
    const void* in = nullptr;
    const void* out = nullptr;
    const void* ka = nullptr;
    const void* cnw = nullptr;
    int direct = 0;                   // direct calls with this key (capture on the second)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;            // kernel nodes of the graph
    std::vector<ProfRec> recs;        // capture-time profile records; events owned by the graph
    bool pending = false;             // a replay whose events were recorded but not yet read
  };
  HGraph hg[2];
  HGraph* cap = nullptr;              // graph being captured (profile events go to it)
  long long graph_launches = 0;       // replays of captured graphs
  bool graphs_off = false;            // set when capture is not possible on this system
  // SCF initial guess: evaluations keep the potential (built from the mixed input density) and
  // minimise the band energy f sum_k w_k tr(Phi_k^* H Phi_k) of that fixed Hamiltonian
  bool frozen = false;
  double* d_rho_in = nullptr;         // SCF input density (allocated by the first SCF call)
  bool tc_proj = false;               // FP32 projector overlaps on the tensor cores
  cudaEvent_t ev_sync = nullptr;      // blocking-sync event of the host waits (stream_wait)
};

namespace {
std::atomic<long long> g_launches{0};
// slots of the FP64 variants; the FP32 variant of a slot is slot + P_F32
const char* const PROF_NAMES[] = {"xpass_inv_f64",  "plane_h_f64",  "xpass_fwd_f64", "nonlocal_f64",
                                  "xpass_rho_f64",  "plane_rho_f64", "fom_solve_f64", "potential",
                                  "xpass_inv_f32",  "plane_h_f32",  "xpass_fwd_f32", "nonlocal_f32",
                                  "xpass_rho_f32",  "plane_rho_f32", "fom_solve_f32", "nonlocal_eval_f32",
                                  "fom_setup",      "fom_residual", "fom_orth",      "fom_block",
                                  "trial_retract",  "fom_final",    "unused2",       "unused3"};
enum { P_XINV = 0, P_PLANE_H, P_XFWD, P_NONLOCAL, P_XINV_RHO, P_PLANE_RHO, P_FOMSOLVE, P_POT, P_F32,
       P_NONLOCAL32 = P_F32 + 7, P_FOM_SETUP = 16, P_FOM_RES, P_FOM_ORTH, P_FOM_BLOCK, P_TRIAL_RET, P_FOM_FINAL, P_NSLOTS = 24 };
// algorithmic FLOPs of one N-point complex transform (5 N log2 N convention)
inline double fft_flops(int N) { return 5.0 * N * std::log2((double)N); }

cudaEvent_t prof_event(eacg_system* s) {
  if (s->evused == s->evpool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    s->evpool.push_back(e);
  }
  return s->evpool[s->evused++];
}
}  // namespace

void eacg::count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
namespace {
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace

namespace {
std::mutex g_smem_mu;
std::map<std::pair<int, const void*>, size_t> g_smem_set;
}  // namespace

void eacg::ensure_smem(const void* func, size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_smem_mu);
  size_t& cur = g_smem_set[{dev, func}];
  if (bytes > cur) {
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
      cur = bytes;
  }
}

// Records CUDA events around a kernel (group) when profiling is on.  While a graph is being
// captured the events always go into the graph (they become event-record nodes whose times
// are read back after each profiled replay).
namespace {
cudaEvent_t cap_event(eacg_system*) {
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
// While capturing, an event record must be marked external to become a node whose time can be
// read after each replay (a plain record would only order captured work).
void record_event(eacg_system* s, cudaEvent_t e) {
  if (s->cap)
    cudaEventRecordWithFlags(e, s->st, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s->st);
}
}  // namespace
#define PROF_RUN(slot, bytes_, flops_, units_, ...)                                       \
  do {                                                                            \
    cudaEvent_t a_ = nullptr;                                                     \
    const bool rec_ = s->prof_on || s->cap;                                       \
    if (rec_) {                                                                   \
      a_ = s->cap ? cap_event(s) : prof_event(s);                                 \
      record_event(s, a_);                                                        \
    }                                                                             \
    __VA_ARGS__;                                                                  \
    if (rec_) {                                                                   \
      cudaEvent_t b_ = s->cap ? cap_event(s) : prof_event(s);                     \
      record_event(s, b_);                                                        \
      (s->cap ? s->cap->recs : s->prof)                                           \
          .push_back({(slot), a_, b_, (double)(bytes_), (double)(flops_), (double)(units_)}); \
    }                                                                             \
  } while (0)

// ============================================================================ helpers
#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      s->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return EACG_ECUDA;                                                          \
    }                                                                             \
  } while (0)
#define CKL(s)                                                                    \
  do {                                                                            \
    cudaError_t e_ = cudaGetLastError();                                          \
    if (e_ != cudaSuccess) {                                                      \
      (s)->err = std::string("kernel launch: ") + cudaGetErrorString(e_);         \
      return EACG_ECUDA;                                                          \
    }                                                                             \
  } while (0)
#define TRY(x)                        \
  do {                                            \
    eacg_status st_ = (x);                        \
    if (st_ != EACG_OK) return st_;               \
  } while (0)

template <typename P>
static eacg_status dalloc(eacg_system* s, P** ptr, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->err = "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e);
    return EACG_ENOMEM;
  }
  cudaMemsetAsync(p, 0, bytes, s->st);
  s->allocs.push_back(p);
  *ptr = reinterpret_cast<P*>(p);
  return EACG_OK;
}

static void dfree(eacg_system* s, void* p) {
  if (!p) return;
  auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
  if (it != s->allocs.end()) s->allocs.erase(it);
  cudaFree(p);
}

// Waits for the system's stream.  A short poll (with yields) covers the usual sub-millisecond
// waits of small problems; after it the thread blocks on an event created with
// cudaEventBlockingSync instead of spinning, so that the host threads of many concurrent
// systems do not keep every core busy polling the GPU.
static cudaError_t stream_wait(eacg_system* s) {
  if (!s->ev_sync) return cudaStreamSynchronize(s->st);
  cudaError_t e = cudaEventRecord(s->ev_sync, s->st);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 64; ++i) {
    e = cudaEventQuery(s->ev_sync);
    if (e != cudaErrorNotReady) return e;
    std::this_thread::yield();
  }
  return cudaEventSynchronize(s->ev_sync);
}

static eacg_status sync_read(eacg_system* s, int ndouble) {
  CK(cudaMemcpyAsync(s->h_out, s->d_out, sizeof(double) * ndouble, cudaMemcpyDeviceToHost, s->st));
  CK(stream_wait(s));
  return EACG_OK;
}

// ============================================================================ model set-up
static eacg_status validate(const eacg_model* m, const eacg_params* prm, std::string* why) {
  if (!m) {
    *why = "model is NULL";
    return EACG_EINVAL;
  }
  if (!(m->a > 0) || m->N < 8 || m->N > 128 || m->nbands < 1 || m->nk < 1 || !(m->ecut > 0) || m->natoms < 0) {
    *why = "invalid cell, grid, band, k-point or cutoff";
    return EACG_EINVAL;
  }
  if (m->natoms > 0 && (!m->pos || !m->Z || !m->rc)) {
    *why = "atoms without positions / charges / radii";
    return EACG_EINVAL;
  }
  if (!(m->nproj_per_atom == 0 || m->nproj_per_atom == 1 || m->nproj_per_atom == 4)) {
    *why = "nproj_per_atom must be 0, 1 or 4";
    return EACG_EINVAL;
  }
  if (m->nproj_per_atom > 0 && m->natoms > 0 && !m->D) {
    *why = "projectors without couplings";
    return EACG_EINVAL;
  }
  if (m->xc < 0 || m->xc > 2) {
    *why = "xc must be 0 (none), 1 (Slater exchange) or 2 (LDA: Slater exchange + PW92 correlation)";
    return EACG_EINVAL;
  }
  if (!m->kfrac || !m->kweight) {
    *why = "k-points missing";
    return EACG_EINVAL;
  }
  if (m->nbands > EACG_MAX_BANDS) {
    *why = "nbands above the largest supported block (1024 bands)";
    return EACG_EUNSUPPORTED;
  }
  if ((long long)m->nk * m->nbands > 65535) {
    *why = "nk * nbands above 65535 (the transforms launch one CTA row per band)";
    return EACG_EUNSUPPORTED;
  }
  if (!grid_supported(m->N)) {
    *why = "grid size N must be one of 8, 12, 16, 20, 24, 32, 36, 40, 48, 64, 72, 80, 96, 128";
    return EACG_EUNSUPPORTED;
  }
  if (prm && (!(prm->mu > 0) || prm->max_ls < 1 || prm->max_fom < 1 || prm->method < 0 || prm->method > 1)) {
    *why = "invalid parameters";
    return EACG_EINVAL;
  }
  return EACG_OK;
}

extern "C" void eacg_default_params(eacg_params* prm) {
  if (!prm) return;
  prm->mu = 0.01;
  prm->res_tol = 1e-8;
  prm->fom_rtol = 2.5e-2;
  prm->delta = 0.05;
  prm->sigma = 0.1;
  prm->gamma = 0.5;
  prm->eps = 1e-12;
  prm->warm_res = 1e-2;
  prm->switch_res = 1e-3;
  prm->max_outer = 300;
  prm->max_warm = 100;
  prm->max_fom = 50;
  prm->max_ls = 30;
  prm->precision = 0;
  prm->graphs = 1;
  prm->fft_plan = -1;
  prm->method = 0;
  prm->tensor_cores = 1;
  prm->df_transforms = 1;
}

static double sphere_volume_estimate(const eacg_model* m) {
  const double b = 2.0 * M_PI / m->a;
  const double r = std::sqrt(2.0 * m->ecut) / b + 1.0;
  return 4.0 / 3.0 * M_PI * r * r * r;
}

extern "C" size_t eacg_bytes_required(const eacg_model* m, const eacg_params* prm, size_t* fom_per_iter) {
  std::string why;
  if (validate(m, prm, &why) != EACG_OK) return 0;
  const size_t N3 = (size_t)m->N * m->N * m->N;
  const size_t nmax = (size_t)sphere_volume_estimate(m) + 64;
  const size_t K = m->nk, p = m->nbands;
  const size_t blk = K * p * nmax * 16;
  const size_t ncols = (size_t)(M_PI * std::pow(std::sqrt(2.0 * m->ecut) / (2.0 * M_PI / m->a) + 1.0, 2)) + 16;
  const size_t tb = K * p * m->N * ncols * 16;
  const size_t nproj = (size_t)m->natoms * m->nproj_per_atom;
  size_t tot = 17 * blk + tb + N3 * (8 * 6 + 16 + 4) + K * nproj * nmax * 16 + 8 * N3 * 8 + (64 << 20);
  tot += eacg::dense_pp_scratch((int)K, (int)p);
  if (fom_per_iter) *fom_per_iter = 2 * blk + K * p * p * 16 * 8;
  return tot;
}

static eacg_status build_basis(eacg_system* s) {
  const int N = s->N, K = s->K;
  int* d_rowoff = nullptr;
  int* d_colmark = nullptr;
  int* d_colidx = nullptr;
  int* d_scal = nullptr;
  TRY(dalloc(s, &d_rowoff, sizeof(int) * (size_t)K * (N * N + 1)));
  TRY(dalloc(s, &d_colmark, sizeof(int) * N * N));
  TRY(dalloc(s, &d_colidx, sizeof(int) * N * N));
  TRY(dalloc(s, &d_scal, sizeof(int) * 4));
  TRY(dalloc(s, &s->d_nk, sizeof(int) * K));
  grid_build_sphere(N, K, s->d_kfrac, s->thr, s->b, 0, s->d_nk, d_rowoff, nullptr, nullptr, d_colmark, s->st);
  CKL(s);
  s->nk.assign(K, 0);
  CK(cudaMemcpyAsync(s->nk.data(), s->d_nk, sizeof(int) * K, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  s->n_max = *std::max_element(s->nk.begin(), s->nk.end());
  if (s->n_max <= 0) {
    s->err = "empty basis (cutoff below the smallest |k+G|^2/2)";
    return EACG_EINVAL;
  }
  for (int k = 0; k < K; ++k) {
    if (s->nk[k] < s->p) {
      s->err = "fewer plane waves than bands at some k-point";
      return EACG_EINVAL;
    }
  }
  // the sphere must sit strictly inside the grid's frequency box
  {
    double kmax = 0;
    for (double v : s->kfrac) kmax = std::max(kmax, std::fabs(v));
    if (std::sqrt(s->thr) + kmax >= N / 2 - 0.5) {
      s->err = "grid too small for the cutoff sphere (N must exceed 2 |k+G|_max / b + 1)";
      return EACG_EINVAL;
    }
  }
  TRY(dalloc(s, &s->d_m, sizeof(int) * 3 * (size_t)K * s->n_max));
  TRY(dalloc(s, &s->d_kin, sizeof(double) * (size_t)K * s->n_max));
  grid_build_sphere(N, K, s->d_kfrac, s->thr, s->b, s->n_max, s->d_nk, d_rowoff, s->d_m, s->d_kin, d_colmark, s->st);
  CKL(s);
  TRY(dalloc(s, &s->d_cmapy, sizeof(int) * N * (N + 1)));
  TRY(dalloc(s, &s->d_rowmask, sizeof(int) * N));
  TRY(dalloc(s, &s->d_ylist, sizeof(int) * N));
  grid_columns(N, d_colmark, d_colidx, s->d_cmapy, s->d_rowmask, d_scal, s->d_ylist, d_scal + 1, s->st);
  CKL(s);
  int hs[2];
  CK(cudaMemcpyAsync(hs, d_scal, sizeof(int) * 2, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  s->ncols = hs[0];
  s->ny = hs[1];
  TRY(dalloc(s, &s->d_xmap, sizeof(int) * (size_t)K * s->ncols * N));
  grid_xmap(N, K, s->n_max, s->d_nk, s->d_m, d_colidx, s->ncols, s->d_xmap, s->st);
  CKL(s);
  CK(cudaStreamSynchronize(s->st));
  dfree(s, d_rowoff);
  dfree(s, d_colmark);
  dfree(s, d_colidx);
  dfree(s, d_scal);
  return EACG_OK;
}

static eacg_status build_potential_and_projectors(eacg_system* s) {
  const int N = s->N;
  const size_t N3 = (size_t)N * N * N;
  TRY(dalloc(s, &s->d_fft3, sizeof(double2) * N3));
  TRY(dalloc(s, &s->d_vloc, sizeof(double) * N3));
  TRY(dalloc(s, &s->d_vtot, sizeof(double) * N3));
  TRY(dalloc(s, &s->d_vtot32, sizeof(float) * N3));
  TRY(dalloc(s, &s->d_vtotdf, sizeof(float2) * N3));
  TRY(dalloc(s, &s->d_vh, sizeof(double) * N3));
  TRY(dalloc(s, &s->d_rho, sizeof(double) * N3));
  grid_vloc_g(N, s->b, s->omega, s->natoms, s->d_pos, s->d_Z, s->d_rc, s->d_fft3, s->st);
  CKL(s);
  grid_fft3(s->g, s->d_fft3, true, s->st);
  grid_complex_real_part(s->d_fft3, s->d_vloc, N3, s->st);
  CKL(s);
  // initial potential: local part only (rho = 0), FP64 and FP32 copies
  {
    double* esum = nullptr;
    TRY(dalloc(s, &esum, sizeof(double) * 3 * 256));
    grid_vtot_energy(N3, s->d_vloc, s->d_vh, s->d_rho, 0, 0, s->d_vtot, s->d_vtot32, s->d_vtotdf, esum, s->st);
    CKL(s);
    CK(cudaStreamSynchronize(s->st));
    dfree(s, esum);
  }
  if (s->nproj > 0) {
    TRY(dalloc(s, &s->d_B, sizeof(double2) * (size_t)s->K * s->nproj * s->n_max));
    TRY(dalloc(s, &s->d_P, sizeof(double2) * (size_t)s->K * s->nproj * s->p));
    TRY(dalloc(s, &s->d_P2, sizeof(double2) * (size_t)s->K * s->nproj * s->p));
    grid_projectors(s->K, s->n_max, s->d_nk, s->d_m, s->d_kfrac, s->b, s->omega, s->natoms, s->d_pos, s->npa,
                    s->width, s->d_B, s->st);
    CKL(s);
    TRY(dalloc(s, &s->d_B32, sizeof(float2) * (size_t)s->K * s->nproj * s->n_max));
    dense_to32((size_t)s->K * s->nproj * s->n_max, s->d_B, 1.0, s->d_B32, s->st);
    CKL(s);
  }
  return EACG_OK;
}

static eacg_status alloc_work(eacg_system* s) {
  const int K = s->K, p = s->p, N = s->N;
  s->blk = (size_t)K * p * s->n_max;
  const size_t bb = sizeof(double2) * s->blk;
  double2** blocks[] = {&s->phi, &s->hphi, &s->res, &s->eta, &s->gv, &s->teta, &s->tg, &s->psi_t, &s->phi_t,
                        &s->hphi_t, &s->res_t, &s->teta_t, &s->tmp1, &s->tmp2, &s->tmp3, &s->Xb, &s->Cb, &s->fvt, &s->fwt, &s->c32};
  for (auto b : blocks) TRY(dalloc(s, b, bb));
  const size_t sp = sizeof(double2) * (size_t)K * p * p;
  double2** smalls[] = {&s->lam, &s->lam_t, &s->sm1, &s->sm2, &s->sm3, &s->evec, &s->evec_t, &s->sinv_t,
                        &s->sig, &s->sigv, &s->sigvh};
  for (auto m : smalls) TRY(dalloc(s, m, sp));
  double** vecs[] = {&s->eval, &s->eval_t, &s->alpha, &s->sqd, &s->lref};
  for (auto v : vecs) TRY(dalloc(s, v, sizeof(double) * (size_t)K * p));
  if (const size_t ppb = dense_pp_scratch(K, p)) TRY(dalloc(s, &s->ppscr, ppb));
  // tbuf: one FP64 complex value per (band, jx, column)
  TRY(dalloc(s, &s->d_tbuf, sizeof(double2) * (size_t)K * p * N * s->ncols));
  // rho groups: enough CTAs to fill the GPU
  s->rho_groups = std::max(1, std::min(K * p, (8 * 152 + N - 1) / N));
  TRY(dalloc(s, &s->d_partial, sizeof(double) * (size_t)s->rho_groups * N * N * N));
  TRY(dalloc(s, &s->d_bw, sizeof(double) * (size_t)K * p));
  {
    std::vector<double> bw((size_t)K * p);
    for (int k = 0; k < K; ++k)
      for (int i = 0; i < p; ++i) bw[(size_t)k * p + i] = s->kw[k] * s->occ / s->omega;
    CK(cudaMemcpyAsync(s->d_bw, bw.data(), sizeof(double) * bw.size(), cudaMemcpyHostToDevice, s->st));
    CK(cudaStreamSynchronize(s->st));
  }
  const size_t cnw = std::max(dense_cn_work(K, s->n_max, 64 * 64, 1),
                              dense_cn_work(K, s->n_max, std::max(p, s->nproj), p));
  s->cn_elems = std::max(cnw, (size_t)K * 4096);
  TRY(dalloc(s, &s->cn_work, sizeof(double2) * s->cn_elems));
  TRY(dalloc(s, &s->d_red, sizeof(double) * ((size_t)K * std::max(p, 64) + 4096)));
  TRY(dalloc(s, &s->d_out, sizeof(double) * 4096));
  TRY(dalloc(s, &s->d_esum, sizeof(double) * 3 * 256));
  TRY(dalloc(s, &s->d_kactive, sizeof(int) * K));
  TRY(dalloc(s, &s->d_nzero, sizeof(int) * K));
  TRY(dalloc(s, &s->d_info, sizeof(int) * (size_t)K * 64));
  TRY(dalloc(s, &s->d_take, sizeof(int) * K));
  {


    CK(cudaMallocHost(&s->h_out, sizeof(double) * 4096));
    CK(cudaMallocHost(&s->h_int, sizeof(int) * 4 * K + 64));
  }
  return EACG_OK;
}

// Krylov storage for q columns per k; grows by doubling and keeps the contents.
// Strides and leading dimensions in elements of es bytes (16: complex128, 8: complex64).
static eacg_status copy_cols(eacg_system* s, double2* dst, int ldd, size_t sd, const double2* src, int lds, size_t ss,
                             int rows, int cols, size_t es = sizeof(double2)) {
  if (!src || rows <= 0 || cols <= 0) return EACG_OK;
  char* d = reinterpret_cast<char*>(dst);
  const char* c = reinterpret_cast<const char*>(src);
  for (int k = 0; k < s->K; ++k) {
    CK(cudaMemcpy2DAsync(d + k * sd * es, es * ldd, c + k * ss * es, es * lds, es * rows, cols,
                         cudaMemcpyDeviceToDevice, s->st));
  }
  return EACG_OK;
}

static eacg_status fom_reserve(eacg_system* s, int qneed) {
  if (qneed <= s->qcap) return EACG_OK;
  const int K = s->K, p = s->p, nm = s->n_max;
  int qc = std::max(s->qcap, std::min(s->prm.max_fom, 6) * p);
  while (qc < qneed) qc *= 2;
  qc = std::min(qc, std::max(qneed, s->prm.max_fom * p));
  double2 *nV, *nW, *nA, *nC, *nY, *nYt, *nYf;
  TRY(dalloc(s, &nV, sizeof(double2) * (size_t)K * qc * nm));
  TRY(dalloc(s, &nW, sizeof(double2) * (size_t)K * qc * nm));
  TRY(dalloc(s, &nA, sizeof(double2) * (size_t)K * qc * qc));
  TRY(dalloc(s, &nC, sizeof(double2) * (size_t)K * qc * p));
  TRY(dalloc(s, &nY, sizeof(double2) * (size_t)K * qc * p));
  TRY(dalloc(s, &nYt, sizeof(double2) * (size_t)K * qc * p));
  TRY(dalloc(s, &nYf, sizeof(double2) * (size_t)K * qc * p));
  const int oc = s->qcap;
  if (oc > 0) {
    TRY(copy_cols(s, nV, nm, (size_t)qc * nm, s->fV, nm, (size_t)oc * nm, nm, oc, s->fom_es));
    TRY(copy_cols(s, nW, nm, (size_t)qc * nm, s->fW, nm, (size_t)oc * nm, nm, oc, s->fom_es));
    TRY(copy_cols(s, nA, qc, (size_t)qc * qc, s->fA, oc, (size_t)oc * oc, oc, oc));
    TRY(copy_cols(s, nC, qc, (size_t)qc * p, s->fC, oc, (size_t)oc * p, oc, p));
    TRY(copy_cols(s, nY, qc, (size_t)qc * p, s->fY, oc, (size_t)oc * p, oc, p));
    TRY(copy_cols(s, nYt, qc, (size_t)qc * p, s->fYt, oc, (size_t)oc * p, oc, p));
    TRY(copy_cols(s, nYf, qc, (size_t)qc * p, s->fYf, oc, (size_t)oc * p, oc, p));
  }
  CK(cudaStreamSynchronize(s->st));
  dfree(s, s->fV);
  dfree(s, s->fW);
  dfree(s, s->fA);
  dfree(s, s->fC);
  dfree(s, s->fY);
  dfree(s, s->fYt);
  dfree(s, s->fYf);
  s->fV = nV;
  s->fW = nW;
  s->fA = nA;
  s->fC = nC;
  s->fY = nY;
  s->fYt = nYt;
  s->fYf = nYf;
  s->qcap = qc;
  const size_t fw = (fom_shifted_work(K, p, qc, 0) + sizeof(double2) - 1) / sizeof(double2);
  if (fw > s->fwork_elems) {
    dfree(s, s->fwork);
    s->fwork = nullptr;
    TRY(dalloc(s, &s->fwork, sizeof(double2) * fw));
    s->fwork_elems = fw;
  }
  const size_t cnw = std::max(dense_cn_work(K, nm, qc, p), (size_t)K * 4096);
  if (cnw > s->cn_elems) {
    dfree(s, s->cn_work);
    s->cn_work = nullptr;
    TRY(dalloc(s, &s->cn_work, sizeof(double2) * cnw));
    s->cn_elems = cnw;
  }
  return EACG_OK;
}

// ============================================================================ operators
// The potential the plane kernels multiply by: FP32 copy for FP32 transforms, the double-float
// copy or the FP64 grid for FP64-accurate ones.
static const void* vpot(const eacg_system* s, int prec) {
  if (prec) return s->d_vtot32;
  return s->g.df64 ? (const void*)s->d_vtotdf : (const void*)s->d_vtot;
}

// ---- cross-system batching of the transforms
// Systems stepped together (eacg_step_many, or eacg_step with eacg_batching on) run in their
// own host threads on their own streams.  When a system reaches the plane-wave transforms of
// an H application or a density it hands them to the batcher and waits; the first system to
// arrive leads: it waits until every stepping system is waiting, or the window has passed,
// then launches the transforms of all waiting systems that share the grid size, line plan and
// precision as one launch per kernel over a table of (system, band) work items (the segment
// tables of the transform kernels) on the leader's stream, ordered against every member's
// stream by events.  Each band is transformed by the same arithmetic as in a launch of its own,
// so batched results equal unbatched ones bit for bit.
struct XformOp {
  eacg_system* s = nullptr;
  int kind = 0;                 // 0: H application transforms, 1: density transforms
  int plan = 0, xmode = 0, pprec = 0;
  GridReq req{};
  bool done = false;
  eacg_status status = EACG_OK;
};

// process-wide counts of batched transform groups and of the system requests they covered
std::atomic<long long> g_batch_groups{0}, g_batch_members{0};

class Batcher {
 public:
  explicit Batcher(int window_us) : window_us_(window_us) {}
  void enter() {
    std::lock_guard<std::mutex> lk(mu_);
    ++live_;
  }
  void leave() {
    std::lock_guard<std::mutex> lk(mu_);
    --live_;
    cv_.notify_all();
  }
  int window_us() const { return window_us_; }
  long long launches() const { return batched_launches_.load(); }

  eacg_status submit(XformOp* op) {
    std::unique_lock<std::mutex> lk(mu_);
    pending_.push_back(op);
    ++waiting_;
    cv_.notify_all();
    if (!leading_) {
      leading_ = true;
      const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(window_us_);
      cv_.wait_until(lk, deadline, [&] { return waiting_ >= live_; });
      std::vector<XformOp*> batch;
      batch.swap(pending_);
      leading_ = false;
      lk.unlock();
      execute(batch);
      lk.lock();
      waiting_ -= (int)batch.size();
      for (XformOp* o : batch) o->done = true;
      cv_.notify_all();
    }
    cv_.wait(lk, [&] { return op->done; });
    return op->status;
  }

 private:
  void execute(std::vector<XformOp*>& batch) {
    std::vector<bool> used(batch.size(), false);
    for (size_t i = 0; i < batch.size(); ++i) {
      if (used[i]) continue;
      std::vector<XformOp*> grp;
      for (size_t j = i; j < batch.size(); ++j) {
        XformOp* a = batch[i];
        XformOp* b = batch[j];
        if (!used[j] && a->kind == b->kind && a->s->N == b->s->N && a->plan == b->plan && a->xmode == b->xmode &&
            a->pprec == b->pprec) {
          used[j] = true;
          grp.push_back(b);
        }
      }
      launch_group(grp);
    }
  }

  void launch_group(std::vector<XformOp*>& grp) {
    cudaStream_t ls = grp[0]->s->st;
    std::vector<GridReq> reqs;
    std::vector<cudaEvent_t> evs;
    cudaError_t err = cudaSuccess;
    for (XformOp* o : grp) {
      reqs.push_back(o->req);
      if (o->s->st != ls) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
          err = cudaErrorUnknown;
          break;
        }
        evs.push_back(e);
        cudaEventRecord(e, o->s->st);
        cudaStreamWaitEvent(ls, e, 0);
      }
    }
    const int N = grp[0]->s->N, n = (int)reqs.size();
    const XformOp& k0 = *grp[0];
    if (err == cudaSuccess) {
      grid_xpass_inv_multi(N, k0.plan, k0.xmode, reqs.data(), n, ls);
      if (k0.kind == 0) {
        grid_plane_h_multi(N, k0.plan, k0.pprec, reqs.data(), n, ls);
        grid_xpass_fwd_multi(N, k0.plan, k0.xmode, reqs.data(), n, ls);
      } else {
        grid_plane_rho_multi(N, k0.plan, k0.pprec, reqs.data(), n, ls);
      }
      batched_launches_ += (k0.kind == 0 ? 3 : 2) * ((n + GRID_MAX_SEGS - 1) / GRID_MAX_SEGS);
      g_batch_groups += 1;
      g_batch_members += n;
      err = cudaGetLastError();
    }
    cudaEvent_t done = nullptr;
    if (err == cudaSuccess && cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(done, ls);
      for (XformOp* o : grp)
        if (o->s->st != ls) cudaStreamWaitEvent(o->s->st, done, 0);
      cudaEventDestroy(done);
    } else if (err == cudaSuccess) {
      err = cudaErrorUnknown;
    }
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    for (XformOp* o : grp) {
      if (err != cudaSuccess) {
        o->status = EACG_ECUDA;
        o->s->err = std::string("batched transform launch: ") + cudaGetErrorString(err);
      }
    }
  }

  std::mutex mu_;
  std::condition_variable cv_;
  int live_ = 0, waiting_ = 0;
  bool leading_ = false;
  std::vector<XformOp*> pending_;
  int window_us_;
  std::atomic<long long> batched_launches_{0};
};

// the batcher of the calling thread's step (set by eacg_step_many and by eacg_step when
// batching is on), and the process-wide batcher of eacg_batching
thread_local Batcher* tl_batch = nullptr;
std::mutex g_batch_mu;
Batcher* g_batch = nullptr;

// The transforms of an H application (kind 0) or of a density (kind 1) of the bands of one
// system through the batcher.
static eacg_status batched_xform(eacg_system* s, int kind, int prec32_blocks, int prec, const void* in, void* out,
                                 const double* kin, double scale, const void* v, const int* kactive) {
  XformOp op;
  op.s = s;
  op.kind = kind;
  op.plan = prec ? s->g.plan32 : s->g.plan64;
  op.xmode = prec32_blocks ? 2 : prec ? 1 : (s->g.df64 ? 3 : 0);
  op.pprec = prec ? 1 : (s->g.df64 ? 2 : 0);
  GridReq& r = op.req;
  r.g = &s->g;
  r.in = in;
  r.tbuf = s->d_tbuf;
  r.out = out;
  r.kin = kin;
  r.scale = scale;
  r.v = v;
  r.kactive = kactive;
  r.nbands = s->K * s->p;
  r.bw = s->d_bw;
  r.partial = s->d_partial;
  r.groups = s->rho_groups;
  return tl_batch->submit(&op);
}

// P = B32^* in32 (projector overlaps of complex64 blocks): on the tensor cores (3 x TF32) when
// the shape allows it, else the SIMT FP32 block-overlap kernel.
static void projector_overlaps32(eacg_system* s, const float2* in32, const int* kactive) {
  const int K = s->K, p = s->p, np = s->nproj, nm = s->n_max;
  if (s->tc_proj)
    dense_overlap_tf32x3(K, nm, np, p, s->d_B32, (size_t)np * nm, nm, in32, (size_t)p * nm, nm, s->d_P,
                         (size_t)np * p, np, ONE, ZERO, s->cn_work, kactive, s->st);
  else
    dense_gemm_cn32(K, nm, np, p, s->d_B32, (size_t)np * nm, nm, in32, (size_t)p * nm, nm, s->d_P, (size_t)np * p,
                    np, ONE, ZERO, s->cn_work, kactive, s->st);
}

// FP64-accurate transforms hold a plane of 16-byte values in one CTA's shared memory: grids up
// to N = 96.  Larger grids (N = 128) have the FP32 transforms only.
constexpr int MAX_N_FP64_TRANSFORMS = 96;
static eacg_status check_fp64_grid(eacg_system* s, int prec) {
  if (prec == 0 && s->N > MAX_N_FP64_TRANSFORMS) {
    s->err = "FP64-accurate transforms support grids up to N = 96; N = 128 has FP32 transforms (precision 1)";
    return EACG_EUNSUPPORTED;
  }
  return EACG_OK;
}

// out = H in with the current potential (prec 0: FP64 transforms, 1: FP32).
static eacg_status apply_H_block(eacg_system* s, const double2* in, double2* out, int prec, const int* kactive) {
  TRY(check_fp64_grid(s, prec));
  const int nb = s->K * s->p;
  // algorithmic bytes per band: coefficients read/written in FP64, the x-pass
  // intermediate (N * ncols values of the transform precision) written, read, written, read
  const double tv = prec ? 8.0 : 16.0;
  const double inter = (double)s->N * s->ncols * tv;
  const double coef = (double)s->n_max * 16.0;
  const double N3 = (double)s->N * s->N * s->N;
  const int off = prec ? P_F32 : 0;
  const double fx = nb * s->ncols * fft_flops(s->N);
  const double fp = nb * 2.0 * s->N * (s->ny + s->N) * fft_flops(s->N);
  if (tl_batch) {
    TRY(batched_xform(s, 0, 0, prec, in, out, s->d_kin, 1.0 / N3, vpot(s, prec), kactive));
  } else {
    PROF_RUN(P_XINV + off, nb * (coef + inter), fx, nb,
             grid_xpass_inv(s->g, prec, in, s->d_tbuf, nb, kactive, s->st));
    PROF_RUN(P_PLANE_H + off, nb * 2.0 * inter + N3 * (prec ? 4.0 : 8.0), fp, nb,
             grid_plane_h(s->g, prec, s->d_tbuf, vpot(s, prec), nb, kactive, s->st));
    PROF_RUN(P_XFWD + off, nb * (inter + 2.0 * coef), fx, nb,
             grid_xpass_fwd(s->g, prec, s->d_tbuf, in, s->d_kin, 1.0 / N3, out, nb, kactive, s->st));
  }
  CKL(s);
  if (s->nproj > 0 && prec == 0) {
    const int K = s->K, p = s->p, np = s->nproj, nm = s->n_max;
    PROF_RUN(P_NONLOCAL, (double)K * np * nm * 16.0 * 2 + 3.0 * nb * coef, 16.0 * K * np * nm * p, nb, {
      dense_gemm_cn(K, nm, np, p, s->d_B, (size_t)np * nm, nm, in, (size_t)p * nm, nm, s->d_P, (size_t)np * p, np,
                    ONE, ZERO, s->cn_work, kactive, s->st, s->g.df64);
      dense_copy(s->d_P2, s->d_P, (size_t)K * np * p, s->st);
      dense_scale_rows(K, np, p, s->d_P, s->d_dvec, s->st);
      dense_gemm_nn(K, nm, np, p, s->d_B, (size_t)np * nm, nm, s->d_P, (size_t)np * p, np, out, (size_t)p * nm, nm,
                    ONE, ONE, kactive, s->st, s->g.df64);
    });
    CKL(s);
  } else if (s->nproj > 0) {
    // FP32 phase: projector overlaps of complex64 copies (FP32 products, FP64 chunk sums), the
    // back-projection accumulated in FP32 and added into the FP64 result
    const int K = s->K, p = s->p, np = s->nproj, nm = s->n_max;
    float2* in32 = reinterpret_cast<float2*>(s->c32);
    PROF_RUN(P_NONLOCAL32, (double)K * np * nm * 8.0 * 2 + nb * nm * (16.0 + 8.0 + 8.0 + 32.0), 16.0 * K * np * nm * p,
             nb, {
               dense_to32(s->blk, in, 1.0, in32, s->st);
               projector_overlaps32(s, in32, kactive);
               dense_copy(s->d_P2, s->d_P, (size_t)K * np * p, s->st);
               dense_scale_rows(K, np, p, s->d_P, s->d_dvec, s->st);
               if (s->tc_proj && p % 16 == 0) {
                 // tensor-core back-projection in column blocks of at most 256 bands (one MMA N)
                 for (int j0 = 0; j0 < p; j0 += 256) {
                   const int nc = std::min(256, p - j0);
                   dense_backproject_tf32x3(K, nm, np, nc, s->d_B32, (size_t)np * nm, nm, s->d_P + (size_t)j0 * np,
                                            (size_t)np * p, np, out + (size_t)j0 * nm, (size_t)p * nm, nm, kactive,
                                            s->st);
                 }
               } else
                 dense_gemm_nn32_into64(K, nm, np, p, s->d_B32, (size_t)np * nm, nm, s->d_P, (size_t)np * p, np,
                                        out, (size_t)p * nm, nm, ONE, ONE, kactive, s->st);
             });
    CKL(s);
  }
  s->h_apps += (long long)s->K * s->p;
  return EACG_OK;
}

// rho of an orthonormal block into d_rho.
static eacg_status density_only(eacg_system* s, const double2* phi, int prec) {
  TRY(check_fp64_grid(s, prec));
  const int nb = s->K * s->p;
  const int N = s->N;
  const size_t N3 = (size_t)N * N * N;
  const double tv = prec ? 8.0 : 16.0;
  const double inter = (double)s->N * s->ncols * tv;
  const int off = prec ? P_F32 : 0;
  if (tl_batch) {
    TRY(batched_xform(s, 1, 0, prec, phi, nullptr, nullptr, 1.0, nullptr, nullptr));
    grid_reduce_groups(s->d_partial, s->rho_groups, N3, s->d_rho, s->st);
  } else {
    PROF_RUN(P_XINV_RHO + off, nb * ((double)s->n_max * 16.0 + inter), nb * s->ncols * fft_flops(s->N), nb,
             grid_xpass_inv(s->g, prec, phi, s->d_tbuf, nb, nullptr, s->st));
    PROF_RUN(P_PLANE_RHO + off, nb * inter + (double)s->rho_groups * N3 * 8.0,
             nb * (double)s->N * (s->ny + s->N) * fft_flops(s->N), nb, {
      grid_plane_rho(s->g, prec, s->d_tbuf, nb, s->rho_groups, s->d_bw, s->d_partial, s->st);
      grid_reduce_groups(s->d_partial, s->rho_groups, N3, s->d_rho, s->st);
    });
  }
  CKL(s);
  return EACG_OK;
}

// The potential of the density in d_rho (FP64 and FP32 copies); E_loc, E_H, E_xc integrands
// into d_esum.
static eacg_status potential_from_rho(eacg_system* s) {
  const int N = s->N;
  const size_t N3 = (size_t)N * N * N;
  int nblk = 0;
  PROF_RUN(P_POT, (double)N3 * 8.0 * 8, 6.0 * N * N * fft_flops(N), 0, {
    if (s->hartree) {
      grid_real_to_complex(s->d_rho, s->d_fft3, N3, s->st);
      grid_fft3(s->g, s->d_fft3, false, s->st);
      grid_hartree_scale(s->d_fft3, N, s->b, s->st);
      grid_fft3(s->g, s->d_fft3, true, s->st);
      grid_complex_real_part(s->d_fft3, s->d_vh, N3, s->st);
    }
    nblk = grid_vtot_energy(N3, s->d_vloc, s->d_vh, s->d_rho, s->hartree, s->xc, s->d_vtot, s->d_vtot32,
                            s->d_vtotdf, s->d_esum, s->st);
  });
  CKL(s);
  return (nblk == 256) ? EACG_OK : EACG_ECUDA;
}

// rho of an orthonormal block and the potential built from it.
static eacg_status density_and_potential(eacg_system* s, const double2* phi, int prec) {
  TRY(density_only(s, phi, prec));
  return potential_from_rho(s);
}

// ============================================================================ reductions to host
// Sum of the 3 * nblk strided block sums of k_vtot_energy, done on the host after one copy.
static eacg_status fetch_grid_energies(eacg_system* s, double* eloc, double* eh, double* ex) {
  const int nblk = 256;
  CK(cudaMemcpyAsync(s->h_out, s->d_esum, sizeof(double) * 3 * nblk, cudaMemcpyDeviceToHost, s->st));
  CK(stream_wait(s));
  double a = 0, b = 0, c = 0;
  for (int i = 0; i < nblk; ++i) {
    a += s->h_out[3 * i];
    b += s->h_out[3 * i + 1];
    c += s->h_out[3 * i + 2];
  }
  const double dv = s->omega / ((double)s->N * s->N * s->N);
  *eloc = a * dv;
  *eh = b * dv;
  *ex = c * dv;
  return EACG_OK;
}

// weighted pairing <V, W> = sum_k w_k Re tr(V_k^* W_k) into d_out[slot]
static void pairing_dev(eacg_system* s, const double2* V, const double2* W, int slot, bool weighted) {
  const int np = dense_dot(s->K, (size_t)s->p * s->n_max, V, W, weighted ? s->d_kw : nullptr, s->d_red, s->st);
  dense_sum_partials(s->d_red, np, s->d_out + slot, s->st);
}

// ============================================================================ evaluation
struct EvalOut {
  double E, rnorm, terms[5];
};

// Density, potential, H phi, Lambda, R and the energy at an orthonormal phi.
// A non-finite energy or residual; names a tensor-core wait that gave up (its tile is NaN) when
// the device's give-up count is not zero.
static eacg_status nan_status(eacg_system* s, const char* what) {
  s->err = what;
  if (s->prm.tensor_cores) {
    const unsigned int n = dense_tc_gaveup_count(s->st);
    if (n != 0u && n != ~0u) s->err += " (a tensor-core MMA wait gave up on this device)";
  }
  return EACG_ENAN;
}

static eacg_status evaluate(eacg_system* s, const double2* phi, double2* hphi, double2* res, double2* lam, int prec,
                            EvalOut* out) {
  const int K = s->K, p = s->p, nm = s->n_max;
  if (!s->frozen) TRY(density_and_potential(s, phi, prec));
  TRY(apply_H_block(s, phi, hphi, prec, nullptr));
  // Lambda = herm(Phi^* H Phi)
  dense_gemm_cn(K, nm, p, p, phi, (size_t)p * nm, nm, hphi, (size_t)p * nm, nm, lam, (size_t)p * p, p, ONE, ZERO,
                s->cn_work, nullptr, s->st, s->g.df64);
  dense_herm(K, p, lam, s->st);
  // R = H Phi - Phi Lambda
  dense_copy(res, hphi, s->blk, s->st);
  dense_gemm_nn(K, nm, p, p, phi, (size_t)p * nm, nm, lam, (size_t)p * p, p, res, (size_t)p * nm, nm, MONE, ONE,
                nullptr, s->st, s->g.df64);
  CKL(s);
  if (s->frozen) {
    // band energy of the fixed Hamiltonian: f <Phi, H Phi> in the weighted pairing
    pairing_dev(s, phi, hphi, 0, true);
    pairing_dev(s, res, res, 1, false);
    CKL(s);
    TRY(sync_read(s, 2));
    for (double& t : out->terms) t = 0.0;
    out->E = s->occ * s->h_out[0];
    out->rnorm = std::sqrt(std::max(s->h_out[1], 0.0));
    if (!std::isfinite(out->E) || !std::isfinite(out->rnorm)) return nan_status(s, "non-finite band energy or residual");
    return EACG_OK;
  }
  // kinetic energy partials -> d_red[0..K*p), summed into d_out[0]
  dense_kin_energy(K, p, nm, s->d_kin, phi, s->d_kw, s->occ, s->d_red, s->st);
  dense_sum_partials(s->d_red, K * p, s->d_out + 0, s->st);
  // nonlocal energy: sum_k w_k f sum D |P|^2 = pairing of unscaled and scaled projections
  if (s->nproj > 0) {
    const int npp = dense_dot(K, (size_t)s->nproj * p, s->d_P2, s->d_P, s->d_kw, s->d_red, s->st);
    dense_sum_partials(s->d_red, npp, s->d_out + 1, s->st);
  } else {
    cudaMemsetAsync(s->d_out + 1, 0, sizeof(double), s->st);
  }
  // ||R||^2 (unweighted)
  pairing_dev(s, res, res, 2, false);
  CKL(s);
  TRY(sync_read(s, 3));
  const double ekin = s->h_out[0];
  const double enl = s->occ * s->h_out[1];
  const double r2 = s->h_out[2];
  double eloc, eh, ex;
  TRY(fetch_grid_energies(s, &eloc, &eh, &ex));
  out->terms[0] = ekin;
  out->terms[1] = eloc;
  out->terms[2] = s->hartree ? eh : 0.0;
  out->terms[3] = s->xc ? ex : 0.0;
  out->terms[4] = enl;
  out->E = ekin + eloc + out->terms[2] + out->terms[3] + enl;
  out->rnorm = std::sqrt(std::max(r2, 0.0));
  if (!std::isfinite(out->E) || !std::isfinite(out->rnorm)) return nan_status(s, "non-finite energy or residual");
  return EACG_OK;
}

// out = pf(psi) = psi V D^{-1/2} V^H; keeps the eigenpairs of psi^* psi and S^{-1}.
static eacg_status polar(eacg_system* s, const double2* psi, double2* out, double* ev, double2* evv, double2* sinv) {
  const int K = s->K, p = s->p, nm = s->n_max;
  dense_gemm_cn(K, nm, p, p, psi, (size_t)p * nm, nm, psi, (size_t)p * nm, nm, s->sm1, (size_t)p * p, p, ONE, ZERO,
                s->cn_work, nullptr, s->st, s->g.df64);
  dense_heig(K, p, s->sm1, (size_t)p * p, ev, evv, nullptr, s->st, s->ppscr);
  dense_eig_func(K, p, evv, ev, -0.5, 0.0, sinv, nullptr, s->st);
  dense_gemm_nn(K, nm, p, p, psi, (size_t)p * nm, nm, sinv, (size_t)p * p, p, out, (size_t)p * nm, nm, ONE, ZERO,
                nullptr, s->st, s->g.df64);
  CKL(s);
  return EACG_OK;
}

// ============================================================================ directions
// Warm-up direction g = Z - Phi herm(Phi^* Z), Z = TPA (unit gain) applied to R.
static eacg_status precond_gradient(eacg_system* s, const double2* phi, const double2* res, double2* g) {
  const int K = s->K, p = s->p, nm = s->n_max;
  dense_kinetic_alpha(K, p, nm, s->d_kin, phi, s->alpha, s->st);
  dense_tpa(K, p, nm, s->d_kin, s->alpha, res, s->tmp1, true, s->st);
  dense_gemm_cn(K, nm, p, p, phi, (size_t)p * nm, nm, s->tmp1, (size_t)p * nm, nm, s->sm1, (size_t)p * p, p, ONE,
                ZERO, s->cn_work, nullptr, s->st, s->g.df64);
  dense_herm(K, p, s->sm1, s->st);
  dense_copy(g, s->tmp1, s->blk, s->st);
  dense_gemm_nn(K, nm, p, p, phi, (size_t)p * nm, nm, s->sm1, (size_t)p * p, p, g, (size_t)p * nm, nm, MONE, ONE,
                nullptr, s->st, s->g.df64);
  CKL(s);
  return EACG_OK;
}

// Kernel wrappers of one block precision for the FOM: T = double (FP64 mode) or float
// (mixed mode, FP32 Krylov blocks and transforms; small projected matrices stay FP64).
template <typename T>
struct FomOps;
template <>
struct FomOps<double> {
  using V = double2;
  static constexpr double drop_tol = 1e-12;
  static void cn(int K, int L, int m, int n, const V* A, size_t sA, int lda, const V* B, size_t sB, int ldb,
                 double2* C, size_t sC, int ldc, double2 al, double2 be, double2* w, const int* ka, cudaStream_t st,
                 int df) {
    dense_gemm_cn(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, al, be, w, ka, st, df);
  }
  static void nn(int K, int L, int m, int n, const V* A, size_t sA, int lda, const double2* B, size_t sB, int ldb,
                 V* C, size_t sC, int ldc, double2 al, double2 be, const int* ka, cudaStream_t st, int df) {
    dense_gemm_nn(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, al, be, ka, st, df);
  }
  static void axpby(size_t n, double2 a, const V* x, double2 b, const V* y, V* o, cudaStream_t st) {
    dense_axpby(n, a, x, b, y, o, st);
  }
  static void norms2(int K, size_t len, const V* v, double* o, cudaStream_t st) { dense_norms2(K, len, v, o, st); }
  static void tpa(int K, int p, int nm, const double* kin, const double* al, const V* in, V* out, cudaStream_t st) {
    dense_tpa(K, p, nm, kin, al, in, out, false, st);
  }
};
template <>
struct FomOps<float> {
  using V = float2;
  static constexpr double drop_tol = 1e-6;
  static void cn(int K, int L, int m, int n, const V* A, size_t sA, int lda, const V* B, size_t sB, int ldb,
                 double2* C, size_t sC, int ldc, double2 al, double2 be, double2* w, const int* ka, cudaStream_t st,
                 int) {
    dense_gemm_cn32(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, al, be, w, ka, st);
  }
  static void nn(int K, int L, int m, int n, const V* A, size_t sA, int lda, const double2* B, size_t sB, int ldb,
                 V* C, size_t sC, int ldc, double2 al, double2 be, const int* ka, cudaStream_t st, int) {
    dense_gemm_nn32(K, L, m, n, A, sA, lda, B, sB, ldb, C, sC, ldc, al, be, ka, st);
  }
  static void axpby(size_t n, double2 a, const V* x, double2 b, const V* y, V* o, cudaStream_t st) {
    dense_axpby32(n, a, x, b, y, o, st);
  }
  static void norms2(int K, size_t len, const V* v, double* o, cudaStream_t st) { dense_norms2_32(K, len, v, o, st); }
  static void tpa(int K, int p, int nm, const double* kin, const double* al, const V* in, V* out, cudaStream_t st) {
    dense_tpa32(K, p, nm, kin, al, in, out, st);
  }
};

// H applied to FP32 blocks with FP32 transforms (the FOM of the mixed mode).
static eacg_status apply_H_block32(eacg_system* s, const float2* in, float2* out, const int* kactive) {
  const int nb = s->K * s->p;
  const double inter = (double)s->N * s->ncols * 8.0;
  const double coef = (double)s->n_max * 8.0;
  const double N3 = (double)s->N * s->N * s->N;
  const double fx = nb * s->ncols * fft_flops(s->N);
  const double fp = nb * 2.0 * s->N * (s->ny + s->N) * fft_flops(s->N);
  if (tl_batch) {
    TRY(batched_xform(s, 0, 1, 1, in, out, s->d_kin, 1.0 / N3, s->d_vtot32, kactive));
  } else {
    PROF_RUN(P_XINV + P_F32, nb * (coef + inter), fx, nb,
             grid_xpass_inv32(s->g, in, s->d_tbuf, nb, kactive, s->st));
    PROF_RUN(P_PLANE_H + P_F32, nb * 2.0 * inter + N3 * 4.0, fp, nb,
             grid_plane_h(s->g, 1, s->d_tbuf, s->d_vtot32, nb, kactive, s->st));
    PROF_RUN(P_XFWD + P_F32, nb * (inter + 2.0 * coef), fx, nb,
             grid_xpass_fwd32(s->g, s->d_tbuf, in, s->d_kin, 1.0 / N3, out, nb, kactive, s->st));
  }
  CKL(s);
  if (s->nproj > 0) {
    const int K = s->K, p = s->p, np = s->nproj, nm = s->n_max;
    PROF_RUN(P_NONLOCAL + P_F32, (double)K * np * nm * 8.0 * 2 + 3.0 * nb * coef, 16.0 * K * np * nm * p, nb, {
      projector_overlaps32(s, in, kactive);
      dense_scale_rows(K, np, p, s->d_P, s->d_dvec, s->st);
      dense_gemm_nn32(K, nm, np, p, s->d_B32, (size_t)np * nm, nm, s->d_P, (size_t)np * p, np, out, (size_t)p * nm,
                      nm, ONE, ONE, kactive, s->st);
    });
    CKL(s);
  }
  s->h_apps += (long long)s->K * s->p;
  return EACG_OK;
}

static eacg_status apply_H_t(eacg_system* s, const double2* in, double2* out, const int* ka) {
  return apply_H_block(s, in, out, 0, ka);
}
static eacg_status apply_H_t(eacg_system* s, const float2* in, float2* out, const int* ka) {
  return apply_H_block32(s, in, out, ka);
}

// ---- CUDA graph of the FOM's block H application
// The FOM applies H to the same device blocks every iteration, so the whole launch sequence
// (x pass, plane, x pass back, projector GEMMs) is captured once per system and block
// precision and replayed.  The first call with a given set of buffers runs directly (it sets
// the kernels' shared-memory limits), the second is captured (thread-local mode, so other
// systems' host threads are unaffected) and every later call replays it.  The graph holds
// event-record nodes at the profile slots; after a profiled replay their times are read back
// before the next replay.  Any capture error turns graphs off for the system.
static void hg_release(eacg_system::HGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  for (auto& r : g.recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g = eacg_system::HGraph();
}

static void hg_resolve(eacg_system* s, eacg_system::HGraph& g) {
  if (!g.pending) return;
  for (const auto& r : g.recs) {
    float ms = 0.f;
    cudaEventSynchronize(r.b);
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess)
      s->prof_ms.push_back({r.slot, ms, r.bytes, r.flops, r.units});
    else
      cudaGetLastError();  // a time that cannot be read is dropped, not reported as a launch error
  }
  g.pending = false;
}

template <typename V>
static eacg_status apply_H_fom(eacg_system* s, const V* in, V* out, const int* ka) {
  auto& g = s->hg[sizeof(V) == sizeof(float2) ? 1 : 0];
  // batched steps launch the transforms together with other systems: no per-system graph
  if (!s->prm.graphs || s->graphs_off || tl_batch) return apply_H_t(s, in, out, ka);
  const bool same = g.in == in && g.out == out && g.ka == ka && g.cnw == s->cn_work;
  if (!same) {
    hg_resolve(s, g);  // keep the last replay's profile records
    hg_release(g);
    g.in = in;
    g.out = out;
    g.ka = ka;
    g.cnw = s->cn_work;
  }
  if (!g.exec) {
    if (g.direct++ == 0) return apply_H_t(s, in, out, ka);
    // capture
    cudaGetLastError();
    if (cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      s->graphs_off = true;
      return apply_H_t(s, in, out, ka);
    }
    const long long h0 = s->h_apps;
    s->cap = &g;
    const eacg_status st = apply_H_t(s, in, out, ka);
    s->cap = nullptr;
    cudaGraph_t graph = nullptr;
    const cudaError_t e1 = cudaStreamEndCapture(s->st, &graph);
    s->h_apps = h0;
    cudaGraphExec_t exec = nullptr;
    if (st != EACG_OK || e1 != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      hg_release(g);
      s->graphs_off = true;
      return st != EACG_OK ? st : apply_H_t(s, in, out, ka);
    }
    g.graph = graph;
    g.exec = exec;
    // kernel nodes of the graph: the capture counted them as launches, the replays launch them
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(graph, nodes.data(), &nn);
    g.kernels = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++g.kernels;
    }
    count_launches(-g.kernels);
  }
  hg_resolve(s, g);
  CK(cudaGraphLaunch(g.exec, s->st));
  ++s->graph_launches;
  count_launches(g.kernels);
  s->h_apps += (long long)s->K * s->p;
  if (s->prof_on) g.pending = true;
  return EACG_OK;
}

// Rank-revealing orthonormalisation of R (n x p per k) against the first q columns of V
// (Algorithm 4's rank-revealing QR, reading: two projections, then QR with column pivoting
// written as a diagonally pivoted Cholesky of the Gram matrix, stopped below a relative
// tolerance of the largest squared column norm of R before projection; a second pivoted
// Cholesky pass on the kept block).  Result into out (n x p per k, dropped directions as
// leading zero columns), nzero[k].
template <typename T>
static eacg_status orthonormalise(eacg_system* s, cplx<T>* R, const cplx<T>* V, int q, size_t sV, cplx<T>* out,
                                  cplx<T>* scratch, const int* kactive) {
  using O = FomOps<T>;
  const int K = s->K, p = s->p, nm = s->n_max;
  const size_t sb = (size_t)p * nm;
  // reference: largest squared column norm before projection
  O::cn(K, nm, p, p, R, sb, nm, R, sb, nm, s->sm1, (size_t)p * p, p, ONE, ZERO, s->cn_work, kactive, s->st, s->g.df64);
  small_max_diag(K, p, s->sm1, s->lref, s->st);
  if (q > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      O::cn(K, nm, q, p, V, sV, nm, R, sb, nm, s->fYt, (size_t)s->qcap * p, s->qcap, ONE, ZERO, s->cn_work, kactive,
            s->st, s->g.df64);
      O::nn(K, nm, q, p, V, sV, nm, s->fYt, (size_t)s->qcap * p, s->qcap, R, sb, nm, MONE, ONE, kactive, s->st, s->g.df64);
    }
  }
  // first (rank-revealing) pass
  O::cn(K, nm, p, p, R, sb, nm, R, sb, nm, s->sm1, (size_t)p * p, p, ONE, ZERO, s->cn_work, kactive, s->st, s->g.df64);
  small_pivchol(K, p, s->sm1, s->lref, O::drop_tol, s->sm3, s->d_nzero, kactive, s->st, s->ppscr);
  O::nn(K, nm, p, p, R, sb, nm, s->sm3, (size_t)p * p, p, scratch, sb, nm, ONE, ZERO, kactive, s->st, s->g.df64);
  // second pass on the kept block (reference: its own largest column norm)
  O::cn(K, nm, p, p, scratch, sb, nm, scratch, sb, nm, s->sm1, (size_t)p * p, p, ONE, ZERO, s->cn_work, kactive,
        s->st, s->g.df64);
  small_pivchol(K, p, s->sm1, nullptr, O::drop_tol, s->sm3, s->d_info, kactive, s->st, s->ppscr);
  O::nn(K, nm, p, p, scratch, sb, nm, s->sm3, (size_t)p * p, p, out, sb, nm, ONE, ZERO, kactive, s->st, s->g.df64);
  CKL(s);
  return EACG_OK;
}

// Copies contiguous [K][p][n_max] blocks into columns [q0, q0 + p) of the Krylov storage.
template <typename V>
static eacg_status put_cols(eacg_system* s, const V* v, const V* w, int q0) {
  const size_t wb = sizeof(V) * (size_t)s->p * s->n_max;
  const size_t dp = sizeof(V) * (size_t)s->qcap * s->n_max;
  V* fV = reinterpret_cast<V*>(s->fV);
  V* fW = reinterpret_cast<V*>(s->fW);
  CK(cudaMemcpy2DAsync(fV + (size_t)q0 * s->n_max, dp, v, wb, wb, s->K, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaMemcpy2DAsync(fW + (size_t)q0 * s->n_max, dp, w, wb, wb, s->K, cudaMemcpyDeviceToDevice, s->st));
  return EACG_OK;
}

// Energy-adaptive gradient by the preconditioned block FOM, per k (Algorithm 4, Sec. 5.2),
// with Krylov blocks of precision T.  Uses the current potential (the one of phi).
// fom_iters: host array of K ints or NULL.
template <typename T>
static eacg_status ea_gradient_t(eacg_system* s, const double2* phi, const double2* hphi, const double2* lam,
                                 double2* g, int* fom_iters) {
  using O = FomOps<T>;
  using V = cplx<T>;
  const int K = s->K, p = s->p, nm = s->n_max;
  const size_t sb = (size_t)p * nm;
  const double mu = s->prm.mu;
  const bool f32 = sizeof(T) == 4;
  s->fom_es = sizeof(V);
  TRY(fom_reserve(s, 2 * p));
  // Sigma = Lambda - mu I, its eigenpairs and Q^H
  dense_shift_diag(K, p, lam, mu, s->sig, s->st);
  dense_heig(K, p, s->sig, (size_t)p * p, s->eval, s->sigv, nullptr, s->st, s->ppscr);
  small_conj_transpose(K, p, s->sigv, s->sigvh, s->st);
  dense_kinetic_alpha(K, p, nm, s->d_kin, phi, s->alpha, s->st);
  // C = Phi - (H X0 - X0 Sigma), X0 = Phi / mu, H X0 = H Phi / mu  (FP64, then in T)
  dense_copy(s->Cb, hphi, s->blk, s->st);
  dense_gemm_nn(K, nm, p, p, phi, sb, nm, s->sig, (size_t)p * p, p, s->Cb, sb, nm, MONE, ONE, nullptr, s->st, s->g.df64);
  dense_axpby(s->blk, ONE, phi, cr(-1.0 / mu), s->Cb, s->Cb, s->st);
  dense_norms2(K, sb, s->Cb, s->d_out + 64, s->st);
  V* C = reinterpret_cast<V*>(s->Cb);
  if (f32) {
    C = reinterpret_cast<V*>(s->c32);
    dense_to32(s->blk, s->Cb, 1.0, reinterpret_cast<float2*>(s->c32), s->st);
  }
  V* t1 = reinterpret_cast<V*>(s->tmp1);
  V* t2 = reinterpret_cast<V*>(s->tmp2);
  V* t3 = reinterpret_cast<V*>(s->tmp3);
  V* vt = reinterpret_cast<V*>(s->fvt);
  V* wt = reinterpret_cast<V*>(s->fwt);
  CKL(s);
  TRY(sync_read(s, 64 + K));
  std::vector<double> cnorm(K);
  std::vector<int> active(K, 1), iters(K, 0);
  for (int k = 0; k < K; ++k) {
    cnorm[k] = std::sqrt(s->h_out[64 + k]);
    if (!(cnorm[k] > 0)) active[k] = 0;
  }
  auto upload_active = [&]() -> eacg_status {
    for (int k = 0; k < K; ++k) s->h_int[k] = active[k];
    CK(cudaMemcpyAsync(s->d_kactive, s->h_int, sizeof(int) * K, cudaMemcpyHostToDevice, s->st));
    return EACG_OK;
  };
  TRY(upload_active());
  cudaMemsetAsync(s->fYf, 0, sizeof(double2) * (size_t)K * s->qcap * p, s->st);
  cudaMemsetAsync(s->fA, 0, sizeof(double2) * (size_t)K * s->qcap * s->qcap, s->st);
  // V_1 = orth(P^{-1} C), W_1 = H V_1, A_1 = herm(V_1^* W_1), C_1 = V_1^* C
  O::tpa(K, p, nm, s->d_kin, s->alpha, C, t2, s->st);
  cudaMemsetAsync(vt, 0, sizeof(V) * s->blk, s->st);
  cudaMemsetAsync(wt, 0, sizeof(V) * s->blk, s->st);
  TRY(orthonormalise<T>(s, t2, nullptr, 0, 0, vt, t3, s->d_kactive));
  TRY(apply_H_fom(s, vt, wt, s->d_kactive));
  TRY(put_cols(s, vt, wt, 0));
  int q = 0;
  auto add_block = [&](int q0) -> eacg_status {
    // columns [q0, q0 + p) of V and W are new: fill A and C
    const size_t sV = (size_t)s->qcap * nm;
    const size_t sA = (size_t)s->qcap * s->qcap;
    V* fV = reinterpret_cast<V*>(s->fV);
    V* Vn = fV + (size_t)q0 * nm;
    V* Wn = reinterpret_cast<V*>(s->fW) + (size_t)q0 * nm;
    if (q0 > 0) {
      O::cn(K, nm, q0, p, fV, sV, nm, Wn, sV, nm, s->fA + (size_t)q0 * s->qcap, sA, s->qcap, ONE, ZERO, s->cn_work,
            s->d_kactive, s->st, s->g.df64);
      fom_mirror(K, q0, p, s->fA, s->qcap, sA, s->d_kactive, s->st);
    }
    O::cn(K, nm, p, p, Vn, sV, nm, Wn, sV, nm, s->sm1, (size_t)p * p, p, ONE, ZERO, s->cn_work, s->d_kactive, s->st, s->g.df64);
    small_put_herm_block(K, p, s->sm1, s->fA, s->qcap, sA, q0, s->st);
    fom_pad_diag(K, q0, p, s->fA, s->qcap, sA, s->d_nzero, s->eval, s->st);
    O::cn(K, nm, p, p, Vn, sV, nm, C, sb, nm, s->fC + q0, (size_t)s->qcap * p, s->qcap, ONE, ZERO, s->cn_work,
          s->d_kactive, s->st, s->g.df64);
    CKL(s);
    return EACG_OK;
  };
  TRY(add_block(0));
  q = p;
  // rank of the first block
  CK(cudaMemcpyAsync(s->h_int + K, s->d_nzero, sizeof(int) * K, cudaMemcpyDeviceToHost, s->st));
  CK(stream_wait(s));
  for (int k = 0; k < K; ++k)
    if (active[k] && s->h_int[K + k] >= p) active[k] = 0;  // rank 0: nothing to solve
  int j = 0;
  while (true) {
    ++j;
    const size_t sC = (size_t)s->qcap * p;
    const size_t sA = (size_t)s->qcap * s->qcap;
    const size_t sV = (size_t)s->qcap * nm;
    V* fV = reinterpret_cast<V*>(s->fV);
    V* fW = reinterpret_cast<V*>(s->fW);
    TRY(upload_active());
    // Y = solve(A Y - Y Sigma = C_j) via C~ = C Q, (A - s_m) y~_m = c~_m, Y = Y~ Q^H
    dense_gemm_nn(K, q, p, p, s->fC, sC, s->qcap, s->sigv, (size_t)p * p, p, s->fYt, sC, s->qcap, ONE, ZERO,
                  s->d_kactive, s->st, s->g.df64);
    // algorithmic: A, C read and Y written once per k; (16/3) q^3 for the Householder reduction
    // plus two reflector transforms of 8 q^2 per shift
    PROF_RUN(P_FOMSOLVE + (f32 ? P_F32 : 0), (double)K * ((double)q * q + 2.0 * q * p) * 16.0,
             (double)K * ((16.0 / 3.0) * q * q * q + 16.0 * q * q * p), 0,
             fom_shifted_solve(K, p, q, s->fA, s->qcap, sA, s->eval, s->fYt, s->qcap, sC, s->fY, s->fwork,
                               s->d_kactive, nullptr, f32 ? 1 : 0, s->st));
    PROF_RUN(P_FOM_RES, 2.0 * K * q * nm * sizeof(V) + 2.0 * s->blk * sizeof(V), 16.0 * K * nm * q * p, 0, {
      dense_gemm_nn(K, q, p, p, s->fY, sC, s->qcap, s->sigvh, (size_t)p * p, p, s->fYt, sC, s->qcap, ONE, ZERO,
                    s->d_kactive, s->st, s->g.df64);
      // fYt now holds Y.  Res = C - (W Y - V Y Sigma)
      O::nn(K, nm, q, p, fW, sV, nm, s->fYt, sC, s->qcap, t1, sb, nm, ONE, ZERO, s->d_kactive, s->st, s->g.df64);
      dense_gemm_nn(K, q, p, p, s->fYt, sC, s->qcap, s->sig, (size_t)p * p, p, s->fY, sC, s->qcap, ONE, ZERO,
                    s->d_kactive, s->st, s->g.df64);
      O::nn(K, nm, q, p, fV, sV, nm, s->fY, sC, s->qcap, t1, sb, nm, MONE, ONE, s->d_kactive, s->st, s->g.df64);
      O::axpby(s->blk, ONE, C, MONE, t1, t1, s->st);
      O::norms2(K, sb, t1, s->d_out + 64, s->st);
    });
    CKL(s);
    TRY(sync_read(s, 64 + K));
    bool any = false;
    for (int k = 0; k < K; ++k) {
      s->h_int[2 * K + k] = 0;
      if (!active[k]) continue;
      iters[k] = j;
      const double rel = std::sqrt(s->h_out[64 + k]) / cnorm[k];
      if (!(rel <= s->prm.fom_rtol) && j < s->prm.max_fom) {
        any = true;
      } else {
        s->h_int[2 * K + k] = 1;  // take Y now
      }
      if (!std::isfinite(rel)) {
        s->err = "non-finite FOM residual";
        return EACG_EBREAKDOWN;
      }
    }
    CK(cudaMemcpyAsync(s->d_take, s->h_int + 2 * K, sizeof(int) * K, cudaMemcpyHostToDevice, s->st));
    small_take_y(K, q, s->qcap, p, s->fYt, s->fYf, s->d_take, s->st);
    for (int k = 0; k < K; ++k)
      if (s->h_int[2 * K + k]) active[k] = 0;
    if (!any) break;
    // next block: R_j = P^{-1} Res, orthonormalised against V_j
    TRY(fom_reserve(s, q + p));
    fV = reinterpret_cast<V*>(s->fV);
    TRY(upload_active());
    O::tpa(K, p, nm, s->d_kin, s->alpha, t1, t2, s->st);
    cudaMemsetAsync(vt, 0, sizeof(V) * s->blk, s->st);
    cudaMemsetAsync(wt, 0, sizeof(V) * s->blk, s->st);
    PROF_RUN(P_FOM_ORTH, 4.0 * K * q * nm * sizeof(V), 32.0 * K * nm * q * p, 0,
             TRY(orthonormalise<T>(s, t2, fV, q, (size_t)s->qcap * nm, vt, t3, s->d_kactive)));
    CK(cudaMemcpyAsync(s->h_int + K, s->d_nzero, sizeof(int) * K, cudaMemcpyDeviceToHost, s->st));
    CK(stream_wait(s));
    bool any2 = false;
    for (int k = 0; k < K; ++k) {
      if (active[k] && s->h_int[K + k] >= p) {
        // rank 0: the iteration ends with the current Y
        s->h_int[2 * K + k] = 1;
        active[k] = 0;
      } else {
        s->h_int[2 * K + k] = 0;
      }
      any2 |= active[k] != 0;
    }
    CK(cudaMemcpyAsync(s->d_take, s->h_int + 2 * K, sizeof(int) * K, cudaMemcpyHostToDevice, s->st));
    small_take_y(K, q, s->qcap, p, s->fYt, s->fYf, s->d_take, s->st);
    if (!any2) break;
    TRY(upload_active());
    TRY(apply_H_fom(s, vt, wt, s->d_kactive));
    TRY(put_cols(s, vt, wt, q));
    // the H application above advanced h_apps by all K; keep the per-k count honest
    {
      int na = 0;
      for (int k = 0; k < K; ++k) na += active[k];
      s->h_apps -= (long long)(K - na) * p;
    }
    PROF_RUN(P_FOM_BLOCK, 1.0 * K * q * nm * sizeof(V), 8.0 * K * nm * q * p, 0, TRY(add_block(q)));
    q += p;
  }
  // X = Phi / mu + V Y_final;  G = Phi - X (Phi^* X)^{-1}
  const size_t sC = (size_t)s->qcap * p;
  PROF_RUN(P_FOM_FINAL, 1.0 * K * q * nm * sizeof(V) + 6.0 * s->blk * 16, 8.0 * K * nm * q * p, 0, {
    dense_axpby(s->blk, cr(1.0 / mu), phi, ZERO, nullptr, s->Xb, s->st);
    if (!f32) {
      dense_gemm_nn(K, nm, q, p, s->fV, (size_t)s->qcap * nm, nm, s->fYf, sC, s->qcap, s->Xb, sb, nm, ONE, ONE,
                    nullptr, s->st, s->g.df64);
    } else {
      O::nn(K, nm, q, p, reinterpret_cast<V*>(s->fV), (size_t)s->qcap * nm, nm, s->fYf, sC, s->qcap, t1, sb, nm, ONE,
            ZERO, nullptr, s->st, s->g.df64);
      dense_to64(s->blk, reinterpret_cast<float2*>(s->tmp1), s->tmp3, s->st);
      dense_axpby(s->blk, ONE, s->Xb, ONE, s->tmp3, s->Xb, s->st);
    }
    dense_gemm_cn(K, nm, p, p, phi, sb, nm, s->Xb, sb, nm, s->sm1, (size_t)p * p, p, ONE, ZERO, s->cn_work, nullptr,
                  s->st, s->g.df64);
    dense_inverse(K, p, s->sm1, s->sm2, nullptr, s->st, s->ppscr);
    dense_copy(g, phi, s->blk, s->st);
    dense_gemm_nn(K, nm, p, p, s->Xb, sb, nm, s->sm2, (size_t)p * p, p, g, sb, nm, MONE, ONE, nullptr, s->st, s->g.df64);
  });
  CKL(s);
  int mx = 0;
  for (int k = 0; k < K; ++k) mx = std::max(mx, iters[k]);
  s->last_fom_max = mx;
  if (fom_iters)
    for (int k = 0; k < K; ++k) fom_iters[k] = iters[k];
  return EACG_OK;
}

// prec 0: FP64 FOM; 1: FP32 Krylov blocks, transforms and projected solves.
static eacg_status ea_gradient(eacg_system* s, const double2* phi, const double2* hphi, const double2* lam,
                               double2* g, int prec, int* fom_iters) {
  if (prec) return ea_gradient_t<float>(s, phi, hphi, lam, g, fom_iters);
  return ea_gradient_t<double>(s, phi, hphi, lam, g, fom_iters);
}

// ============================================================================ line search
// f(t) = E(pf(Phi + t eta)), f'(t) = 2 f <R(t), T_{t eta}(eta)> (Algorithm 2 input).  The trial
// point, its H Phi, R, Lambda, transport of eta and S^{-1} stay in the *_t buffers.
struct TrialOut {
  EvalOut ev;
  double df;
};

static eacg_status trial(eacg_system* s, double t, int prec, TrialOut* out) {
  const int K = s->K, p = s->p, nm = s->n_max;
  const size_t sb = (size_t)p * nm;
  dense_axpby(s->blk, ONE, s->phi, cr(t), s->eta, s->psi_t, s->st);
  PROF_RUN(P_TRIAL_RET, 8.0 * s->blk * 16, 40.0 * s->blk * p, 0, {
    TRY(polar(s, s->psi_t, s->phi_t, s->eval_t, s->evec_t, s->sinv_t));
    // T(eta) = eta S^{-1} - t Phi+ [[eta S^{-1}, eta S^{-1}]]
    dense_gemm_nn(K, nm, p, p, s->eta, sb, nm, s->sinv_t, (size_t)p * p, p, s->teta_t, sb, nm, ONE, ZERO, nullptr,
                  s->st, s->g.df64);
    dense_gemm_cn(K, nm, p, p, s->teta_t, sb, nm, s->teta_t, sb, nm, s->sm2, (size_t)p * p, p, ONE, ZERO,
                  s->cn_work, nullptr, s->st, s->g.df64);
    dense_gemm_nn(K, nm, p, p, s->phi_t, sb, nm, s->sm2, (size_t)p * p, p, s->teta_t, sb, nm, cr(-t), ONE, nullptr,
                  s->st, s->g.df64);
  });
  CKL(s);
  TRY(evaluate(s, s->phi_t, s->hphi_t, s->res_t, s->lam_t, prec, &out->ev));
  pairing_dev(s, s->res_t, s->teta_t, 0, true);
  TRY(sync_read(s, 1));
  out->df = 2.0 * s->occ * s->h_out[0];
  ++s->ls_total;
  return EACG_OK;
}

// EARGD (the paper's gradient-descent comparator; details are the readings listed with the
// library): tau0 gamma^j for the first j with f(tau) <= C + NM_DELTA tau f'(0), C the
// Zhang-Hager reference value.  The accepted point is the last trial evaluated.
constexpr double NM_RHO = 0.85, NM_DELTA = 1e-4;
static eacg_status trial(eacg_system* s, double t, int prec, TrialOut* out);
static eacg_status nonmonotone(eacg_system* s, double df0, double tau0, int prec, double* tau_out, TrialOut* acc,
                               int* trials_out) {
  double t = tau0;
  for (int n = 1; n <= s->prm.max_ls; ++n) {
    TRY(trial(s, t, prec, acc));
    if (acc->ev.E <= s->nm_C + NM_DELTA * t * df0) {
      *tau_out = t;
      *trials_out = n;
      return EACG_OK;
    }
    t *= s->prm.gamma;
  }
  s->err = "non-monotone backtracking: no acceptable step within max_ls trials";
  return EACG_ELINESEARCH;
}

// Algorithm 2 (with the readings stated in the header): returns the accepted step in *tau;
// the accepted point is the last trial evaluated.
static eacg_status modified_secant(eacg_system* s, double f0, double df0, double tau0, int prec, double* tau_out,
                                   TrialOut* acc, int* trials_out) {
  const eacg_params& P = s->prm;
  const double ftol = f0 + P.eps * std::fabs(f0);
  const double cmax = std::min(P.sigma, 1.0 - 2.0 * P.delta) * std::fabs(df0);
  int trials = 0;
  auto ev = [&](double t, TrialOut* o) -> eacg_status {
    if (trials >= P.max_ls) {
      s->err = "step-size search reached its trial cap";
      return EACG_ELINESEARCH;
    }
    ++trials;
    return trial(s, t, prec, o);
  };
  double a = 0.0, dfa = df0, b = tau0;
  TrialOut tb;
  TRY(ev(b, &tb));
  double fb = tb.ev.E, dfb = tb.df;
  double cur_t = b;
  TrialOut cur = tb;
  while (!(cur.ev.E <= ftol && std::fabs(cur.df) <= cmax)) {
    const double den = dfb - dfa;
    double tau = std::fabs(den) >= 1e-300 ? (a * dfb - b * dfa) / den : NAN;
    if (!std::isfinite(tau)) {
      b = P.gamma * b;
      a = 0.0;
      dfa = df0;
      TRY(ev(b, &tb));
      fb = tb.ev.E;
      dfb = tb.df;
      cur_t = b;
      cur = tb;
      continue;
    }
    if (tau < a) {
      b = b / P.gamma;
      a = 0.0;
      dfa = df0;
      TRY(ev(b, &tb));
      fb = tb.ev.E;
      dfb = tb.df;
      cur_t = b;
      cur = tb;
      continue;
    }
    TrialOut tt;
    TRY(ev(tau, &tt));
    if (tt.ev.E > ftol && tt.df < 0) {
      b = P.gamma * b;
      a = 0.0;
      dfa = df0;
      TRY(ev(b, &tb));
      fb = tb.ev.E;
      dfb = tb.df;
      cur_t = b;
      cur = tb;
    } else if (tau > b) {
      a = b;
      dfa = dfb;
      b = tau;
      fb = tt.ev.E;
      dfb = tt.df;
      cur_t = tau;
      cur = tt;
    } else {
      if (tt.df >= 0) {
        b = tau;
        fb = tt.ev.E;
        dfb = tt.df;
      } else {
        a = tau;
        dfa = tt.df;
      }
      cur_t = tau;
      cur = tt;
    }
  }
  (void)fb;
  *tau_out = cur_t;
  *acc = cur;
  *trials_out = trials;
  return EACG_OK;
}

// T_{tau eta}(g) = (g - Phi+ X) S^{-1}, S X + X S = tau ([[eta, g]] + [[g, eta]]) with S = Sf(Phi + tau eta)
// from the accepted trial (eigenvectors evec_t, eigenvalues sqrt(eval_t)).
static eacg_status transport_g(eacg_system* s, double tau) {
  const int K = s->K, p = s->p, nm = s->n_max;
  const size_t sb = (size_t)p * nm;
  dense_gemm_cn(K, nm, p, p, s->eta, sb, nm, s->gv, sb, nm, s->sm1, (size_t)p * p, p, ONE, ZERO, s->cn_work, nullptr,
                s->st, s->g.df64);
  small_add_herm(K, p, s->sm1, tau, s->sm2, s->st);  // sm2 = tau (M + M^H)
  small_sqrt_vals(K, p, s->eval_t, s->sqd, s->st);
  dense_lyapunov(K, p, s->evec_t, s->sqd, s->sm2, s->sm3, s->st, s->ppscr);
  dense_copy(s->tmp1, s->gv, s->blk, s->st);
  dense_gemm_nn(K, nm, p, p, s->phi_t, sb, nm, s->sm3, (size_t)p * p, p, s->tmp1, sb, nm, MONE, ONE, nullptr, s->st, s->g.df64);
  dense_gemm_nn(K, nm, p, p, s->tmp1, sb, nm, s->sinv_t, (size_t)p * p, p, s->tg, sb, nm, ONE, ZERO, nullptr, s->st, s->g.df64);
  CKL(s);
  return EACG_OK;
}

// g at the current point: EA gradient, or the preconditioned direction in the warm-up or when
// <r, g_EA> <= 0.  Returns <r, g> in *rg and the kind (1 EA, 0 preconditioned) in *kind.
static eacg_status direction(eacg_system* s, int prec, double* rg, int* kind) {
  if (s->phase == 1) {
    // The FOM stops at a relative Sylvester residual of 2.5e-2, five orders above FP32
    // rounding: in mixed mode its H applications and projected solves stay in FP32 at every
    // residual level (the residual, energy and retraction stay FP64).
    (void)prec;
    TRY(ea_gradient(s, s->phi, s->hphi, s->lam, s->gv, s->prm.precision ? 1 : 0, nullptr));
    pairing_dev(s, s->res, s->gv, 0, true);
    TRY(sync_read(s, 1));
    if (s->h_out[0] > 0) {
      *rg = s->h_out[0];
      *kind = 1;
      return EACG_OK;
    }
  }
  TRY(precond_gradient(s, s->phi, s->res, s->gv));
  pairing_dev(s, s->res, s->gv, 0, true);
  TRY(sync_read(s, 1));
  *rg = s->h_out[0];
  *kind = 0;
  return EACG_OK;
}

static int step_precision(const eacg_system* s) {
  if (s->prm.precision == 0) return 0;
  return s->rnorm > s->prm.switch_res ? 1 : 0;
}

static void swap_trial_into_current(eacg_system* s) {
  std::swap(s->phi, s->phi_t);
  std::swap(s->hphi, s->hphi_t);
  std::swap(s->res, s->res_t);
  std::swap(s->lam, s->lam_t);
  std::swap(s->teta, s->teta_t);
}

static eacg_status start_iteration(eacg_system* s) {
  EvalOut ev;
  s->cur_prec = s->prm.precision ? 1 : 0;
  TRY(evaluate(s, s->phi, s->hphi, s->res, s->lam, s->cur_prec, &ev));
  s->eval_prec = s->cur_prec;
  s->E = ev.E;
  s->rnorm = ev.rnorm;
  std::memcpy(s->eterms, ev.terms, sizeof(ev.terms));
  s->phase = (s->prm.max_warm > 0 && s->rnorm > s->prm.warm_res) ? 0 : 1;
  s->iter = 0;
  s->warm_iter = 0;
  s->tau = 1.0;
  s->nm_C = s->E;
  s->nm_Q = 1.0;
  s->ea_steps = 0;
  s->fresh = 0;
  if (s->rnorm <= s->prm.res_tol) return EACG_OK;
  int kind;
  s->cur_prec = step_precision(s);
  TRY(direction(s, s->cur_prec, &s->rg, &kind));
  dense_axpby(s->blk, MONE, s->gv, ZERO, nullptr, s->eta, s->st);
  CKL(s);
  return EACG_OK;
}

// The current point evaluated again with transforms of precision prec (mixed mode, when the
// step's precision differs from the one its energy came from): the step-size test of
// Algorithm 2 then compares energies and slopes of one precision.  The direction is kept while
// it is still a descent direction for the new residual, else it restarts from -g.
static eacg_status reevaluate(eacg_system* s, int prec) {
  EvalOut ev;
  TRY(evaluate(s, s->phi, s->hphi, s->res, s->lam, prec, &ev));
  s->E = ev.E;
  s->rnorm = ev.rnorm;
  std::memcpy(s->eterms, ev.terms, sizeof(ev.terms));
  s->eval_prec = prec;
  if (s->rnorm <= s->prm.res_tol) return EACG_OK;
  pairing_dev(s, s->res, s->eta, 0, true);
  pairing_dev(s, s->res, s->gv, 1, true);
  CKL(s);
  TRY(sync_read(s, 2));
  s->rg = s->h_out[1];
  if (!(s->h_out[0] < 0)) {
    int kind;
    TRY(direction(s, prec, &s->rg, &kind));
    dense_axpby(s->blk, MONE, s->gv, ZERO, nullptr, s->eta, s->st);
    CKL(s);
  }
  return EACG_OK;
}

static eacg_status do_step(eacg_system* s, eacg_step_info* info) {
  if (!s->have_psi) {
    s->err = "no iterate: call eacg_set_psi first";
    return EACG_EINVAL;
  }
  if (s->fresh) TRY(start_iteration(s));
  if (info) std::memset(info, 0, sizeof(*info));
  int prec = step_precision(s);
  if (s->rnorm > s->prm.res_tol && prec != s->eval_prec) TRY(reevaluate(s, prec));
  if (s->rnorm <= s->prm.res_tol) {
    if (info) {
      info->E = s->E;
      info->rnorm = s->rnorm;
      info->converged = 1;
      info->phase = s->phase;
      info->h_band_apps = s->h_apps;
    }
    return EACG_OK;
  }
  if (s->iter >= s->prm.max_outer) {
    s->err = "outer iteration cap reached";
    return EACG_ENOTCONV;
  }
  // f'(0) = 2 f <r, eta>
  pairing_dev(s, s->res, s->eta, 0, true);
  TRY(sync_read(s, 1));
  double df0 = 2.0 * s->occ * s->h_out[0];
  double tau = 0;
  TrialOut acc;
  int trials = 0;
  const bool gd = s->prm.method == 1 && s->phase == 1;  // EARGD step
  auto search = [&]() {
    return gd ? nonmonotone(s, df0, s->tau, prec, &tau, &acc, &trials)
              : modified_secant(s, s->E, df0, s->tau, prec, &tau, &acc, &trials);
  };
  eacg_status st = search();
  if (st == EACG_ELINESEARCH && prec == 1) {
    // FP32 transforms can no longer resolve the energy decrease: continue in FP64, from the
    // current point evaluated in FP64
    s->prm.switch_res = std::max(s->prm.switch_res, 2.0 * s->rnorm);
    prec = 0;
    TRY(reevaluate(s, 0));
    if (s->rnorm <= s->prm.res_tol) {
      if (info) {
        info->E = s->E;
        info->rnorm = s->rnorm;
        info->converged = 1;
        info->phase = s->phase;
        info->h_band_apps = s->h_apps;
      }
      return EACG_OK;
    }
    pairing_dev(s, s->res, s->eta, 0, true);
    TRY(sync_read(s, 1));
    df0 = 2.0 * s->occ * s->h_out[0];
    st = search();
  }
  if (st != EACG_OK) return st;
  s->eval_prec = prec;  // the accepted trial becomes the current point
  if (gd) {
    const double Qn = NM_RHO * s->nm_Q + 1.0;
    s->nm_C = (NM_RHO * s->nm_Q * s->nm_C + acc.ev.E) / Qn;
    s->nm_Q = Qn;
    s->ea_steps += 1;
  }
  s->iter += 1;
  if (s->phase == 0) s->warm_iter += 1;
  // transport of the old g (needs old Phi, eta, g and the accepted trial's S)
  TRY(transport_g(s, tau));
  const bool sw = s->phase == 0 && (acc.ev.rnorm <= s->prm.warm_res || s->warm_iter >= s->prm.max_warm);
  if (sw) s->phase = 1;
  swap_trial_into_current(s);
  s->E = acc.ev.E;
  s->rnorm = acc.ev.rnorm;
  std::memcpy(s->eterms, acc.ev.terms, sizeof(acc.ev.terms));
  s->tau = tau;
  double beta = 0.0;
  int kind = 0;
  if (s->rnorm > s->prm.res_tol) {
    // the potential in the system is the accepted trial's (the last one evaluated)
    const int dprec = step_precision(s) && prec;
    double rgn;
    TRY(direction(s, dprec, &rgn, &kind));
    if (sw) {
      beta = 0.0;
      s->tau = 1.0;
      s->nm_C = s->E;
      s->nm_Q = 1.0;
      s->ea_steps = 0;
    } else if (gd) {
      // alternating Barzilai-Borwein step from s = tau T(eta), y = g_new - T(g_old)
      beta = 0.0;
      dense_axpby(s->blk, ONE, s->gv, MONE, s->tg, s->tmp2, s->st);
      pairing_dev(s, s->teta, s->teta, 0, true);
      pairing_dev(s, s->teta, s->tmp2, 1, true);
      pairing_dev(s, s->tmp2, s->tmp2, 2, true);
      TRY(sync_read(s, 3));
      const double ss = tau * tau * s->h_out[0], sy = std::fabs(tau * s->h_out[1]), yy = s->h_out[2];
      double t = (s->ea_steps % 2 == 1) ? ss / sy : sy / yy;
      if (!std::isfinite(t) || t <= 0.0) t = 1.0;
      s->tau = std::min(std::max(t, 1e-10), 1e10);
    } else {
      pairing_dev(s, s->res, s->tg, 0, true);
      TRY(sync_read(s, 1));
      const double bfr = rgn / s->rg;
      const double bprp = (rgn - s->h_out[0]) / s->rg;
      beta = std::max(0.0, std::min(bfr, bprp));
    }
    // eta = -g + beta T(eta)
    dense_axpby(s->blk, MONE, s->gv, cr(beta), s->teta, s->eta, s->st);
    pairing_dev(s, s->res, s->eta, 0, true);
    TRY(sync_read(s, 1));
    if (s->h_out[0] >= 0) {
      dense_axpby(s->blk, MONE, s->gv, ZERO, nullptr, s->eta, s->st);
      beta = 0.0;
    }
    CKL(s);
    s->rg = rgn;
  }
  if (info) {
    info->E = s->E;
    info->rnorm = s->rnorm;
    info->tau = tau;
    info->beta = beta;
    info->fom_iters_max = s->phase == 1 ? s->last_fom_max : 0;
    info->ls_trials = trials;
    info->phase = s->phase;
    info->precision = prec;
    info->converged = s->rnorm <= s->prm.res_tol;
    info->h_band_apps = s->h_apps;
  }
  return EACG_OK;
}

// ============================================================================ C ABI
#define SYS_CHECK(sys)                      \
  do {                                      \
    if (!(sys)) return EACG_EINVAL;         \
  } while (0)

// Calls that need the p x p dense kernels (eigen-decompositions, inverses, Lyapunov solves,
// pivoted Cholesky, projected FOM solves): one CTA per k, up to 512 bands.
#define DENSE_CHECK(sys)                                                                         \
  do {                                                                                           \
    if ((sys)->p > EACG_MAX_BANDS_DENSE) {                                                      \
      (sys)->err = "this call needs the p x p dense kernels, which support at most 512 bands";   \
      return EACG_EUNSUPPORTED;                                                                  \
    }                                                                                            \
  } while (0)

// ---- autotune of the line-FFT plan
// For grid sizes with two compiled line plans, time both on this system's transform pipeline
// (inverse x pass, plane, forward x pass over all bands) in each precision and keep the faster.
// The two plans round differently, so plan 1 replaces the default plan 0 only when it is at
// least 3 % faster: near-ties, where timing noise could flip the choice from one run or GPU to
// the next, resolve to plan 0 and the results stay reproducible.  The transforms' time does not
// depend on the values, so zeroed buffers are used.  Choices are cached per (device, N,
// columns, rows, bands, n_max) for the whole process.
namespace {
std::mutex g_tune_mu;
std::map<std::array<int, 6>, std::pair<int, int>> g_tune;
}  // namespace

static eacg_status autotune_plans(eacg_system* s) {
  s->g.plan64 = s->g.plan32 = 0;
  if (!grid_has_plan1(s->N)) return EACG_OK;
  if (s->prm.fft_plan == 0 || s->prm.fft_plan == 1) {
    s->g.plan64 = s->g.plan32 = s->prm.fft_plan;
    return EACG_OK;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  const std::array<int, 6> key = {dev, s->N, s->ncols, s->ny, s->K * s->p, s->n_max};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      s->g.plan64 = it->second.first;
      s->g.plan32 = it->second.second;
      return EACG_OK;
    }
  }
  const int nb = s->K * s->p;
  CK(cudaMemsetAsync(s->phi, 0, sizeof(double2) * s->blk, s->st));
  CK(cudaMemsetAsync(s->d_tbuf, 0, sizeof(double2) * (size_t)nb * s->N * s->ncols, s->st));
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  int choice[2] = {0, 0};
  for (int prec = 0; prec < 2; ++prec) {
    const void* v = vpot(s, prec);
    const int reps = prec == 0 ? 1 : 4;
    float best = 0.f;
    for (int plan = 0; plan < 2; ++plan) {
      (prec == 0 ? s->g.plan64 : s->g.plan32) = plan;
      auto run = [&]() {
        grid_xpass_inv(s->g, prec, s->phi, s->d_tbuf, nb, nullptr, s->st);
        grid_plane_h(s->g, prec, s->d_tbuf, v, nb, nullptr, s->st);
        grid_xpass_fwd(s->g, prec, s->d_tbuf, s->phi, nullptr, 1.0, s->tmp1, nb, nullptr, s->st);
      };
      run();  // first launch of each kernel outside the timing
      CK(cudaEventRecord(a, s->st));
      for (int r = 0; r < reps; ++r) run();
      CK(cudaEventRecord(b, s->st));
      CK(cudaEventSynchronize(b));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, a, b));
      if (plan == 0) {
        best = ms;
      } else if (ms < 0.97f * best) {
        choice[prec] = plan;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  CKL(s);
  s->g.plan64 = choice[0];
  s->g.plan32 = choice[1];
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = {choice[0], choice[1]};
  return EACG_OK;
}

// ---- autotune of the A^H B tiles: the shapes this system uses (Gram p x p, projector overlaps
// nproj x p, the FOM's q x p for q up to 16 p), both block precisions, on temporary operands
// of at most 8 k-points (the choice is recorded per shape bucket for the whole process).
static eacg_status autotune_gemm(eacg_system* s) {
  const int p = s->p, nm = s->n_max, Kt = std::min(s->K, 8);
  // Krylov shapes q x p exist only where the FOM runs (p within the dense kernels' limit)
  const bool fom = p <= EACG_MAX_BANDS_DENSE;
  const int mmax = fom ? std::min(16 * p, 1024) : p;
  std::vector<int> ms = fom ? std::vector<int>{p, 2 * p, 4 * p, 8 * p, 16 * p} : std::vector<int>{p};
  if (s->nproj > 0) ms.push_back(s->nproj);
  double2 *A = nullptr, *C = nullptr, *W = nullptr;
  const size_t na = (size_t)Kt * std::max(mmax, s->nproj) * nm;
  if (cudaMalloc(&A, sizeof(double2) * na) != cudaSuccess) {
    cudaGetLastError();
    return EACG_OK;  // tuning is optional: untuned shapes use the default tile
  }
  const int mm = std::max(mmax, s->nproj);
  const size_t nc = (size_t)Kt * mm * p, nw = dense_cn_work(Kt, nm, mm, p);
  if (cudaMalloc(&C, sizeof(double2) * nc) != cudaSuccess || cudaMalloc(&W, sizeof(double2) * nw) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(A);
    if (C) cudaFree(C);
    return EACG_OK;
  }
  CK(cudaMemsetAsync(A, 0, sizeof(double2) * na, s->st));
  for (int prec = 0; prec < 2; ++prec)
    for (int m : ms) {
      if (m > mm) continue;
      dense_tune_cn(Kt, nm, m, p, prec, A, (size_t)m * nm, nm, A, (size_t)m * nm, nm, C, W, s->st);
    }
  cudaStreamSynchronize(s->st);
  cudaFree(A);
  cudaFree(C);
  cudaFree(W);
  CKL(s);
  return EACG_OK;
}

extern "C" eacg_status eacg_create_system(const eacg_model* m, const eacg_params* prm, void* stream,
                                          eacg_system** out) {
  if (!out) return EACG_EINVAL;
  *out = nullptr;
  std::string why;
  eacg_status v = validate(m, prm, &why);
  if (v != EACG_OK) return v;
  eacg_system* s = new eacg_system();
  s->st = (cudaStream_t)stream;
  if (prm)
    s->prm = *prm;
  else
    eacg_default_params(&s->prm);
  s->N = m->N;
  s->K = m->nk;
  s->p = m->nbands;
  s->natoms = m->natoms;
  s->npa = m->nproj_per_atom;
  s->nproj = m->natoms * m->nproj_per_atom;
  s->hartree = m->hartree;
  s->xc = m->xc;
  s->a = m->a;
  s->omega = m->a * m->a * m->a;
  s->b = 2.0 * M_PI / m->a;
  s->ecut = m->ecut;
  s->occ = m->occ;
  s->width = m->proj_width;
  s->thr = (2.0 * m->ecut) / (s->b * s->b);
  s->kfrac.assign(m->kfrac, m->kfrac + 3 * m->nk);
  s->kw.assign(m->kweight, m->kweight + m->nk);
  for (int i = 0; i < m->natoms; ++i) {
    for (int c = 0; c < 3; ++c) s->pos.push_back(m->pos[3 * i + c]);
    s->Z.push_back((double)m->Z[i]);
    s->rc.push_back(m->rc[i]);
    for (int l = 0; l < m->nproj_per_atom; ++l) s->dvec.push_back(l == 0 ? m->D[2 * i] : m->D[2 * i + 1]);
  }
  auto fail = [&](eacg_status st) {
    eacg_destroy(s);
    return st;
  };
  auto up = [&](double** d, const std::vector<double>& h) -> eacg_status {
    TRY(dalloc(s, d, sizeof(double) * std::max<size_t>(1, h.size())));
    if (!h.empty()) {
      cudaError_t e = cudaMemcpyAsync(*d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s->st);
      if (e != cudaSuccess) {
        s->err = cudaGetErrorString(e);
        return EACG_ECUDA;
      }
    }
    return EACG_OK;
  };
  eacg_status st;
  if ((st = up(&s->d_kfrac, s->kfrac)) != EACG_OK) return fail(st);
  if ((st = up(&s->d_kw, s->kw)) != EACG_OK) return fail(st);
  if ((st = up(&s->d_pos, s->pos)) != EACG_OK) return fail(st);
  if ((st = up(&s->d_Z, s->Z)) != EACG_OK) return fail(st);
  if ((st = up(&s->d_rc, s->rc)) != EACG_OK) return fail(st);
  if ((st = up(&s->d_dvec, s->dvec)) != EACG_OK) return fail(st);
  // FFT twiddles e^{-2 pi i k / N}
  s->g.N = s->N;
  {
    std::vector<double2> tw(s->N);
    std::vector<float2> tw32(s->N);
    for (int k = 0; k < s->N; ++k) {
      const double ang = 2.0 * M_PI * (double)k / (double)s->N;
      tw[k] = make_double2(std::cos(ang), -std::sin(ang));
      tw32[k] = make_float2((float)tw[k].x, (float)tw[k].y);
    }
    // double-float twiddles: each component as its nearest (hi, lo) FP32 pair
    std::vector<float> twdf(4 * (size_t)s->N);
    for (int k = 0; k < s->N; ++k) {
      const double c[2] = {tw[k].x, tw[k].y};
      for (int q = 0; q < 2; ++q) {
        const float hi = (float)c[q];
        twdf[4 * k + 2 * q] = hi;
        twdf[4 * k + 2 * q + 1] = (float)(c[q] - (double)hi);
      }
    }
    if ((st = dalloc(s, &s->d_tw64, sizeof(double2) * s->N)) != EACG_OK) return fail(st);
    if ((st = dalloc(s, &s->d_tw32, sizeof(float2) * s->N)) != EACG_OK) return fail(st);
    if ((st = dalloc(s, &s->d_twdf, sizeof(float) * twdf.size())) != EACG_OK) return fail(st);
    cudaMemcpyAsync(s->d_tw64, tw.data(), sizeof(double2) * s->N, cudaMemcpyHostToDevice, s->st);
    cudaMemcpyAsync(s->d_tw32, tw32.data(), sizeof(float2) * s->N, cudaMemcpyHostToDevice, s->st);
    cudaMemcpyAsync(s->d_twdf, twdf.data(), sizeof(float) * twdf.size(), cudaMemcpyHostToDevice, s->st);
    if (cudaStreamSynchronize(s->st) != cudaSuccess) {
      s->err = "stream synchronise failed during set-up";
      return fail(EACG_ECUDA);
    }
  }
  if ((st = build_basis(s)) != EACG_OK) return fail(st);
  s->g.K = s->K;
  s->g.p = s->p;
  s->g.n_max = s->n_max;
  s->g.ncols = s->ncols;
  s->g.ny = s->ny;
  s->g.nk = s->d_nk;
  s->g.xmap = s->d_xmap;
  s->g.cmapy = s->d_cmapy;
  s->g.rowmask = s->d_rowmask;
  s->g.ylist = s->d_ylist;
  s->g.tw64 = s->d_tw64;
  s->g.tw32 = s->d_tw32;
  s->g.twdf = s->d_twdf;
  s->g.df64 = s->prm.df_transforms ? 1 : 0;
  if ((st = build_potential_and_projectors(s)) != EACG_OK) return fail(st);
  s->tc_proj = s->prm.tensor_cores && s->nproj > 0 && dense_overlap_tc_eligible(s->nproj, s->p);
  if ((st = alloc_work(s)) != EACG_OK) return fail(st);
  if (cudaEventCreateWithFlags(&s->ev_sync, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    s->ev_sync = nullptr;  // waits fall back to cudaStreamSynchronize
  }
  if ((st = autotune_plans(s)) != EACG_OK) return fail(st);
  if ((st = autotune_gemm(s)) != EACG_OK) return fail(st);
  if (cudaStreamSynchronize(s->st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    s->err = "set-up kernels failed";
    return fail(EACG_ECUDA);
  }
  *out = s;
  return EACG_OK;
}

extern "C" void eacg_destroy(eacg_system* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  for (auto& g : s->hg) hg_release(g);
  for (cudaEvent_t e : s->evpool) cudaEventDestroy(e);
  if (s->ev_sync) cudaEventDestroy(s->ev_sync);
  for (void* p : s->allocs) cudaFree(p);
  if (s->h_out) cudaFreeHost(s->h_out);
  if (s->h_int) cudaFreeHost(s->h_int);
  delete s;
}

extern "C" eacg_status eacg_get_plans(const eacg_system* s, int* plan64, int* plan32) {
  SYS_CHECK(s);
  if (plan64) *plan64 = s->g.plan64;
  if (plan32) *plan32 = s->g.plan32;
  return EACG_OK;
}

extern "C" long long eacg_graph_launches(const eacg_system* s) { return s ? s->graph_launches : -1; }

extern "C" int eacg_gemm_tile(int m, int n, int L, int precision) {
  return dense_cn_groups(m, n, L, precision ? 1 : 0);
}

extern "C" eacg_status eacg_force_gemm_tile(int groups) {
  return dense_cn_force(groups) == 0 ? EACG_OK : EACG_EINVAL;
}

extern "C" const char* eacg_last_error(const eacg_system* s) { return s ? s->err.c_str() : "null system"; }

extern "C" eacg_status eacg_get_dims(const eacg_system* s, int* nk_host, int* n_max, int* ncols) {
  SYS_CHECK(s);
  if (nk_host)
    for (int k = 0; k < s->K; ++k) nk_host[k] = s->nk[k];
  if (n_max) *n_max = s->n_max;
  if (ncols) *ncols = s->ncols;
  return EACG_OK;
}

extern "C" eacg_status eacg_get_basis(const eacg_system* cs, int* m_dev) {
  SYS_CHECK(cs);
  eacg_system* s = const_cast<eacg_system*>(cs);
  if (!m_dev) return EACG_EINVAL;
  CK(cudaMemcpyAsync(m_dev, s->d_m, sizeof(int) * 3 * (size_t)s->K * s->n_max, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return EACG_OK;
}

extern "C" eacg_status eacg_set_psi(eacg_system* s, const double* psi_dev) {
  SYS_CHECK(s);
  DENSE_CHECK(s);
  if (!psi_dev) return EACG_EINVAL;
  CK(cudaMemcpyAsync(s->tmp2, psi_dev, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  TRY(polar(s, s->tmp2, s->phi, s->eval, s->evec, s->sm3));
  CK(cudaStreamSynchronize(s->st));
  s->have_psi = 1;
  s->fresh = 1;
  s->h_apps = 0;
  s->ls_total = 0;
  return EACG_OK;
}

extern "C" eacg_status eacg_get_psi(eacg_system* s, double* psi_dev_out) {
  SYS_CHECK(s);
  if (!psi_dev_out) return EACG_EINVAL;
  CK(cudaMemcpyAsync(psi_dev_out, s->phi, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return EACG_OK;
}

extern "C" eacg_status eacg_density(eacg_system* s, const double* psi_dev, double* rho_dev, int precision) {
  SYS_CHECK(s);
  if (!psi_dev) return EACG_EINVAL;
  TRY(density_and_potential(s, reinterpret_cast<const double2*>(psi_dev), precision ? 1 : 0));
  const size_t N3 = (size_t)s->N * s->N * s->N;
  if (rho_dev) CK(cudaMemcpyAsync(rho_dev, s->d_rho, sizeof(double) * N3, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return EACG_OK;
}

extern "C" eacg_status eacg_get_potential(eacg_system* s, double* vtot_dev) {
  SYS_CHECK(s);
  if (!vtot_dev) return EACG_EINVAL;
  const size_t N3 = (size_t)s->N * s->N * s->N;
  CK(cudaMemcpyAsync(vtot_dev, s->d_vtot, sizeof(double) * N3, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return EACG_OK;
}

extern "C" eacg_status eacg_apply_H(eacg_system* s, const double* psi_dev, double* hpsi_dev, int precision) {
  SYS_CHECK(s);
  if (!psi_dev || !hpsi_dev || psi_dev == hpsi_dev) return EACG_EINVAL;
  TRY(apply_H_block(s, reinterpret_cast<const double2*>(psi_dev), reinterpret_cast<double2*>(hpsi_dev),
                    precision ? 1 : 0, nullptr));
  CK(cudaStreamSynchronize(s->st));
  return EACG_OK;
}

extern "C" eacg_status eacg_energy(eacg_system* s, const double* psi_dev, double* terms, double* lam_dev,
                                   double* res_dev, double* rnorm, int precision) {
  SYS_CHECK(s);
  if (!psi_dev) return EACG_EINVAL;
  EvalOut ev;
  CK(cudaMemcpyAsync(s->tmp3, psi_dev, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  TRY(evaluate(s, s->tmp3, s->hphi_t, s->res_t, s->lam_t, precision ? 1 : 0, &ev));
  if (terms) {
    for (int i = 0; i < 5; ++i) terms[i] = ev.terms[i];
    terms[5] = ev.E;
  }
  if (rnorm) *rnorm = ev.rnorm;
  if (lam_dev)
    CK(cudaMemcpyAsync(lam_dev, s->lam_t, sizeof(double2) * (size_t)s->K * s->p * s->p, cudaMemcpyDeviceToDevice,
                       s->st));
  if (res_dev) CK(cudaMemcpyAsync(res_dev, s->res_t, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  s->fresh = 1;  // the trial buffers were used
  return EACG_OK;
}

extern "C" eacg_status eacg_ea_gradient(eacg_system* s, const double* psi_dev, double* g_dev, int* fom_iters,
                                        int precision) {
  SYS_CHECK(s);
  DENSE_CHECK(s);
  if (!psi_dev || !g_dev) return EACG_EINVAL;
  EvalOut ev;
  CK(cudaMemcpyAsync(s->phi_t, psi_dev, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  TRY(evaluate(s, s->phi_t, s->hphi_t, s->res_t, s->lam_t, precision ? 1 : 0, &ev));
  TRY(ea_gradient(s, s->phi_t, s->hphi_t, s->lam_t, s->teta_t, precision ? 1 : 0, fom_iters));
  CK(cudaMemcpyAsync(g_dev, s->teta_t, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  s->fresh = 1;
  return EACG_OK;
}

extern "C" eacg_status eacg_retract(eacg_system* s, const double* phi_dev, const double* eta_dev, double tau,
                                    double* phi_out_dev, double* teta_out_dev) {
  SYS_CHECK(s);
  DENSE_CHECK(s);
  if (!phi_dev || !eta_dev || !phi_out_dev) return EACG_EINVAL;
  const int K = s->K, p = s->p, nm = s->n_max;
  const size_t sb = (size_t)p * nm;
  dense_axpby(s->blk, ONE, reinterpret_cast<const double2*>(phi_dev), cr(tau),
              reinterpret_cast<const double2*>(eta_dev), s->psi_t, s->st);
  TRY(polar(s, s->psi_t, s->tmp1, s->eval_t, s->evec_t, s->sinv_t));
  if (teta_out_dev) {
    dense_gemm_nn(K, nm, p, p, reinterpret_cast<const double2*>(eta_dev), sb, nm, s->sinv_t, (size_t)p * p, p,
                  s->tmp2, sb, nm, ONE, ZERO, nullptr, s->st, s->g.df64);
    dense_gemm_cn(K, nm, p, p, s->tmp2, sb, nm, s->tmp2, sb, nm, s->sm2, (size_t)p * p, p, ONE, ZERO, s->cn_work,
                  nullptr, s->st, s->g.df64);
    dense_gemm_nn(K, nm, p, p, s->tmp1, sb, nm, s->sm2, (size_t)p * p, p, s->tmp2, sb, nm, cr(-tau), ONE, nullptr,
                  s->st, s->g.df64);
    CK(cudaMemcpyAsync(teta_out_dev, s->tmp2, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  }
  CK(cudaMemcpyAsync(phi_out_dev, s->tmp1, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  CKL(s);
  CK(cudaStreamSynchronize(s->st));
  s->fresh = 1;
  return EACG_OK;
}

// Initial guess of the experiments (Sec. 5.2): SCF iterations until the density difference of
// two successive iterates is below drho_tol.  Readings: the first input density is that of
// polar(psi0); one step minimises the band energy of the Hamiltonian of the input density (this
// library's warm-up and energy-adaptive iterations with the potential held fixed) to
// ||H Phi - Phi Lambda||_F <= eig_tol; ||rho_out - rho_in||_2 is the L2 norm over the cell;
// otherwise simple mixing rho_in <- rho_in + alpha (rho_out - rho_in).
extern "C" eacg_status eacg_scf_guess(eacg_system* s, const double* psi0_dev, double drho_tol, double alpha,
                                      int max_scf, double eig_tol, int* steps_out, double* history_host) {
  SYS_CHECK(s);
  DENSE_CHECK(s);
  if (!psi0_dev || !(drho_tol > 0) || !(alpha > 0 && alpha <= 1) || max_scf < 1 || !(eig_tol > 0))
    return EACG_EINVAL;
  if (steps_out) *steps_out = 0;
  const size_t N3 = (size_t)s->N * s->N * s->N;
  const size_t nh = N3 / 2;  // real grids viewed as complex pairs (every supported N is even)
  if (!s->d_rho_in) TRY(dalloc(s, &s->d_rho_in, sizeof(double) * N3));
  CK(cudaMemcpyAsync(s->tmp2, psi0_dev, sizeof(double2) * s->blk, cudaMemcpyDeviceToDevice, s->st));
  TRY(polar(s, s->tmp2, s->phi, s->eval, s->evec, s->sm3));
  s->have_psi = 1;
  s->h_apps = 0;
  s->ls_total = 0;
  TRY(density_only(s, s->phi, 0));
  CK(cudaMemcpyAsync(s->d_rho_in, s->d_rho, sizeof(double) * N3, cudaMemcpyDeviceToDevice, s->st));
  TRY(potential_from_rho(s));
  const eacg_params saved = s->prm;
  s->prm.res_tol = eig_tol;
  s->frozen = true;
  bool inner = false;  // an inner minimisation failed (its message is kept)
  double2* rin = reinterpret_cast<double2*>(s->d_rho_in);
  double2* rout = reinterpret_cast<double2*>(s->d_rho);
  double2* delta = s->d_fft3;  // scratch: rebuilt by the next potential build
  auto iterate = [&]() -> eacg_status {
    for (int step = 1; step <= max_scf; ++step) {
      s->fresh = 1;
      eacg_step_info info;
      eacg_status e = EACG_OK;
      do {
        e = do_step(s, &info);
      } while (e == EACG_OK && !info.converged);
      if (e != EACG_OK) {
        inner = true;
        return e;
      }
      TRY(density_only(s, s->phi, 0));
      dense_axpby(nh, ONE, rout, MONE, rin, delta, s->st);
      dense_norms2(1, nh, delta, s->d_out, s->st);
      CKL(s);
      TRY(sync_read(s, 1));
      const double d = std::sqrt(s->omega / (double)N3 * std::max(s->h_out[0], 0.0));
      if (history_host) history_host[step - 1] = d;
      if (steps_out) *steps_out = step;
      if (d < drho_tol) return EACG_OK;
      dense_axpby(nh, ONE, rin, cr(alpha), delta, rin, s->st);
      CK(cudaMemcpyAsync(s->d_rho, s->d_rho_in, sizeof(double) * N3, cudaMemcpyDeviceToDevice, s->st));
      TRY(potential_from_rho(s));
    }
    return EACG_ENOTCONV;
  };
  const eacg_status st = iterate();
  // leave the system in its normal mode whatever happened
  s->frozen = false;
  s->prm = saved;
  s->fresh = 1;  // the next step evaluates Phi with its own density and potential
  if (st == EACG_ENOTCONV && !inner) s->err = "SCF did not reach the density tolerance within max_scf steps";
  CK(cudaStreamSynchronize(s->st));
  return st;
}

extern "C" eacg_status eacg_overlap_c64(int K, int L, int m, int n, const float* a_dev, const float* b_dev,
                                        double* c_dev, int method, void* stream) {
  if (K < 0 || L < 0 || m < 0 || n < 0 || method < 0 || method > 1) return EACG_EINVAL;
  if (K == 0 || m == 0 || n == 0) return EACG_OK;
  if (!a_dev || !b_dev || !c_dev) return EACG_EINVAL;
  if (method == 1 && !dense_overlap_tc_eligible(m, n)) return EACG_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nw = std::max<size_t>(1, method ? dense_overlap_tc_work(K, L, m, n) : dense_cn_work(K, L, m, n));
  double2* work = nullptr;
  if (cudaMalloc(&work, sizeof(double2) * nw) != cudaSuccess) {
    cudaGetLastError();
    return EACG_ENOMEM;
  }
  const float2* A = reinterpret_cast<const float2*>(a_dev);
  const float2* B = reinterpret_cast<const float2*>(b_dev);
  double2* C = reinterpret_cast<double2*>(c_dev);
  const unsigned int gaveup0 = method ? dense_tc_gaveup_count(st) : 0u;
  if (method)
    dense_overlap_tf32x3(K, L, m, n, A, (size_t)m * L, L, B, (size_t)n * L, L, C, (size_t)m * n, m, ONE, ZERO, work,
                         nullptr, st);
  else
    dense_gemm_cn32(K, L, m, n, A, (size_t)m * L, L, B, (size_t)n * L, L, C, (size_t)m * n, m, ONE, ZERO, work,
                    nullptr, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFree(work);
  if (e == cudaSuccess && method && dense_tc_gaveup_count(st) != gaveup0) return EACG_ECUDA;
  return e == cudaSuccess ? EACG_OK : EACG_ECUDA;
}

extern "C" eacg_status eacg_backproject_c64(int K, int L, int m, int n, const float* a_dev, const double* q_dev,
                                            double* c_dev, int method, void* stream) {
  if (K < 0 || L < 0 || m < 0 || n < 0 || method < 0 || method > 1) return EACG_EINVAL;
  if (K == 0 || L == 0 || n == 0) return EACG_OK;
  if (!a_dev || !q_dev || !c_dev) return EACG_EINVAL;
  if (method == 1 && !dense_backproject_tc_eligible(m, n)) return EACG_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  const float2* A = reinterpret_cast<const float2*>(a_dev);
  const double2* Q = reinterpret_cast<const double2*>(q_dev);
  double2* C = reinterpret_cast<double2*>(c_dev);
  const unsigned int gaveup0 = (method && m > 0) ? dense_tc_gaveup_count(st) : 0u;
  if (m > 0) {
    if (method)
      dense_backproject_tf32x3(K, L, m, n, A, (size_t)m * L, L, Q, (size_t)n * m, m, C, (size_t)n * L, L, nullptr,
                               st);
    else
      dense_gemm_nn32_into64(K, L, m, n, A, (size_t)m * L, L, Q, (size_t)n * m, m, C, (size_t)n * L, L, ONE, ONE,
                             nullptr, st);
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess && method && m > 0 && dense_tc_gaveup_count(st) != gaveup0) return EACG_ECUDA;
  return e == cudaSuccess ? EACG_OK : EACG_ECUDA;
}

// One step of one system, inside the batcher b when it is not null.
static eacg_status step_in(eacg_system* s, eacg_step_info* info, Batcher* b) {
  if (b) {
    b->enter();
    tl_batch = b;
  }
  eacg_status st = do_step(s, info);
  if (b) {
    tl_batch = nullptr;
    b->leave();
  }
  if (st == EACG_OK) {
    cudaError_t e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
      s->err = cudaGetErrorString(e);
      return EACG_ECUDA;
    }
  }
  return st;
}

extern "C" eacg_status eacg_step(eacg_system* s, eacg_step_info* info) {
  SYS_CHECK(s);
  DENSE_CHECK(s);
  Batcher* b = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    b = g_batch;
  }
  return step_in(s, info, b);
}

extern "C" eacg_status eacg_step_many(eacg_system* const* sys, int nsys, eacg_step_info* infos, int* statuses,
                                      int window_us) {
  if (nsys < 0 || (nsys > 0 && !sys) || window_us < 0) return EACG_EINVAL;
  for (int i = 0; i < nsys; ++i) {
    if (!sys[i]) return EACG_EINVAL;
    if (sys[i]->p > EACG_MAX_BANDS_DENSE) {
      sys[i]->err = "this call needs the p x p dense kernels, which support at most 512 bands";
      return EACG_EUNSUPPORTED;
    }
    for (int j = 0; j < i; ++j)
      if (sys[j] == sys[i]) return EACG_EINVAL;  // a system steps once per call
  }
  Batcher b(window_us);
  std::vector<eacg_status> st(nsys, EACG_OK);
  std::vector<std::thread> th;
  th.reserve(nsys);
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < nsys; ++i)
    th.emplace_back([&, i] {
      cudaSetDevice(dev);  // the worker threads use the caller's device
      st[i] = step_in(sys[i], infos ? infos + i : nullptr, &b);
    });
  for (auto& t : th) t.join();
  eacg_status first = EACG_OK;
  for (int i = 0; i < nsys; ++i) {
    if (statuses) statuses[i] = st[i];
    if (first == EACG_OK && st[i] != EACG_OK) first = st[i];
  }
  return first;
}

extern "C" eacg_status eacg_batch_counts(long long* groups, long long* members) {
  if (groups) *groups = g_batch_groups.load();
  if (members) *members = g_batch_members.load();
  return EACG_OK;
}

extern "C" eacg_status eacg_batching(int window_us) {
  if (window_us < -1) return EACG_EINVAL;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  // the old batcher may still be in use by steps in flight: it is kept until process exit
  g_batch = window_us < 0 ? nullptr : new Batcher(window_us);
  return EACG_OK;
}

extern "C" eacg_status eacg_solve(eacg_system* s, eacg_result* out) {
  SYS_CHECK(s);
  DENSE_CHECK(s);
  eacg_status st = EACG_OK;
  eacg_step_info info;
  while (true) {
    st = do_step(s, &info);
    if (st != EACG_OK || info.converged) break;
  }
  if (out) {
    out->E = s->E;
    out->rnorm = s->rnorm;
    out->iterations = s->iter;
    out->warm_iterations = s->warm_iter;
    out->status = (int)st;
    out->ls_trials = s->ls_total;
    out->h_band_apps = s->h_apps;
  }
  cudaError_t e = cudaStreamSynchronize(s->st);
  if (st == EACG_OK && e != cudaSuccess) {
    s->err = cudaGetErrorString(e);
    return EACG_ECUDA;
  }
  return st;
}

extern "C" eacg_status eacg_solve_host(eacg_system* s, const double* psi0_host, double* psi_out_host,
                                       eacg_result* out) {
  SYS_CHECK(s);
  DENSE_CHECK(s);
  if (!psi0_host) return EACG_EINVAL;
  CK(cudaMemcpyAsync(s->tmp2, psi0_host, sizeof(double2) * s->blk, cudaMemcpyHostToDevice, s->st));
  TRY(polar(s, s->tmp2, s->phi, s->eval, s->evec, s->sm3));
  s->have_psi = 1;
  s->fresh = 1;
  s->h_apps = 0;
  s->ls_total = 0;
  eacg_status st = eacg_solve(s, out);
  if (psi_out_host) {
    CK(cudaMemcpyAsync(psi_out_host, s->phi, sizeof(double2) * s->blk, cudaMemcpyDeviceToHost, s->st));
    CK(cudaStreamSynchronize(s->st));
  }
  return st;
}

extern "C" eacg_status eacg_profile_enable(eacg_system* s, int on) {
  SYS_CHECK(s);
  CK(cudaStreamSynchronize(s->st));
  s->prof.clear();
  s->prof_ms.clear();
  for (auto& g : s->hg) g.pending = false;
  s->evused = 0;
  s->prof_on = on != 0;
  return EACG_OK;
}

extern "C" int eacg_profile_read(eacg_system* s, eacg_kernel_stat* out, int max) {
  if (!s) return -(int)EACG_EINVAL;
  if (cudaStreamSynchronize(s->st) != cudaSuccess) return -(int)EACG_ECUDA;
  eacg_kernel_stat acc[P_NSLOTS];
  std::memset(acc, 0, sizeof(acc));
  for (int i = 0; i < P_NSLOTS; ++i) std::snprintf(acc[i].name, sizeof(acc[i].name), "%s", PROF_NAMES[i]);
  for (const auto& r : s->prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return -(int)EACG_ECUDA;
    acc[r.slot].launches += 1;
    acc[r.slot].ms += ms;
    acc[r.slot].bytes += r.bytes;
    acc[r.slot].flops += r.flops;
    acc[r.slot].units += r.units;
  }
  for (auto& g : s->hg) hg_resolve(s, g);
  for (const auto& r : s->prof_ms) {
    acc[r.slot].launches += 1;
    acc[r.slot].ms += r.ms;
    acc[r.slot].bytes += r.bytes;
    acc[r.slot].flops += r.flops;
    acc[r.slot].units += r.units;
  }
  s->prof.clear();
  s->prof_ms.clear();
  s->evused = 0;
  int n = 0;
  for (int i = 0; i < P_NSLOTS && n < max; ++i)
    if (acc[i].launches > 0) out[n++] = acc[i];
  return n;
}

extern "C" long long eacg_launch_count(void) { return g_launches.load(); }

extern "C" eacg_status eacg_stream_create(void** stream) {
  if (!stream) return EACG_EINVAL;
  *stream = nullptr;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return EACG_ECUDA;
  }
  *stream = st;
  return EACG_OK;
}

extern "C" eacg_status eacg_stream_destroy(void* stream) {
  if (!stream) return EACG_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const cudaError_t e1 = cudaStreamSynchronize(st);
  const cudaError_t e2 = cudaStreamDestroy(st);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return EACG_ECUDA;
  }
  return EACG_OK;
}
