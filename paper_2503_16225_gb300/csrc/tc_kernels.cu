// The two projector contractions of the nonlocal term (Sec. 5.1) for complex64 blocks on the
// fifth-generation tensor cores (tcgen05.mma kind::tf32, accumulators in tensor memory), used
// in the FP32 phase of the mixed precision: the block overlaps C_k = A_k^* B_k
// (k_overlap_tf32x3, P = B^* Psi) and the back-projection C_k += A_k Q_k
// (k_backproject_tf32x3, H Psi += B (D P), below).
//
// Complex to real: with the complex rows of a column interleaved (re, im) along the
// reduction index (2 L reals),
//   Re C_ij = sum a'_i b'_j over the interleaved index, a' = (ar, ai), b' = (br, bi);
//   Im C_ij = sum a''_i b'_j,                          a'' = (-ai, ar).
// Both are real GEMMs D = A B^T with K-major operands (the blocks' own storage order).
// Accuracy: each FP32 operand x is split as x = hi + lo with hi = x truncated to TF32, and a
// product is formed from three TF32 products hi*hi + hi*lo + lo*hi (relative error about 2^-21,
// FP32 level).  The tensor-memory accumulator does not round to nearest, so its error grows with
// the length of an accumulation run: every TC_FLUSH stages (48 MMAs per accumulator) the run
// accumulators are added with round-to-nearest FP32 adds into sum accumulators kept in the other
// half of the tensor memory (tcgen05.ld, add in registers, tcgen05.st) and the next MMA starts a
// new run.  A chunk of 1024 rows gives one partial; the partials are summed in FP64 in a fixed
// order (as the SIMT block-overlap kernel does).
//
// CTA = one 128-row tile of C (rows of A) x one tile of up to 128 columns (rows of B) x one
// chunk of rows of the blocks, 256 threads.  Each stage of 16 complex rows: every thread holds
// 8 + 8 elements of A and B in registers (loaded while the previous stage's MMAs run), splits
// and interleaves them into shared memory in the canonical no-swizzle K-major layout (8-row x
// 16-byte core matrices); thread 0 issues 24 MMAs (M = 128, N = tile, K = 8 per MMA) into two
// accumulators (Re, Im) and commits them to the stage's mbarrier.  Two shared-memory stages
// alternate.  Every wait is bounded; a CTA that gives up writes NaN into its partials (the
// caller's energy or residual then reports it) and still releases its tensor memory.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace eacg {

namespace {

constexpr int TC_M = 128;                 // rows of C per CTA (MMA M)
constexpr int TC_N = 128;                 // columns of C per CTA (MMA N at most)
constexpr int TC_ROWS = 16;               // complex rows of the blocks per stage
constexpr int TC_KT = 2 * TC_ROWS;        // reals per stage
constexpr int TC_SBO = (TC_KT / 4) * 128; // bytes between 8-row groups of a tile
constexpr int TC_TILE_A = TC_M * TC_KT * 4;   // bytes of one A tile (16 KB)
constexpr int TC_TILE_B = TC_N * TC_KT * 4;   // bytes of one B tile (16 KB)
constexpr int TC_STAGE = 4 * TC_TILE_A + 2 * TC_TILE_B;  // A' hi/lo, A'' hi/lo, B' hi/lo
constexpr int TC_SMEM = 2 * TC_STAGE;
constexpr int TC_THREADS = 256;
constexpr int TC_CHUNK = 1024;            // complex rows per partial (the SIMT kernel's chunk)
constexpr int TC_FLUSH = 4;              // stages per tensor-memory accumulation run
constexpr long long TC_SPIN = 4000000;    // try_wait polls before a wait gives up
constexpr long long TC_SPIN_DRAIN = 8 * TC_SPIN;  // polls of the final wait before tensor memory is released

// CTAs whose bounded waits gave up since the library was loaded (per device, never reset)
__device__ unsigned int g_tc_gaveup = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K-direction) and stride (M/N-direction)
// byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(((uint32_t)TC_SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// instruction descriptor: D F32, A and B TF32, both K-major, N >> 3, M >> 4
__device__ __forceinline__ uint32_t tc_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}
// bounded wait for the completion of the mbarrier phase with the given parity
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, long long spin = TC_SPIN) {
  for (long long it = 0; it < spin; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (done) return true;
  }
  return false;
}
// 16 consecutive 32-bit columns of the calling thread's tensor-memory lane (warp-collective)
__device__ __forceinline__ void tmem_ld16(uint32_t ta, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
}
__device__ __forceinline__ void tmem_st16(uint32_t ta, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          ta),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]));
}
// TF32 split: hi keeps the sign, exponent and the 10 leading mantissa bits; lo = x - hi
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// byte offset of the float2 holding reals (2c, 2c + 1) of row r in a K-major stage tile
__device__ __forceinline__ int tc_off(int r, int c) {
  return (r >> 3) * TC_SBO + (c >> 1) * 128 + (r & 7) * 16 + (c & 1) * 8;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_overlap_tf32x3(int L, int m, int n, const float2* __restrict__ A, size_t sA, int lda,
                     const float2* __restrict__ B, size_t sB, int ldb, double2* __restrict__ part,
                     const int* __restrict__ kactive) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const int k = blockIdx.z;
  if (kactive && !kactive[k]) return;
  const int tiles_m = (m + TC_M - 1) / TC_M;
  const int i0 = (blockIdx.x % tiles_m) * TC_M, j0 = (blockIdx.x / tiles_m) * TC_N;
  const int nt = min(TC_N, n - j0);  // columns of this tile (a multiple of 16)
  const int ch = blockIdx.y, nch = gridDim.y;
  const int l_beg = ch * TC_CHUNK, l_end = min(L, l_beg + TC_CHUNK);
  const int tid = threadIdx.x, warp = tid >> 5;
  const float2* Ak = A + k * sA;
  const float2* Bk = B + k * sB;
  const uint32_t mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  // columns [0, 128): Re C of the current run, [128, 256): Im C; [256, 512): the sums of the runs
  const uint32_t tmem = tslot;
  const uint32_t idesc = tc_idesc(nt);
  const int nstage = (l_end - l_beg + TC_ROWS - 1) / TC_ROWS;
  const int row = 32 * (warp & 3) + (tid & 31);  // accumulator lane of this thread
  const bool im = warp >= 4;                     // warps 0-3 hold Re C, warps 4-7 Im C
  const uint32_t tcol = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(im ? TC_N : 0);
  const uint32_t tsum = tcol + 2u * TC_N;
  // Stage element map: thread t loads complex row l0 + cq of rows rq + 16 q (q < 8) of the A
  // tile and of the B tile, cq = t % 4 + 4 ((t / 32) % 4), rq = (t / 4) % 8 + 8 (t / 128): a
  // warp reads 8 rows x 32 bytes per q and writes two whole core matrices per store.
  const int cq = (tid & 3) + 4 * ((tid >> 5) & 3), rq = ((tid >> 2) & 7) + 8 * (tid >> 7);
  float2 ra[TC_M / 16], rb[TC_N / 16];
  // the next stage's elements into registers (issued before the current MMAs are waited on)
  auto load_stage = [&](int s) {
    const int l = l_beg + s * TC_ROWS + cq;
    const bool lin = l < l_end;
#pragma unroll
    for (int q = 0; q < TC_M / 16; ++q) {
      const int i = i0 + rq + 16 * q;
      ra[q] = (lin && i < m) ? Ak[(size_t)i * lda + l] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < TC_N / 16; ++q) {
      const int r = rq + 16 * q;
      rb[q] = (lin && r < nt) ? Bk[(size_t)(j0 + r) * ldb + l] : make_float2(0.f, 0.f);
    }
  };
  bool failed = false;
  int issued = 0;  // stages whose MMAs were issued (uniform over the CTA)
  if (nstage > 0) load_stage(0);
  for (int s = 0; s < nstage; ++s) {
    const int buf = s & 1;
    unsigned char* st = smem + buf * TC_STAGE;
    if (s >= 2) {  // the MMAs that read this buffer two stages ago
      const bool ok = tc_wait(buf ? mb1 : mb0, (uint32_t)(((s >> 1) - 1) & 1));
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    // split and interleave: A' hi/lo = (ar, ai), A'' hi/lo = (-ai, ar), B' hi/lo = (br, bi)
#pragma unroll
    for (int q = 0; q < TC_M / 16; ++q) {
      const float2 a = ra[q];
      const float hr = tf32_hi(a.x), hi_ = tf32_hi(a.y);
      const float lr = a.x - hr, li = a.y - hi_;
      const int o = tc_off(rq + 16 * q, cq);
      *reinterpret_cast<float2*>(st + o) = make_float2(hr, hi_);
      *reinterpret_cast<float2*>(st + TC_TILE_A + o) = make_float2(lr, li);
      *reinterpret_cast<float2*>(st + 2 * TC_TILE_A + o) = make_float2(-hi_, hr);
      *reinterpret_cast<float2*>(st + 3 * TC_TILE_A + o) = make_float2(-li, lr);
    }
    unsigned char* sb = st + 4 * TC_TILE_A;
#pragma unroll
    for (int q = 0; q < TC_N / 16; ++q) {
      if (rq + 16 * q < nt) {
        const float2 b = rb[q];
        const float hr = tf32_hi(b.x), hi_ = tf32_hi(b.y);
        const int o = tc_off(rq + 16 * q, cq);
        *reinterpret_cast<float2*>(sb + o) = make_float2(hr, hi_);
        *reinterpret_cast<float2*>(sb + TC_TILE_B + o) = make_float2(b.x - hr, b.y - hi_);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t base = smem_u32(st);
      const uint32_t aH = base, aL = base + TC_TILE_A, xH = base + 2 * TC_TILE_A, xL = base + 3 * TC_TILE_A;
      const uint32_t bH = base + 4 * TC_TILE_A, bL = bH + TC_TILE_B;
      for (int ks = 0; ks < TC_KT / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 256u;  // two core matrices along K per MMA
        const uint32_t first = (s % TC_FLUSH == 0 && ks == 0) ? 0u : 1u;
        tc_mma(tmem, tc_desc(aH + ko), tc_desc(bH + ko), idesc, first);
        tc_mma(tmem, tc_desc(aH + ko), tc_desc(bL + ko), idesc, 1u);
        tc_mma(tmem, tc_desc(aL + ko), tc_desc(bH + ko), idesc, 1u);
        tc_mma(tmem + TC_N, tc_desc(xH + ko), tc_desc(bH + ko), idesc, first);
        tc_mma(tmem + TC_N, tc_desc(xH + ko), tc_desc(bL + ko), idesc, 1u);
        tc_mma(tmem + TC_N, tc_desc(xL + ko), tc_desc(bH + ko), idesc, 1u);
      }
      tc_commit(buf ? mb1 : mb0);
    }
    issued = s + 1;
    if (s + 1 < nstage) load_stage(s + 1);
    if ((s + 1) % TC_FLUSH == 0 || s + 1 == nstage) {
      // end of a run: wait for this stage's MMAs (and so all earlier ones), add the
      // accumulators into registers, then let the next run overwrite them
      const bool ok = tc_wait(buf ? mb1 : mb0, (uint32_t)((s >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const bool first_run = s < TC_FLUSH;
      for (int c0 = 0; c0 < nt; c0 += 16) {
        uint32_t v[16], w[16];
        tmem_ld16(tcol + (uint32_t)c0, v);
        if (!first_run) {
          tmem_ld16(tsum + (uint32_t)c0, w);
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) + __uint_as_float(w[q]));
        }
        tmem_st16(tsum + (uint32_t)c0, v);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
  }
  // completion of the last issued stage of each buffer (also after a wait that gave up, so that
  // no MMA still writes the tensor memory when it is released; this wait polls 8 times longer)
  {
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
      if (issued > b) {
        const int sb = ((issued - 1 - b) >> 1) * 2 + b;  // last issued stage on buffer b
        ok = tc_wait(b ? mb1 : mb0, (uint32_t)((sb >> 1) & 1), TC_SPIN_DRAIN) && ok;
      }
    }
    failed = __syncthreads_or(!ok) || failed;
    if (failed && tid == 0) atomicAdd(&g_tc_gaveup, 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // epilogue: thread (warp w, lane t) owns row 32 (w % 4) + t of Re (w < 4) or Im (w >= 4)
  {
    const int i = i0 + row;
    double* out = reinterpret_cast<double*>(part);
    for (int c0 = 0; c0 < nt; c0 += 16) {
      uint32_t v[16];
      if (!failed) {
        tmem_ld16(tsum + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0x7FC00000u;  // NaN marks a wait that gave up
      }
      if (i < m) {
#pragma unroll
        for (int q = 0; q < 16; ++q)
          out[2 * ((((size_t)k * nch + ch) * n + (j0 + c0 + q)) * m + i) + (im ? 1 : 0)] =
              (double)__uint_as_float(v[q]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// Back-projection C_k += A_k Q_k (the nonlocal term's H Psi += B (D P)): A_k is L x m complex64
// stored column by column ([m][lda], the projectors), Q_k is m x n complex double ([n][ldq]),
// C_k is L x n complex double ([n][ldc]).  With the rows of C interleaved (re, im) and the
// reduction index interleaved the same way, C' = A_exp Q' is one real GEMM of M = 2L, K = 2m:
//   A_exp[2l][2i] = ar, A_exp[2l][2i+1] = -ai, A_exp[2l+1][2i] = ai, A_exp[2l+1][2i+1] = ar,
//   Q'[j][2i] = qr, Q'[j][2i+1] = qi (B operand, K-major: a column of Q is a row).
// Same 3 x TF32 split, stages of 16 complex reduction indices, accumulation runs of 48 MMAs
// summed in the other half of the tensor memory, bounded waits, as k_overlap_tf32x3.  CTA =
// 128 interleaved rows (64 rows of C) x all n <= 256 columns.  Warps 0-3 move the
// accumulators (row 32 w + lane); all 8 warps stage the operands.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_backproject_tf32x3(int L, int m, int n, const float2* __restrict__ A, size_t sA, int lda,
                         const double2* __restrict__ Q, size_t sQ, int ldq, double2* __restrict__ C, size_t sC,
                         int ldc, const int* __restrict__ kactive) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const int k = blockIdx.y;
  if (kactive && !kactive[k]) return;
  const int l0 = blockIdx.x * (TC_M / 2);  // first row of C of this tile
  const int tid = threadIdx.x, warp = tid >> 5;
  const float2* Ak = A + k * sA;
  const double2* Qk = Q + k * sQ;
  const uint32_t mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  // columns [0, n): the current run's accumulator; [256, 256 + n): the sum of the runs
  const uint32_t tmem = tslot;
  const uint32_t idesc = tc_idesc(n);
  const int nstage = (m + TC_ROWS - 1) / TC_ROWS;
  const bool mover = warp < 4;  // warps that read and write the accumulators
  const uint32_t tcol = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t tsum = tcol + 256u;
  // staging maps: A elements (row l0 + la, reduction index ia + 4 q), coalesced along rows;
  // Q elements (column rq + 16 q, reduction index cq) as in k_overlap_tf32x3
  const int la = tid & 63, ia = tid >> 6;
  const int cq = (tid & 3) + 4 * ((tid >> 5) & 3), rq = ((tid >> 2) & 7) + 8 * (tid >> 7);
  float2 ra[4], rb[16];
  auto load_stage = [&](int s) {
    const int i0 = s * TC_ROWS;
    const int l = l0 + la;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ia + 4 * q;
      ra[q] = (l < L && i < m) ? Ak[(size_t)i * lda + l] : make_float2(0.f, 0.f);
    }
    const int i = i0 + cq;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = rq + 16 * q;
      if (j < n) {
        const double2 v = (i < m) ? Qk[(size_t)j * ldq + i] : make_double2(0.0, 0.0);
        rb[q] = make_float2((float)v.x, (float)v.y);
      }
    }
  };
  bool failed = false;
  int issued = 0;
  if (nstage > 0) load_stage(0);
  for (int s = 0; s < nstage; ++s) {
    const int buf = s & 1;
    unsigned char* st = smem + buf * TC_STAGE;
    if (s >= 2) {
      const bool ok = tc_wait(buf ? mb1 : mb0, (uint32_t)(((s >> 1) - 1) & 1));
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
    }
    // A_exp hi/lo: rows 2 la and 2 la + 1, reals 2 i and 2 i + 1
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float2 a = ra[q];
      const float hr = tf32_hi(a.x), hi_ = tf32_hi(a.y);
      const float lr = a.x - hr, li = a.y - hi_;
      const int c = ia + 4 * q;
      const int o0 = tc_off(2 * la, c), o1 = tc_off(2 * la + 1, c);
      *reinterpret_cast<float2*>(st + o0) = make_float2(hr, -hi_);
      *reinterpret_cast<float2*>(st + o1) = make_float2(hi_, hr);
      *reinterpret_cast<float2*>(st + TC_TILE_A + o0) = make_float2(lr, -li);
      *reinterpret_cast<float2*>(st + TC_TILE_A + o1) = make_float2(li, lr);
    }
    // Q' hi/lo: rows = columns of Q (up to 256 rows: two 16 KB halves per part)
    unsigned char* sb = st + 2 * TC_TILE_A;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int j = rq + 16 * q;
      if (j < n) {
        const float2 b = rb[q];
        const float hr = tf32_hi(b.x), hi_ = tf32_hi(b.y);
        const int o = tc_off(j, cq);
        *reinterpret_cast<float2*>(sb + o) = make_float2(hr, hi_);
        *reinterpret_cast<float2*>(sb + 2 * TC_TILE_B + o) = make_float2(b.x - hr, b.y - hi_);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t base = smem_u32(st);
      const uint32_t aH = base, aL = base + TC_TILE_A;
      const uint32_t bH = base + 2 * TC_TILE_A, bL = bH + 2 * TC_TILE_B;
      for (int ks = 0; ks < TC_KT / 8; ++ks) {
        const uint32_t ko = (uint32_t)ks * 256u;
        const uint32_t first = (s % TC_FLUSH == 0 && ks == 0) ? 0u : 1u;
        tc_mma(tmem, tc_desc(aH + ko), tc_desc(bH + ko), idesc, first);
        tc_mma(tmem, tc_desc(aH + ko), tc_desc(bL + ko), idesc, 1u);
        tc_mma(tmem, tc_desc(aL + ko), tc_desc(bH + ko), idesc, 1u);
      }
      tc_commit(buf ? mb1 : mb0);
    }
    issued = s + 1;
    if (s + 1 < nstage) load_stage(s + 1);
    if ((s + 1) % TC_FLUSH == 0 || s + 1 == nstage) {
      const bool ok = tc_wait(buf ? mb1 : mb0, (uint32_t)((s >> 1) & 1));
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (mover) {
        const bool first_run = s < TC_FLUSH;
        for (int c0 = 0; c0 < n; c0 += 16) {
          uint32_t v[16], w[16];
          tmem_ld16(tcol + (uint32_t)c0, v);
          if (!first_run) {
            tmem_ld16(tsum + (uint32_t)c0, w);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = __float_as_uint(__uint_as_float(v[q]) + __uint_as_float(w[q]));
          }
          tmem_st16(tsum + (uint32_t)c0, v);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;");
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
  }
  {
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
      if (issued > b) {
        const int sb = ((issued - 1 - b) >> 1) * 2 + b;
        ok = tc_wait(b ? mb1 : mb0, (uint32_t)((sb >> 1) & 1), TC_SPIN_DRAIN) && ok;
      }
    }
    failed = __syncthreads_or(!ok) || failed;
    if (failed && tid == 0) atomicAdd(&g_tc_gaveup, 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // epilogue: interleaved row 32 w + lane -> row l of C, part re/im; C += the sums (FP64)
  if (mover && nstage > 0) {
    const int r = 32 * warp + (tid & 31);
    const int l = l0 + (r >> 1), part = r & 1;
    double* out = reinterpret_cast<double*>(C + k * sC);
    for (int c0 = 0; c0 < n; c0 += 16) {
      uint32_t v[16];
      if (!failed) {
        tmem_ld16(tsum + (uint32_t)c0, v);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0x7FC00000u;  // NaN marks a wait that gave up
      }
      if (l < L) {
#pragma unroll
        for (int q = 0; q < 16; ++q) out[2 * ((size_t)(c0 + q) * ldc + l) + part] += (double)__uint_as_float(v[q]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

}  // namespace

bool dense_overlap_tc_eligible(int m, int n) { return m >= TC_M && n >= 16 && n % 16 == 0; }

size_t dense_overlap_tc_work(int K, int L, int m, int n) {
  return (size_t)K * ((L + TC_CHUNK - 1) / TC_CHUNK) * m * n;
}

void dense_overlap_tf32x3(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const float2* B,
                          size_t sB, int ldb, double2* C, size_t sC, int ldc, double2 alpha, double2 beta,
                          double2* work, const int* kactive, cudaStream_t st) {
  if (K <= 0 || m <= 0 || n <= 0) return;
  ensure_smem((const void*)k_overlap_tf32x3, TC_SMEM);  // per device
  const int nch = (L + TC_CHUNK - 1) / TC_CHUNK;
  if (nch > 0) {
    const int tiles = ((m + TC_M - 1) / TC_M) * ((n + TC_N - 1) / TC_N);
    dim3 g(tiles, nch, K);
    k_overlap_tf32x3<<<g, TC_THREADS, TC_SMEM, st>>>(L, m, n, A, sA, lda, B, sB, ldb, work, kactive);
    count_launch();
  }
  dense_cn_reduce(K, m, n, nch, work, C, sC, ldc, alpha, beta, kactive, st);
}

unsigned int dense_tc_gaveup_count(cudaStream_t st) {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbolAsync(&v, g_tc_gaveup, sizeof(v), 0, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return ~0u;
  return v;
}

bool dense_backproject_tc_eligible(int m, int n) { return m >= 1 && n >= 16 && n <= 256 && n % 16 == 0; }

void dense_backproject_tf32x3(int K, int L, int m, int n, const float2* A, size_t sA, int lda, const double2* Q,
                              size_t sQ, int ldq, double2* C, size_t sC, int ldc, const int* kactive,
                              cudaStream_t st) {
  if (K <= 0 || L <= 0 || m <= 0 || n <= 0) return;
  ensure_smem((const void*)k_backproject_tf32x3, TC_SMEM);  // per device
  dim3 g((L + TC_M / 2 - 1) / (TC_M / 2), K);
  k_backproject_tf32x3<<<g, TC_THREADS, TC_SMEM, st>>>(L, m, n, A, sA, lda, Q, sQ, ldq, C, sC, ldc, kactive);
  count_launch();
}

}  // namespace eacg
