// FP64-grade products on the BF16 tensor cores by error-free slicing (Ozaki scheme;
// Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012), sm_103a tcgen05.
//
// Each FP64 operand row (of A) / column (of B) is scaled by a power of two so
// that its largest entry is below 1 in magnitude, truncated to 49 bits, and cut
// into seven signed 7-bit digits d_1..d_7 (x ~ 2^E sum_i d_i 2^-7i).  Digit i
// is stored in BF16 as d_i 2^-7(i-1) (exact: 7 significant bits).  The product
// sum_k a_i b_j of digit slices has weight 2^-7(i+j-2); for a fixed t = i + j
// every partial sum is an integer multiple of 2^-7(t-2) below 2^24 of that
// unit (K <= 256 per accumulation group, at most four pairs, digits below 2^7 in
// magnitude: 4 * 256 * 127^2 < 2^24), so the FP32 tensor-core accumulators
// for t = 2, 3, 4, 5 are exact.  The pairs with t = 6..8 share a fifth
// accumulator (their FP32 rounding is below 2^-52 of the result); pairs with
// t > 8 fall below the 49-bit truncation and are dropped.  The epilogue adds
// the five accumulators with error-free FP32 sums into a (hi, lo) pair and
// forms the FP64 result 2^(E_A + E_B - 14) (hi + lo).  The error is within a
// few units of 2^-48 of sum_k |a_k||b_k|, comparable to FP64 GEMM rounding.
//
// Modes:
//   CELL  W(cell nodes) += H^cc_e Y_e for the cells of one parity colour
//         (Sec. V, last paragraph; cells of a colour share no node);
//   ROWS  C = A B for a tall A (rows x K) and a small B (K x N); K is taken in
//         groups of 256 (exact FP32 sums), each group's FP64 value added to C;
//   GRAM  C = A^T B for tall A, B (K x Na, K x N, K large): items are (tile
//         pair, K segment); each segment is formed in 256-row groups (exact
//         FP32 sums for t <= 5) drained into FP64 partial tiles, which a
//         fixed-order reduction adds up.
// Pre-sliced operands arrive in the stages by bulk asynchronous copies: the
// cell matrices' digit images (k_oz_preslice, once per potential) in CELL, and
// both operands' images (k_oz_img_rows / k_oz_img_cols, once per product) in
// ROWS and GRAM; only CELL's vector block is sliced inside the kernel.
//
// Warp roles (512 threads): warp 0 issues the MMAs (one elected lane); while
// an operand is sliced here (CELL's vector block), warps 1-7 slice into the
// shared-memory stage ring (4 stages, two groups taking alternate chunks) and
// warps 8-15 combine the accumulators and write the result; when both operands
// are pre-sliced images (ROWS, GRAM) one thread issues the bulk copies and
// warps 4-15 share the epilogue.  All waits are bounded (about one second); on
// timeout the CTA records an error and leaves.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "efe_kernels.h"

namespace efe {

namespace {

constexpr int OZ_S = 7;            // digits per operand
constexpr int OZ_M = 128;          // MMA rows
constexpr int OZ_KC = 16;          // K per chunk (one BF16 MMA)
constexpr int OZ_TW = 96;          // column tile
constexpr int OZ_NACC = 5;         // accumulators: t = 2, 3, 4, 5 exact; t = 6..8 shared
constexpr int OZ_ROWS_KG = 16;     // ROWS: 16-wide K chunks per exact accumulation group (K <= 256)
constexpr int OZ_STAGES = 4;
constexpr int OZ_GROUPS = 2;        // slicer groups: group g fills the chunks ch = g (mod 2)
constexpr int OZ_CONV_W0 = 1, OZ_CONV_WN = 7, OZ_EPI_W0 = 8;   // slicing: warps 1-7 slice, 8-15 epilogue
constexpr int OZ_THREADS = 16 * 32;                // 16 warps: 128 registers a thread
constexpr int OZ_CONV_T = OZ_CONV_WN * 32;
constexpr int OZ_GT0 = 4 * 32;                     // group 0: warps 1-4; group 1: warps 5-7
__host__ __device__ constexpr int oz_group_threads(int grp) { return grp == 0 ? OZ_GT0 : OZ_CONV_T - OZ_GT0; }
static_assert(OZ_STAGES % OZ_GROUPS == 0, "a stage is always filled by the same group");
constexpr uint32_t OZ_TMEM_COLS = 512;
constexpr long long OZ_WAIT = 2000000000LL;

struct OzL {
  static constexpr uint32_t ASL = OZ_M * OZ_KC * 2;        // one A slice, 4 KB
  static constexpr uint32_t BSL = OZ_TW * OZ_KC * 2;       // one B slice, 3 KB
  static constexpr uint32_t STAGE = OZ_S * (ASL + BSL);    // 49 KB
  static constexpr uint32_t BARS = OZ_STAGES * STAGE;
  static constexpr uint32_t STG = BARS + 256;                // epilogue staging: up to 12 warps x 32 rows x 9 doubles
  static constexpr size_t TOTAL = (size_t)STG + 12 * 32 * 9 * 8;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, no swizzle, BF16: core matrix 8 rows x 16 B; LBO = 128 B (next 8 K), SBO = 256 B (next 8 rows)
__device__ __forceinline__ uint32_t bo(int row, int k) {
  return (uint32_t)(row >> 3) * 256u + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
         ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZ_M >> 4) << 24);
}
__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity) {
  uint32_t done = 0;
  const long long t0 = clock64();
  do {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    if (done) return true;
  } while (clock64() - t0 < OZ_WAIT);
  return false;
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}

// scale exponent of one value: |x| < 2^E (zero -> very small)
__device__ __forceinline__ int exp_of(double x) {
  const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return ex == 0 ? -2000 : ex - 1022;
}

// digits of eight values with scale exponent E, packed slice by slice (two BF16
// per word): pk[i] holds digit i of x[0..7] in K order
__device__ __forceinline__ void oz_pack8(const double (&x)[8], int E, uint32_t (&pk)[OZ_S][4]) {
#pragma unroll
  for (int i = 0; i < OZ_S; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) pk[i][q] = 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long bits = __double_as_longlong(x[q]);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const uint32_t sgn = (uint32_t)((bits >> 48) & 0x8000);
    unsigned long long qq = 0;
    const int rs = 1026 + E - ex;
    if (ex != 0 && rs >= 0 && rs < 64) qq = ((unsigned long long)(bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> rs;
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      const uint32_t d = (uint32_t)(qq >> (42 - 7 * i)) & 127u;
      uint32_t h16 = 0;
      if (d) {
        const int p = 31 - __clz(d);
        h16 = sgn | ((uint32_t)(p + 127 - 7 * i) << 7) | ((d << (7 - p)) & 0x7Fu);
      }
      pk[i][q >> 1] |= h16 << (16 * (q & 1));
    }
  }
}

// x * 2^k in FP64, built from the bit pattern of x (exact; no FP64 arithmetic).
// Every accumulator value and error term here is zero or at least 2^-42 in
// magnitude (the smallest digit-product unit), so x is never subnormal;
// results outside the normal FP64 range take ldexp.
__device__ __forceinline__ double f32_scaled(float x, int k) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xFFu);
  if (e == 0) return 0.0;
  const int E = e - 127 + 1023 + k;
  if (E < 1 || E > 2046) return ldexp((double)x, k);
  return __longlong_as_double((long long)(((unsigned long long)(b >> 31) << 63) | ((unsigned long long)E << 52) |
                                          ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

struct OzArgs {
  int mode;                 // 0: CELL, 1: ROWS, 2: GRAM
  // CELL
  const double* H;          // n_cell x 125 x 125
  const int* hexp;          // n_cell x 128 row exponents
  const unsigned char* Aimg;  // optional pre-sliced digit images of H^cc_e (oz_cell_image_bytes per cell)
  const int32_t* cells;
  int64_t ncells;
  MeshDev m;
  // ROWS
  const double* A;          // rows x K
  int64_t lda, arows;
  const int* aexp;          // per row of A
  const double* B;          // K x N
  int64_t ldb;
  // common
  int K;                    // reduction length (CELL: 125; ROWS: any, in groups of 256)
  const double* Y;          // CELL: vector block (nodes x N)
  int64_t ldy;
  const int* fexp;          // per column of Y (CELL) or of B (ROWS)
  double* out;              // CELL: W (accumulated); ROWS: C (stored)
  int64_t ldo;
  int N, ntiles;
  int* err;
  // GRAM: C = A^T B with A (Kbig x Na, lda), B (Kbig x N, ldb); aexp / fexp per
  // column of A / B; work items = (tile pair, K segment of seg_len rows);
  // FP64 partial tiles to part[segment][Na][N]
  int64_t Kbig, seg_len;
  int Na, nseg, npairs;
  const int2* pairs;        // (M tile, N tile) of every item pair
  double* part;
  // pre-sliced operand images (k_oz_img_rows / k_oz_img_cols); NULL: sliced here.
  // ROWS: Aimg = row image of A, Bimg = column image of B; GRAM: both column
  // images.  img_nch: 16-wide K chunks per 128-wide tile of a column image.
  const unsigned char* Bimg;
  int64_t img_nch;
  int stall;                // tests only: the MMA warp first waits on a barrier nothing completes
};

// work item of a CTA: cell / row block / tile pair and its K range
struct OzItem {
  int64_t ia, e, m0, kb;
  int c0, ncol, nmma, seg;
};

__device__ __forceinline__ OzItem oz_item(const OzArgs& g, int64_t item) {
  OzItem it;
  if (g.mode == 2) {
    // segment-major: the CTAs running at one time share a segment's rows, so the
    // operand images of that segment are read from L2 by every tile pair
    const int64_t pr = item % g.npairs;
    it.seg = (int)(item / g.npairs);
    const int2 tp = g.pairs[pr];
    it.ia = pr;
    it.e = 0;
    it.m0 = (int64_t)tp.x * OZ_M;
    it.c0 = tp.y * OZ_TW;
    it.kb = (int64_t)it.seg * g.seg_len;
  } else {
    it.ia = item / g.ntiles;
    it.c0 = (int)(item % g.ntiles) * OZ_TW;
    it.e = (g.mode == 0) ? g.cells[it.ia] : 0;
    it.m0 = it.ia * OZ_M;
    it.kb = 0;
    it.seg = 0;
  }
  it.ncol = min(OZ_TW, g.N - it.c0);
  it.nmma = ((it.ncol + 15) / 16) * 16;
  return it;
}

__device__ __forceinline__ int64_t oz_cell_node(const MeshDev& m, int64_t e, int k) {
  const int i = (int)(e % m.nc[0]), j = (int)((e / m.nc[0]) % m.nc[1]), kk = (int)(e / ((int64_t)m.nc[0] * m.nc[1]));
  const int a = k % NP1, b = (k / NP1) % NP1, c = k / (NP1 * NP1);
  return (int64_t)(P * i + a) + (int64_t)m.nn[0] * ((int64_t)(P * j + b) + (int64_t)m.nn[1] * (int64_t)(P * kk + c));
}

// IMG: both operands arrive as pre-sliced images (ROWS / GRAM with images), so
// no thread slices; a separate instantiation keeps the slicing code and its
// registers out of that kernel (and the register epilogue out of the other)
template <bool IMG>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz(OzArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ int s_skip;
  if (tid == 0) s_skip = *(volatile int*)g.err;
  __syncthreads();
  if (s_skip) return;
  if (IMG != (g.mode != 0 && g.Aimg != nullptr && g.Bimg != nullptr)) {
    // the host picks the instantiation from the same test; a mismatch is an error
    if (tid == 0) atomicExch(g.err, 1);
    return;
  }
  uint64_t* conv = reinterpret_cast<uint64_t*>(sm + OzL::BARS);  // [stages] slices written
  uint64_t* empty = conv + OZ_STAGES;                           // [stages] MMAs done with the stage
  uint64_t* accf = conv + 2 * OZ_STAGES;
  uint64_t* acce = accf + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accf + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(accf + 3);
  uint64_t* afull = accf + 4;                                   // [stages] bulk-copied operand chunks landed
  uint64_t* never = afull + OZ_STAGES;                          // no thread ever arrives here (test stall)
  const bool apre = IMG || g.Aimg != nullptr;
  const bool bpre = IMG || (g.mode != 0 && g.Bimg != nullptr);
  // both operands pre-sliced: nothing to slice, so one thread issues the copies
  // and warps 4-15 share the epilogue (three warps per TMEM lane quarter)
  constexpr bool img_only = IMG;
  const int n_epi = img_only ? 12 : 8;
  const int epi_w0 = img_only ? 4 : OZ_EPI_W0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < OZ_STAGES; ++s) {
      bar_init(conv + s, img_only ? 1 : oz_group_threads(s % OZ_GROUPS));
      bar_init(empty + s, 1);
      bar_init(afull + s, 1);
    }
    bar_init(accf, 1);
    bar_init(acce, n_epi * 32);
    bar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int64_t nA = (g.mode == 0) ? g.ncells : (g.arows + OZ_M - 1) / OZ_M;
  const int64_t nitems = (g.mode == 2) ? (int64_t)g.npairs * g.nseg : nA * g.ntiles;
  const int64_t my = nitems > blockIdx.x ? (nitems - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  // chunks of 16 K per item; the accumulators are drained every gsz chunks
  // (GRAM: every 256 rows, ROWS: every 256 K -- where the FP32 sums of t <= 5
  // are still exact -- and CELL once, K = 125); later groups add to the result
  const int nch = (g.mode == 2) ? (int)(g.seg_len / OZ_KC) : (g.K + OZ_KC - 1) / OZ_KC;
  const int gsz = (g.mode == 2) ? 16 : (g.mode == 1 ? min(nch, OZ_ROWS_KG) : nch);
  const int ngrp = (nch + gsz - 1) / gsz;
  // the last chunk whose MMAs this thread committed / whose bulk copies it issued
  // (drained before the TMEM and shared memory are released after an abort)
  int64_t last_mma = -1, last_copy = -1;

  if (warp == 0) {
    // ---------------------------------------------------------------- MMA issuer
    if (g.stall && my > 0 && !bar_wait(never, 0u)) {
      // test stall: a wait that nothing completes runs out like a real one
      if (lane == 0) { *abort_flag = 1; atomicExch(g.err, 1); }
    }
    for (int64_t t = 0; t < my && !*abort_flag; ++t) {
      const int64_t item = blockIdx.x + t * gridDim.x;
      const OzItem it = oz_item(g, item);
      const int nmma = it.nmma;
      bool ok = true;
      for (int kc = 0; kc < nch && ok; ++kc) {
        const int64_t gc = t * ngrp + kc / gsz;   // accumulator group counter
        if (kc % gsz == 0) {
          if (gc >= 1) ok = bar_wait(acce, (uint32_t)((gc - 1) & 1));
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          if (!ok) break;
        }
        const int64_t ch = t * nch + kc;
        const int s = (int)(ch % OZ_STAGES);
        ok = bar_wait(conv + s, (uint32_t)((ch / OZ_STAGES) & 1));
        if (ok && (apre || bpre)) ok = bar_wait(afull + s, (uint32_t)((ch / OZ_STAGES) & 1));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;
        if (lane == 0) {
          const uint32_t sA = su32(sm + s * OzL::STAGE);
          const uint32_t sB = sA + OZ_S * OzL::ASL;
          const uint32_t id = idesc_bf16(nmma);
          bool first[OZ_NACC] = {true, true, true, true, true};
#pragma unroll
          for (int tt = 2; tt <= 8; ++tt) {
            const int a = tt <= 5 ? tt - 2 : 4;
#pragma unroll
            for (int i = 1; i < tt; ++i) {
              const int j = tt - i;
              if (i > OZ_S || j > OZ_S) continue;
              const uint32_t acc = (kc % gsz > 0 || !first[a]) ? 1u : 0u;
              first[a] = false;
              mma_bf16(tmem + (uint32_t)(a * OZ_TW), sdesc(sA + (uint32_t)(i - 1) * OzL::ASL),
                       sdesc(sB + (uint32_t)(j - 1) * OzL::BSL), id, acc);
            }
          }
          mma_commit(empty + s);
          if (kc % gsz == gsz - 1 || kc == nch - 1) mma_commit(accf);
        }
        last_mma = ch;
        __syncwarp();
      }
      if (!ok) {
        if (lane == 0) { *abort_flag = 1; atomicExch(g.err, 1); }
        break;
      }
    }
  } else if (img_only ? (warp == OZ_CONV_W0 && lane == 0) : (warp < OZ_CONV_W0 + OZ_CONV_WN)) {
    // ---------------------------------------------------------------- slicers
    // two groups (four and three warps) take alternate chunks, so two chunks are
    // sliced (and their loads are in flight) at a time; with both operands
    // pre-sliced a single thread takes every chunk
    const int grp = img_only ? 0 : ((tid - OZ_CONV_W0 * 32) < OZ_GT0 ? 0 : 1);
    const int ct = img_only ? 0 : (tid - OZ_CONV_W0 * 32) - grp * OZ_GT0;
    const int gsz_t = img_only ? 1 : oz_group_threads(grp);
    for (int64_t t = 0; t < my && !*abort_flag; ++t) {
      const OzItem it = oz_item(g, blockIdx.x + t * gridDim.x);
      const int64_t ia = it.ia, e = it.e;
      const int c0 = it.c0, ncol = it.ncol, nmma = it.nmma;
      bool ok = true;
      for (int kc = 0; kc < nch; ++kc) {
        const int64_t ch = t * nch + kc;
        if (!img_only && (int)(ch % OZ_GROUPS) != grp) continue;
        const int s = (int)(ch % OZ_STAGES);
        if (ch >= OZ_STAGES) {
          ok = bar_wait(empty + s, (uint32_t)((ch / OZ_STAGES - 1) & 1));
          if (!ok) break;
        }
        unsigned char* SA = sm + s * OzL::STAGE;
        unsigned char* SB = SA + OZ_S * OzL::ASL;
        if ((apre || bpre) && ct == 0) {
          // pre-sliced operand chunks: bulk copies of 256-byte row groups into the stage
          const int64_t kA = (g.mode == 2) ? it.kb / OZ_KC + kc : kc;
          const int ga = (g.mode == 2) ? (int)((min((int64_t)OZ_M, (int64_t)g.Na - it.m0) + 7) / 8) : 16;
          const int gb = nmma / 8;
          uint32_t bytes = 0;
          if (apre) bytes += (uint32_t)(OZ_S * ga * 256);
          if (bpre) bytes += (uint32_t)(OZ_S * gb * 256);
          bar_expect_tx(afull + s, bytes);
          if (apre) {
            // CELL: image of cell e; ROWS: of row tile ia; GRAM: of column tile m0 / 128
            const int64_t img = (g.mode == 0) ? e * (int64_t)nch + kA
                              : (g.mode == 1) ? ia * (int64_t)nch + kA
                                              : (it.m0 / OZ_M) * g.img_nch + kA;
            const unsigned char* src = g.Aimg + img * OZ_S * (int64_t)OzL::ASL;
            if (ga == 16) {
              bulk_g2s(SA, src, OZ_S * OzL::ASL, afull + s);
            } else {
              for (int i2 = 0; i2 < OZ_S; ++i2)
                bulk_g2s(SA + i2 * OzL::ASL, src + i2 * OzL::ASL, (uint32_t)(ga * 256), afull + s);
            }
          }
          if (bpre) {
            // columns c0 .. c0 + nmma of B: row groups of the 128-wide column tiles
            const int64_t nchB = (g.mode == 2) ? g.img_nch : nch;
            for (int j = 0; j < gb;) {
              const int G = c0 / 8 + j;
              const int tile = G >> 4, gi = G & 15;
              const int run = min(gb - j, 16 - gi);
              const unsigned char* src = g.Bimg + ((tile * nchB + kA) * OZ_S) * (int64_t)OzL::ASL + gi * 256;
              for (int i2 = 0; i2 < OZ_S; ++i2)
                bulk_g2s(SB + i2 * OzL::BSL + j * 256, src + i2 * OzL::ASL, (uint32_t)(run * 256), afull + s);
              j += run;
            }
          }
          last_copy = ch;
        }
        // one thread per (row, 8-wide K octet): eight loads in flight, then seven
        // 16-byte slice stores (one core-matrix row each); pre-sliced operands
        // (the A tasks, the B tasks) are skipped
        for (int v = ct + (apre ? OZ_M * 2 : 0); v < (bpre ? OZ_M * 2 : (OZ_M + nmma) * 2); v += gsz_t) {
          const bool isA = v < OZ_M * 2;
          const int w = isA ? v : v - OZ_M * 2;
          const int row = w >> 1, oct = w & 1;        // row of A, or column n of the product
          double x[8];
          int E = -2000;
          if (g.mode == 2) {
            const int64_t k0 = it.kb + kc * OZ_KC + oct * 8;
            if (isA) {
              const int64_t col = it.m0 + row;
              if (col < g.Na) E = g.aexp[col];
#pragma unroll
              for (int q = 0; q < 8; ++q) x[q] = (col < g.Na && k0 + q < g.Kbig) ? g.A[(k0 + q) * g.lda + col] : 0.0;
            } else {
              if (row < ncol) E = g.fexp[c0 + row];
#pragma unroll
              for (int q = 0; q < 8; ++q)
                x[q] = (row < ncol && k0 + q < g.Kbig) ? g.B[(k0 + q) * g.ldb + c0 + row] : 0.0;
            }
          } else if (isA) {
            if (g.mode == 0) {
              E = g.hexp[e * OZ_M + row];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int k = kc * OZ_KC + oct * 8 + q;
                x[q] = (row < NL && k < NL) ? g.H[e * (int64_t)(NL * NL) + row * NL + k] : 0.0;
              }
            } else {
              const int64_t ar = ia * OZ_M + row;
              if (ar < g.arows) E = g.aexp[ar];
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const int k = kc * OZ_KC + oct * 8 + q;
                x[q] = (ar < g.arows && k < g.K) ? g.A[ar * g.lda + k] : 0.0;
              }
            }
          } else {
            const int n = row;
            if (n < ncol) E = g.fexp[c0 + n];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int k = kc * OZ_KC + oct * 8 + q;
              double xv = 0.0;
              if (n < ncol) {
                if (g.mode == 0) {
                  if (k < NL) xv = g.Y[oz_cell_node(g.m, e, k) * g.ldy + c0 + n];
                } else {
                  if (k < g.K) xv = g.B[(int64_t)k * g.ldb + c0 + n];
                }
              }
              x[q] = xv;
            }
          }
          // digits of the eight values, packed slice by slice
          uint32_t pk[OZ_S][4];
#pragma unroll
          for (int i2 = 0; i2 < OZ_S; ++i2)
#pragma unroll
            for (int q = 0; q < 4; ++q) pk[i2][q] = 0u;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const long long bits = __double_as_longlong(x[q]);
            const int ex = (int)((bits >> 52) & 0x7FF);
            const uint32_t sgn = (uint32_t)((bits >> 48) & 0x8000);
            unsigned long long qq = 0;
            const int rs = 1026 + E - ex;
            if (ex != 0 && rs >= 0 && rs < 64) qq = ((unsigned long long)(bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> rs;
#pragma unroll
            for (int i2 = 0; i2 < OZ_S; ++i2) {
              const uint32_t d = (uint32_t)(qq >> (42 - 7 * i2)) & 127u;
              uint32_t h16 = 0;
              if (d) {
                const int p = 31 - __clz(d);
                h16 = sgn | ((uint32_t)(p + 127 - 7 * i2) << 7) | ((d << (7 - p)) & 0x7Fu);
              }
              pk[i2][q >> 1] |= h16 << (16 * (q & 1));
            }
          }
          unsigned char* dst = isA ? SA : SB;
          const uint32_t stride = isA ? OzL::ASL : OzL::BSL;
          const uint32_t off = bo(row, oct * 8);
#pragma unroll
          for (int i2 = 0; i2 < OZ_S; ++i2)
            *reinterpret_cast<uint4*>(dst + i2 * stride + off) = make_uint4(pk[i2][0], pk[i2][1], pk[i2][2], pk[i2][3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_arrive(conv + s);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(g.err, 1);
        break;
      }
    }
  } else if (warp >= epi_w0) {
    // ---------------------------------------------------------------- epilogue
    // each thread owns one accumulator row (its TMEM lane); an 8-column block of
    // results goes through a per-warp shared tile so that the global loads and
    // stores run along the rows (8 consecutive values per row, 4 rows per
    // instruction) instead of one row per lane
    const int quarter = warp & 3;   // the TMEM lane quarter this warp may read
    const int r = quarter * 32 + lane;
    const int ew = warp - epi_w0, part = ew >> 2, nparts = n_epi >> 2;   // column blocks part, part + nparts, ...
    double* stg = reinterpret_cast<double*>(sm + OzL::STG) + ew * (32 * 9);
    for (int64_t t = 0; t < my && !*abort_flag; ++t) {
      const OzItem it = oz_item(g, blockIdx.x + t * gridDim.x);
      const int c0 = it.c0, ncol = it.ncol;
      bool live;
      int Er;
      double* orow;
      if (g.mode == 0) {
        live = r < NL;
        Er = g.hexp[it.e * OZ_M + r];
        orow = live ? g.out + oz_cell_node(g.m, it.e, r) * g.ldo + c0 : nullptr;
      } else if (g.mode == 1) {
        const int64_t row = it.m0 + r;
        live = row < g.arows;
        Er = live ? g.aexp[row] : 0;
        orow = live ? g.out + row * g.ldo + c0 : nullptr;
      } else {
        const int64_t row = it.m0 + r;
        live = row < g.Na;
        Er = live ? g.aexp[row] : 0;
        orow = live ? g.part + ((int64_t)it.seg * g.Na + row) * g.N + c0 : nullptr;
      }
      if (img_only) {
        // Both operands pre-sliced (ROWS, GRAM): every K group's sum is added
        // into FP32 (hi, lo) pairs held in registers (error-free two-sum, then a
        // renormalisation: about 48 bits), so the TMEM accumulators are released
        // as soon as they are read and the next group's MMAs run while this
        // thread does its arithmetic; the FP64 result is formed and written once
        // per item.  Twelve epilogue warps: at most four 8-column blocks a thread.
        constexpr int MAXB = 4;
        float hi[MAXB][8], lo[MAXB][8];
        bool stop = false;
        for (int grp = 0; grp < ngrp; ++grp) {
          const int64_t gc = t * ngrp + grp;
          if (!bar_wait(accf, (uint32_t)(gc & 1))) {
            *abort_flag = 1;
            atomicExch(g.err, 1);
            stop = true;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int j = 0; j < MAXB; ++j) {
            const int cb = 8 * part + 8 * nparts * j;
            if (cb >= ncol) break;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {   // four columns at a time (fewer live registers)
              uint32_t v[OZ_NACC][4];
#pragma unroll
              for (int a = 0; a < OZ_NACC; ++a)
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v[a][0]), "=r"(v[a][1]), "=r"(v[a][2]), "=r"(v[a][3])
                             : "r"(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * OZ_TW + cb + 4 * hh))
                             : "memory");
              asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
              for (int qq = 0; qq < 4; ++qq) {
                const int q = 4 * hh + qq;
                float s1, e1, s2, e2, s3, e3;
                two_sum(__uint_as_float(v[0][qq]), __uint_as_float(v[1][qq]), s1, e1);
                two_sum(s1, __uint_as_float(v[2][qq]), s2, e2);
                two_sum(s2, __uint_as_float(v[3][qq]), s3, e3);
                const float lg = ((__uint_as_float(v[4][qq]) + e3) + e2) + e1;
                if (grp == 0) {
                  hi[j][q] = s3;
                  lo[j][q] = lg;
                } else {
                  float sh, eh;
                  two_sum(hi[j][q], s3, sh, eh);
                  const float l = (lo[j][q] + lg) + eh;
                  hi[j][q] = sh + l;
                  lo[j][q] = l - (hi[j][q] - sh);
                }
              }
            }
          }
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          bar_arrive(acce);
        }
        if (stop) break;
        const unsigned long long orow_u = (unsigned long long)orow;
#pragma unroll
        for (int j = 0; j < MAXB; ++j) {
          const int cb = 8 * part + 8 * nparts * j;
          if (cb >= ncol) break;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int n = cb + q;
            double val = 0.0;
            if (live && n < ncol) {
              const int k2 = Er + g.fexp[c0 + n] - 14;
              val = f32_scaled(hi[j][q], k2) + f32_scaled(lo[j][q], k2);
            }
            stg[lane * 9 + q] = val;
          }
          __syncwarp();
          // row rr = 4 jj + lane / 8 of this warp, column cb + lane % 8
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int rr = 4 * jj + (lane >> 3), cq = lane & 7;
            double* rp = (double*)__shfl_sync(0xffffffffu, orow_u, rr);
            const int lv = __shfl_sync(0xffffffffu, (int)live, rr);
            if (lv && cb + cq < ncol) rp[cb + cq] = stg[rr * 9 + cq];
          }
          __syncwarp();
        }
        continue;
      }
      // GRAM (not from images): the row's output segment is pulled towards L2
      // while the MMAs run
      if (live && g.mode == 2)
        for (int cb = 8 * part; cb < ncol; cb += 8 * nparts) asm volatile("prefetch.L2 [%0];" ::"l"(orow + cb));
      bool stop = false;
      for (int grp = 0; grp < ngrp; ++grp) {
        const int64_t gc = t * ngrp + grp;
        if (!bar_wait(accf, (uint32_t)(gc & 1))) {
          *abort_flag = 1;
          atomicExch(g.err, 1);
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // CELL adds to what is there (in L2: FP64 reductions, no read-back; a W value
        // receives one addition per launch since cells of a colour share no node),
        // GRAM and ROWS from their second group on
        const bool red = g.mode == 0;
        const bool add = !red && grp > 0;
        // with twelve epilogue warps the results go out through a per-warp shared
        // tile (rows written 8 values at a time, 4 rows per instruction); with four,
        // each thread writes its own row and loads the values it adds to one
        // 8-column block ahead (fewer instructions, which bound that case)
        const unsigned long long orow_u = (unsigned long long)orow;
        double nxt[8];
        if (!img_only && live && add) {
#pragma unroll
          for (int q = 0; q < 8; ++q) nxt[q] = (8 * part + q < ncol) ? orow[8 * part + q] : 0.0;
        }
        for (int cb = 8 * part; cb < ncol; cb += 8 * nparts) {
          double cur[8];
          if (!img_only) {
#pragma unroll
            for (int q = 0; q < 8; ++q) cur[q] = nxt[q];
            const int cn = cb + 8 * nparts;
            if (live && add && cn < ncol) {
#pragma unroll
              for (int q = 0; q < 8; ++q) nxt[q] = (cn + q < ncol) ? orow[cn + q] : 0.0;
            }
          }
          uint32_t v[OZ_NACC][8];
#pragma unroll
          for (int a = 0; a < OZ_NACC; ++a)
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(v[a][0]), "=r"(v[a][1]), "=r"(v[a][2]), "=r"(v[a][3]), "=r"(v[a][4]), "=r"(v[a][5]),
                  "=r"(v[a][6]), "=r"(v[a][7])
                : "r"(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(a * OZ_TW + cb))
                : "memory");
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          double val[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int n = cb + q;
            val[q] = 0.0;
            if (live && n < ncol) {
              float s1, e1, s2, e2, s3, e3;
              two_sum(__uint_as_float(v[0][q]), __uint_as_float(v[1][q]), s1, e1);
              two_sum(s1, __uint_as_float(v[2][q]), s2, e2);
              two_sum(s2, __uint_as_float(v[3][q]), s3, e3);
              const float lo = ((__uint_as_float(v[4][q]) + e3) + e2) + e1;
              // (s3 + lo) 2^k2: both parts scaled exactly by their bit patterns, one FP64
              // add (the FP64 pipe is the scarce one in this epilogue)
              const int k2 = Er + g.fexp[c0 + n] - 14;
              val[q] = f32_scaled(s3, k2) + f32_scaled(lo, k2);
            }
          }
          if (img_only) {
#pragma unroll
            for (int q = 0; q < 8; ++q) stg[lane * 9 + q] = val[q];
            __syncwarp();
            // row rr = 4 j + lane / 8 of this warp, column cb + lane % 8
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int rr = 4 * j + (lane >> 3), cq = lane & 7;
              double* rp = (double*)__shfl_sync(0xffffffffu, orow_u, rr);
              const int lv = __shfl_sync(0xffffffffu, (int)live, rr);
              if (lv && cb + cq < ncol) {
                const double x = stg[rr * 9 + cq];
                rp[cb + cq] = add ? rp[cb + cq] + x : x;
              }
            }
            __syncwarp();
          } else if (live && red) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              if (cb + q < ncol) asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(orow + cb + q), "d"(val[q]) : "memory");
          } else if (live) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
              if (cb + q < ncol) orow[cb + q] = add ? cur[q] + val[q] : val[q];
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        bar_arrive(acce);
      }
      if (stop) break;
    }
  }
  // all roles done.  After an abort, drain before the TMEM and the shared memory
  // are released: every bulk copy still in flight into the stage ring lands (a
  // copy thread issues into a stage only after its MMAs released it, so at most
  // the last OZ_STAGES chunks of a thread are outstanding; stages filled by the
  // other group are drained by that group's thread), and the last MMA commit --
  // which covers every MMA this CTA issued -- arrives.  Each drain wait is
  // bounded like the pipeline's own.
  __syncthreads();
  if (*abort_flag) {
    if (last_copy >= 0) {
      for (int64_t ch = last_copy - OZ_STAGES + 1; ch <= last_copy; ++ch)
        if (ch >= 0 && (img_only || (int)(ch % OZ_GROUPS) == (int)(last_copy % OZ_GROUPS)))
          bar_wait(afull + (int)(ch % OZ_STAGES), (uint32_t)((ch / OZ_STAGES) & 1));
    }
    if (warp == 0 && lane == 0 && last_mma >= 0)
      bar_wait(empty + (int)(last_mma % OZ_STAGES), (uint32_t)((last_mma / OZ_STAGES) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

// Digit images of every H^cc_e: per cell, per 16-wide K chunk, the seven 4 KB
// BF16 slices in the shared-memory layout of the MMA operand (row exponents hexp).
__global__ void k_oz_preslice(const double* __restrict__ H, const int* __restrict__ hexp, int64_t n_cell,
                              unsigned char* __restrict__ img) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;   // (cell, row, K octet)
  const int nch = (NL + OZ_KC - 1) / OZ_KC;
  if (t >= n_cell * OZ_M * nch * 2) return;
  const int oct = (int)(t % 2);
  const int kc = (int)((t / 2) % nch);
  const int row = (int)((t / (2 * nch)) % OZ_M);
  const int64_t e = t / (2 * nch * OZ_M);
  const int E = hexp[e * OZ_M + row];
  uint32_t pk[OZ_S][4];
#pragma unroll
  for (int i = 0; i < OZ_S; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) pk[i][q] = 0u;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = kc * OZ_KC + oct * 8 + q;
    const double x = (row < NL && k < NL) ? H[e * (int64_t)(NL * NL) + row * NL + k] : 0.0;
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const uint32_t sgn = (uint32_t)((bits >> 48) & 0x8000);
    unsigned long long qq = 0;
    const int rs = 1026 + E - ex;
    if (ex != 0 && rs >= 0 && rs < 64) qq = ((unsigned long long)(bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) >> rs;
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
      const uint32_t d = (uint32_t)(qq >> (42 - 7 * i)) & 127u;
      uint32_t h16 = 0;
      if (d) {
        const int p = 31 - __clz(d);
        h16 = sgn | ((uint32_t)(p + 127 - 7 * i) << 7) | ((d << (7 - p)) & 0x7Fu);
      }
      pk[i][q >> 1] |= h16 << (16 * (q & 1));
    }
  }
  unsigned char* base = img + ((e * nch + kc) * OZ_S) * (int64_t)OzL::ASL + bo(row, oct * 8);
#pragma unroll
  for (int i = 0; i < OZ_S; ++i)
    *reinterpret_cast<uint4*>(base + (int64_t)i * OzL::ASL) = make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
}

// Row image of a tall A (rows x K, the A operand of ROWS): per 128-row tile and
// 16-wide K chunk the seven 4 KB BF16 slices in the shared-memory layout of
// the MMA operand (row exponents aexp); rows past `rows` are zero.  One thread
// per (tile row, K octet); a warp covers 32 rows of one octet.
__global__ void k_oz_img_rows(const double* __restrict__ A, int64_t lda, int64_t rows, int K,
                              const int* __restrict__ aexp, unsigned char* __restrict__ img) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int nch = (K + OZ_KC - 1) / OZ_KC;
  const int64_t ntile = (rows + OZ_M - 1) / OZ_M;
  if (t >= ntile * nch * 2 * OZ_M) return;
  const int rr = (int)(t % OZ_M);
  const int oct = (int)((t / OZ_M) & 1);
  const int64_t tc = t / (2 * OZ_M);   // tile * nch + chunk
  const int c = (int)(tc % nch);
  const int64_t r = (tc / nch) * OZ_M + rr;
  double x[8];
  const int E = r < rows ? aexp[r] : -2000;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = c * OZ_KC + oct * 8 + q;
    x[q] = (r < rows && k < K) ? A[r * lda + k] : 0.0;
  }
  uint32_t pk[OZ_S][4];
  oz_pack8(x, E, pk);
  unsigned char* base = img + tc * OZ_S * (int64_t)OzL::ASL + bo(rr, oct * 8);
#pragma unroll
  for (int i = 0; i < OZ_S; ++i)
    *reinterpret_cast<uint4*>(base + (int64_t)i * OzL::ASL) = make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
}

// Column image of A (Krows x ncols): the K-major operand A^T, element (m, k) =
// A[k][m], per 128-column tile and 16-row chunk (nch chunks per tile, rows past
// Krows zero), seven 4 KB slices in the MMA layout (column exponents cexp).
// Columns past ncols rounded up to 16 are not written.  A warp reads 32
// consecutive columns of one row.
__global__ void k_oz_img_cols(const double* __restrict__ A, int64_t lda, int64_t Krows, int ncols,
                              const int* __restrict__ cexp, int64_t nch, unsigned char* __restrict__ img) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int ntile = (ncols + OZ_M - 1) / OZ_M;
  if (t >= (int64_t)ntile * nch * 2 * OZ_M) return;
  const int m = (int)(t % OZ_M);
  const int oct = (int)((t / OZ_M) & 1);
  const int64_t tc = t / (2 * OZ_M);   // tile * nch + chunk
  const int64_t c = tc % nch;
  const int col = (int)(tc / nch) * OZ_M + m;
  if (col >= ((ncols + 15) & ~15)) return;
  const int E = col < ncols ? cexp[col] : -2000;
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int64_t k = c * OZ_KC + oct * 8 + q;
    x[q] = (col < ncols && k < Krows) ? A[k * lda + col] : 0.0;
  }
  uint32_t pk[OZ_S][4];
  oz_pack8(x, E, pk);
  unsigned char* base = img + tc * OZ_S * (int64_t)OzL::ASL + bo(m, oct * 8);
#pragma unroll
  for (int i = 0; i < OZ_S; ++i)
    *reinterpret_cast<uint4*>(base + (int64_t)i * OzL::ASL) = make_uint4(pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
}

// per-row scale exponents of an FP64 matrix (one warp per row)
__global__ void k_oz_rowexp(const double* __restrict__ A, int64_t lda, int64_t rows, int K, int* __restrict__ eout) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= rows) return;
  int E = -2000;
  for (int k = lane; k < K; k += 32) E = max(E, exp_of(A[w * lda + k]));
  for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_down_sync(0xffffffffu, E, o));
  if (lane == 0) eout[w] = E;
}

// per-column scale exponents (max over rows), combined with integer atomicMax;
// blockIdx.x: a range of rows, blockIdx.y: a range of blockDim.x columns
__global__ void k_oz_colexp(const double* __restrict__ Y, int64_t ldy, int64_t rows, int N, int rows_per_block,
                            int* __restrict__ fout) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
  const int64_t r1 = min(rows, r0 + rows_per_block);
  const int c = blockIdx.y * blockDim.x + threadIdx.x;
  if (c >= N) return;
  int E = -2000;
  for (int64_t r = r0; r < r1; ++r) E = max(E, exp_of(Y[r * ldy + c]));
  atomicMax(fout + c, E);
}

__global__ void k_oz_fill(int* p, int n, int v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// row exponents of every cell block (rows 125..127 of the padded block get -2000)
__global__ void k_oz_hexp(const double* __restrict__ H, int64_t n_cell, int* __restrict__ hexp) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_cell * OZ_M) return;
  const int64_t e = w / OZ_M;
  const int r = (int)(w % OZ_M);
  int E = -2000;
  if (r < NL)
    for (int k = lane; k < NL; k += 32) E = max(E, exp_of(H[e * (int64_t)(NL * NL) + r * NL + k]));
  for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_down_sync(0xffffffffu, E, o));
  if (lane == 0) hexp[w] = E;
}

int oz_launch(const OzArgs& a, int n_sm, cudaStream_t st) {
  const int64_t nA = (a.mode == 0) ? a.ncells : (a.arows + OZ_M - 1) / OZ_M;
  const int64_t items = (a.mode == 2) ? (int64_t)a.npairs * a.nseg : nA * a.ntiles;
  if (items <= 0) return 0;
  const unsigned grid = (unsigned)(items < n_sm ? items : n_sm);
  if (a.mode != 0 && a.Aimg != nullptr && a.Bimg != nullptr) {
    cudaFuncSetAttribute(k_oz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OzL::TOTAL);
    k_oz<true><<<grid, OZ_THREADS, OzL::TOTAL, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_oz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OzL::TOTAL);
    k_oz<false><<<grid, OZ_THREADS, OzL::TOTAL, st>>>(a);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}

}  // namespace

int64_t oz_hexp_elems(int64_t n_cell) { return n_cell * OZ_M; }

void launch_oz_hexp(const double* Hcc, int64_t n_cell, int* hexp, cudaStream_t st) {
  const int64_t w = n_cell * OZ_M;
  if (w <= 0) return;
  k_oz_hexp<<<(unsigned)((w * 32 + 255) / 256), 256, 0, st>>>(Hcc, n_cell, hexp);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_oz_colexp(const double* Y, int64_t ldy, int64_t rows, int N, int* fexp, cudaStream_t st) {
  if (N <= 0) return;
  k_oz_fill<<<(N + 255) / 256, 256, 0, st>>>(fexp, N, -2000);
  // about eight CTAs per SM, each thread on at most 2048 rows of one column
  const int bt = N >= 128 ? 128 : 64;
  const int64_t ncb = (N + bt - 1) / bt;
  const int64_t want = 8LL * current_sm_count();
  const int64_t rpb = std::max<int64_t>(32, std::min<int64_t>(2048, (rows * ncb + want - 1) / want));
  const int64_t nb = (rows + rpb - 1) / rpb;
  if (nb > 0) k_oz_colexp<<<dim3((unsigned)nb, (unsigned)ncb), bt, 0, st>>>(Y, ldy, rows, N, (int)rpb, fexp);
  g_launches.fetch_add(2, std::memory_order_relaxed);
}

void launch_oz_rowexp(const double* A, int64_t lda, int64_t rows, int K, int* aexp, cudaStream_t st) {
  if (rows <= 0) return;
  k_oz_rowexp<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(A, lda, rows, K, aexp);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// W(nodes of the colour's cells) += H^cc_e Y_e, FP64-grade through the BF16 tensor cores.
// fexp: per-column exponents of Y (launch_oz_colexp).
int64_t oz_cell_image_bytes() { return (int64_t)((NL + OZ_KC - 1) / OZ_KC) * OZ_S * OzL::ASL; }

void launch_oz_preslice(const double* Hcc, const int* hexp, int64_t n_cell, unsigned char* img, cudaStream_t st) {
  const int64_t n = n_cell * OZ_M * ((NL + OZ_KC - 1) / OZ_KC) * 2;
  if (n <= 0) return;
  k_oz_preslice<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Hcc, hexp, n_cell, img);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

int launch_oz_cell(const double* Hcc, const int* hexp, const int32_t* cells, int64_t ncells, const MeshDev& m,
                   const double* Y, int64_t ldy, const int* fexp, double* W, int64_t ldw, int N, int n_sm, int* err,
                   cudaStream_t st, const unsigned char* Aimg, int stall) {
  if (ncells <= 0 || N <= 0) return 0;
  OzArgs a{};
  a.mode = 0;
  a.H = Hcc;
  a.hexp = hexp;
  a.Aimg = Aimg;
  a.cells = cells;
  a.ncells = ncells;
  a.m = m;
  a.K = NL;
  a.Y = Y;
  a.ldy = ldy;
  a.fexp = fexp;
  a.out = W;
  a.ldo = ldw;
  a.N = N;
  a.ntiles = (N + OZ_TW - 1) / OZ_TW;
  a.err = err;
  a.stall = stall;
  return oz_launch(a, n_sm, st);
}

int64_t oz_img_rows_bytes(int64_t rows, int K) {
  return ((rows + OZ_M - 1) / OZ_M) * ((K + OZ_KC - 1) / OZ_KC) * OZ_S * (int64_t)OzL::ASL;
}

int64_t oz_img_cols_bytes(int64_t nch, int ncols) {
  return (int64_t)((ncols + OZ_M - 1) / OZ_M) * nch * OZ_S * (int64_t)OzL::ASL;
}

void launch_oz_img_rows(const double* A, int64_t lda, int64_t rows, int K, const int* aexp, unsigned char* img,
                        cudaStream_t st) {
  const int64_t n = ((rows + OZ_M - 1) / OZ_M) * ((K + OZ_KC - 1) / OZ_KC) * 2 * OZ_M;
  if (n <= 0) return;
  k_oz_img_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A, lda, rows, K, aexp, img);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_oz_img_cols(const double* A, int64_t lda, int64_t Krows, int ncols, const int* cexp, int64_t nch,
                        unsigned char* img, cudaStream_t st) {
  const int64_t n = (int64_t)((ncols + OZ_M - 1) / OZ_M) * nch * 2 * OZ_M;
  if (n <= 0) return;
  k_oz_img_cols<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A, lda, Krows, ncols, cexp, nch, img);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// C = A B (A: rows x K; B: K x N), FP64-grade; aexp / bexp from
// launch_oz_rowexp(A) and launch_oz_colexp(B).  Aimg / Bimg (optional):
// launch_oz_img_rows(A) and launch_oz_img_cols(B, nch = ceil(K / 16)).
int launch_oz_rows(const double* A, int64_t lda, int64_t rows, int K, const int* aexp, const double* B, int64_t ldb,
                   const int* bexp, double* C, int64_t ldc, int N, int n_sm, int* err, cudaStream_t st,
                   const unsigned char* Aimg, const unsigned char* Bimg, int stall) {
  if (rows <= 0 || N <= 0 || K <= 0) return 0;
  OzArgs a{};
  a.Aimg = Aimg;
  a.Bimg = Bimg;
  a.mode = 1;
  a.A = A;
  a.lda = lda;
  a.arows = rows;
  a.aexp = aexp;
  a.B = B;
  a.ldb = ldb;
  a.K = K;
  a.fexp = bexp;
  a.out = C;
  a.ldo = ldc;
  a.N = N;
  a.ntiles = (N + OZ_TW - 1) / OZ_TW;
  a.err = err;
  a.stall = stall;
  return oz_launch(a, n_sm, st);
}

// C (Na x N) = A^T B for tall A (K x Na) and B (K x N), FP64-grade: the K rows
// are cut into segments (work items with the tile pairs), each segment's
// product is formed in 256-row groups (exact FP32 accumulation) and summed in
// FP64 into its partial tile; partials are then added in fixed order.  sym:
// C is symmetric, only tiles that meet the upper triangle are formed and the
// rest is mirrored.  aexp / bexp: launch_oz_colexp of A and B.  work: at least
// oz_gram_work_elems doubles; pairs_dev: at least oz_gram_max_pairs int2.
int64_t oz_gram_segments(int64_t K, int npairs, int n_sm) {
  int64_t nseg = std::max<int64_t>(1, (2 * (int64_t)n_sm + npairs - 1) / npairs);
  nseg = std::min<int64_t>(nseg, (K + 255) / 256);
  return std::max<int64_t>(nseg, 1);
}

int oz_gram_pairs(int Na, int N, bool sym, int2* pairs_host) {
  const int mt = (Na + OZ_M - 1) / OZ_M, nt = (N + OZ_TW - 1) / OZ_TW;
  int np = 0;
  for (int i = 0; i < mt; ++i)
    for (int j = 0; j < nt; ++j) {
      if (sym && i * OZ_M > j * OZ_TW + OZ_TW - 1) continue;   // tile entirely below the diagonal
      if (pairs_host) pairs_host[np] = make_int2(i, j);
      ++np;
    }
  return np;
}

namespace {
__global__ void k_oz_gram_reduce(int nseg, int Na, int N, const double* __restrict__ part, int sym, int accumulate,
                                 double* __restrict__ C, int64_t ldc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)Na * N) return;
  const int i = (int)(idx / N), j = (int)(idx % N);
  const bool mirror = sym && i > j;
  const int64_t src = mirror ? (int64_t)j * N + i : idx;
  double s = accumulate ? C[(int64_t)i * ldc + j] : 0.0;
  for (int k = 0; k < nseg; ++k) s += part[(int64_t)k * Na * N + src];
  C[(int64_t)i * ldc + j] = s;
}
}  // namespace

int launch_oz_gram(int64_t K, int Na, int N, const double* A, int64_t lda, const int* aexp, const double* B,
                   int64_t ldb, const int* bexp, double* C, int64_t ldc, bool sym, double* work, int64_t work_elems,
                   int2* pairs_dev, int n_sm, int* err, cudaStream_t st, unsigned char* img_a,
                   int64_t img_a_bytes, unsigned char* img_b, int64_t img_b_bytes, bool accumulate, int stall) {
  if (K <= 0 || Na <= 0 || N <= 0) return 0;
  if (sym && Na != N) return 1;
  std::vector<int2> pairs(oz_gram_pairs(Na, N, sym, nullptr));
  const int np = oz_gram_pairs(Na, N, sym, pairs.data());
  int64_t nseg = oz_gram_segments(K, np, n_sm);
  while (nseg > 1 && nseg * (int64_t)Na * N > work_elems) --nseg;
  if (nseg * (int64_t)Na * N > work_elems) return 1;
  const int64_t seg_len = ((K + nseg - 1) / nseg + 255) / 256 * 256;
  nseg = (K + seg_len - 1) / seg_len;
  if (cudaMemcpyAsync(pairs_dev, pairs.data(), sizeof(int2) * np, cudaMemcpyHostToDevice, st) != cudaSuccess) return 1;
  OzArgs a{};
  a.mode = 2;
  a.A = A;
  a.lda = lda;
  a.B = B;
  a.ldb = ldb;
  a.aexp = aexp;
  a.fexp = bexp;
  a.Kbig = K;
  a.seg_len = seg_len;
  a.Na = Na;
  a.N = N;
  a.nseg = (int)nseg;
  a.npairs = np;
  a.pairs = pairs_dev;
  a.part = work;
  a.ntiles = (N + OZ_TW - 1) / OZ_TW;
  a.err = err;
  a.stall = stall;
  // column images of A and B (one image when B is A) covering every segment
  const int64_t nch = nseg * seg_len / OZ_KC;
  if (img_a && oz_img_cols_bytes(nch, Na) <= img_a_bytes &&
      (B == A || (img_b && oz_img_cols_bytes(nch, N) <= img_b_bytes))) {
    launch_oz_img_cols(A, lda, K, Na, aexp, nch, img_a, st);
    if (B != A) launch_oz_img_cols(B, ldb, K, N, bexp, nch, img_b, st);
    a.Aimg = img_a;
    a.Bimg = (B == A) ? img_a : img_b;
    a.img_nch = nch;
  }
  if (oz_launch(a, n_sm, st)) return 1;
  k_oz_gram_reduce<<<(unsigned)(((int64_t)Na * N + 255) / 256), 256, 0, st>>>((int)nseg, Na, N, work, sym ? 1 : 0,
                                                                             accumulate ? 1 : 0, C, ldc);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}

int oz_gram_max_pairs(int Na, int N) { return oz_gram_pairs(Na, N, false, nullptr); }

}  // namespace efe