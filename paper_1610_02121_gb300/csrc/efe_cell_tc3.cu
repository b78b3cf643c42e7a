// Warp-specialised tensor-core cell products (tcgen05 + bulk async copies, sm_103a).
//
// Paper, Sec. V (last paragraph): W_c(e) += H^cc_e Y_c(e) for every cell of
// one parity colour (cells of a colour share no node, so the scatter needs no
// atomics), one M = 128, K = 128 (four 32-wide chunks), N <= 160 TF32 product
// per cell and column tile, FP32 accumulation in tensor memory.
//
// Roles of the 16 warps of a persistent CTA:
//   warp 0      producer: per chunk one bulk copy of the cell's FP32 image
//               (H^cc_e, 16 KB, already in the core-matrix layout) and one
//               bulk copy per node row of Y into a raw staging buffer, all
//               completing on mbarrier `full`;
//   warp 1      MMA issuer: 4 (one pass) or 12 (3-term split: A1 B1 + A1 B2 +
//               A2 B1) tcgen05.mma per chunk into one of two TMEM
//               accumulators, commits to `empty` (stage reusable) and, after
//               the last chunk, to `acc_full`;
//   warps 2-7   converters: the A chunk in place -> A1 = TF32(A) (and A2 =
//               the TF32 remainder), raw rows -> K-major core-matrix B1 (and
//               B2), arrive on `conv`;
//   warps 8-15  epilogue: tcgen05.ld of the accumulator rows, scatter-add into
//               W as vector reductions performed in L2 (no read-back), arrive
//               on `acc_empty`.
// Two stages ring the chunks.  Every wait is bounded (about one second); on
// timeout the CTA records an error, stops issuing, drains and frees its TMEM.
#include <cuda_bf16.h>
#include <stdint.h>

#include "efe_kernels.h"

namespace efe {

namespace {

constexpr int T3_M = 128, T3_K = 128, T3_KC = 32, T3_NCH = 4;
constexpr int T3_STAGES = 2;
// column tile (template parameter TW of the kernel): 64, 96 or 160, picked per
// system and N by the autotuner (efe_autotune); 160 by default
constexpr int T3_THREADS = 512;
constexpr int T3_CONV_WARP0 = 2, T3_CONV_WARPS = 6;
constexpr int T3_EPI_WARP0 = 8, T3_EPI_WARPS = 8;
constexpr uint32_t T3_TMEM_COLS = 512;     // accumulators at columns 0 and 256
constexpr long long T3_WAIT = 2000000000LL;

template <int TW>
struct T3Layout {
  // stage: A1 | A2 | B1 | B2 | Braw      (bytes)
  static constexpr uint32_t A = T3_M * T3_KC * 4;           // 16 KB
  static constexpr uint32_t B = TW * T3_KC * 4;             // 20 KB at TW = 160
  static constexpr uint32_t RAW = T3_KC * TW * 4;           // 20 KB at TW = 160
  static constexpr uint32_t STAGE = 2 * A + 2 * B + RAW;    // 92 KB at TW = 160
  static constexpr uint32_t BARS = T3_STAGES * STAGE;       // barrier area offset
  static constexpr size_t TOTAL = (size_t)BARS + 256;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  // K-major, no swizzle: LBO = 128 B (next K core matrix), SBO = 1024 B (next 8 rows), version 1
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(T3_M >> 4) << 24);
}

// BF16 operands (kind::f16): FP32 accumulate, BF16 A and B
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(T3_M >> 4) << 24);
}

// K-major BF16 chunk of 32 K: core matrix 8 rows x 16 B (8 K); LBO = 128 B (next 8 K),
// SBO = 512 B (next 8 rows)
__device__ __forceinline__ uint64_t sdesc_bf16(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
         ((uint64_t)1 << 46);
}
__device__ __forceinline__ uint32_t bmo(int row, int k) {
  return (uint32_t)(row >> 3) * 512u + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}
__device__ __forceinline__ uint16_t bf16r(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
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
  } while (clock64() - t0 < T3_WAIT);
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}

// node id of local row k (0..124) of cell e
__device__ __forceinline__ int64_t cell_node(const MeshDev& m, int64_t e, int k) {
  const int i = (int)(e % m.nc[0]), j = (int)((e / m.nc[0]) % m.nc[1]), kk = (int)(e / ((int64_t)m.nc[0] * m.nc[1]));
  const int a = k % NP1, b = (k / NP1) % NP1, c = k / (NP1 * NP1);
  return (int64_t)(P * i + a) + (int64_t)m.nn[0] * ((int64_t)(P * j + b) + (int64_t)m.nn[1] * (int64_t)(P * kk + c));
}

// K-major core-matrix offset (bytes) within a 32-wide chunk
__device__ __forceinline__ uint32_t cmo(int row, int k) {
  return (uint32_t)(row >> 3) * 1024u + (uint32_t)(k >> 2) * 128u + (uint32_t)(row & 7) * 16u;
}

// MODE 0: one TF32 pass; 1: 3-term TF32 split (a1 b1 + a1 b2 + a2 b1); 2: BF16 operands
template <int MODE, int TW>
__global__ void __launch_bounds__(T3_THREADS, 1) k_cell_tc3(const float* __restrict__ Ag,
                                                            const int32_t* __restrict__ cells, int64_t ncells,
                                                            MeshDev m, const float* __restrict__ Y, int64_t ldy,
                                                            float* __restrict__ W, int64_t ldw, int N, int ntiles,
                                                            int* __restrict__ err, int stall) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // an earlier launch already failed: leave at once (CTA-uniform decision)
  __shared__ int s_skip;
  if (tid == 0) s_skip = *(volatile int*)err;
  __syncthreads();
  if (s_skip) return;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + T3Layout<TW>::BARS);  // [2]
  uint64_t* conv = full + 2;                                          // [2]
  uint64_t* empty = full + 4;                                         // [2]
  uint64_t* accf = full + 6;                                          // [2]
  uint64_t* acce = full + 8;                                          // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(full + 10);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(full + 11);
  uint64_t* never = full + 12;   // no thread ever arrives here (the test stall waits on it)

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(T3_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    for (int s = 0; s < T3_STAGES; ++s) {
      bar_init(full + s, 1);
      bar_init(conv + s, T3_CONV_WARPS * 32);
      bar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(accf + b, 1);
      bar_init(acce + b, T3_EPI_WARPS * 32);
    }
    bar_init(never, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const int64_t nitems = ncells * ntiles;
  const int64_t my_items = nitems > blockIdx.x ? (nitems - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  // the last chunk whose bulk copies this thread issued / whose MMAs it committed
  // (drained before the TMEM is released if the CTA aborts)
  int64_t last_copy = -1, last_mma = -1;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    for (int64_t t = 0; t < my_items && !*abort_flag; ++t) {
      const int64_t item = blockIdx.x + t * gridDim.x;
      const int64_t e = cells[item / ntiles];
      const int c0 = (int)(item % ntiles) * TW;
      const int ncol = min(TW, N - c0);
      const uint32_t row_bytes = (uint32_t)((ncol + 3) / 4) * 16u;
      for (int kc = 0; kc < T3_NCH; ++kc) {
        const int64_t ch = t * T3_NCH + kc;
        const int s = (int)(ch % T3_STAGES);
        if (ch >= T3_STAGES && !bar_wait(empty + s, (uint32_t)((ch / T3_STAGES - 1) & 1))) {
          if (lane == 0) { *abort_flag = 1; atomicExch(err, 1); }
          break;
        }
        unsigned char* S = sm + s * T3Layout<TW>::STAGE;
        const int nrows = min(T3_KC, NL - kc * T3_KC);
        if (lane == 0) bar_expect_tx(full + s, T3Layout<TW>::A + (uint32_t)nrows * row_bytes);
        __syncwarp();
        if (lane == 0) bulk_g2s(S, Ag + (e * T3_NCH + kc) * (T3_M * T3_KC), T3Layout<TW>::A, full + s);
        if (lane < nrows) {
          const int64_t g = cell_node(m, e, kc * T3_KC + lane);
          bulk_g2s(S + 2 * T3Layout<TW>::A + 2 * T3Layout<TW>::B + (uint32_t)lane * (TW * 4), Y + g * ldy + c0, row_bytes,
                   full + s);
        }
        last_copy = ch;
        __syncwarp();
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (stall && my_items > 0 && !bar_wait(never, 0u)) {
      // test stall: a wait that nothing completes runs out like a real one
      if (lane == 0) { *abort_flag = 1; atomicExch(err, 1); }
    }
    for (int64_t t = 0; t < my_items && !*abort_flag; ++t) {
      const int64_t item = blockIdx.x + t * gridDim.x;
      const int c0 = (int)(item % ntiles) * TW;
      const int ncol = min(TW, N - c0);
      const int nmma = ((ncol + 15) / 16) * 16;
      const int b = (int)(t & 1);
      bool ok = true;
      if (t >= 2) ok = bar_wait(acce + b, (uint32_t)((t / 2 - 1) & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kc = 0; kc < T3_NCH && ok; ++kc) {
        const int64_t ch = t * T3_NCH + kc;
        const int s = (int)(ch % T3_STAGES);
        ok = bar_wait(conv + s, (uint32_t)((ch / T3_STAGES) & 1));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;
        if (lane == 0) {
          unsigned char* S = sm + s * T3Layout<TW>::STAGE;
          const uint32_t a1 = su32(S), a2 = a1 + T3Layout<TW>::A, b1 = a1 + 2 * T3Layout<TW>::A, b2 = b1 + T3Layout<TW>::B;
          const uint32_t d = tmem + (uint32_t)(b * 256);
          if (MODE == 2) {
            // BF16: the A chunk's BF16 copy in the A2 area, B in the B1 area; K = 16 per MMA
            const uint32_t id = idesc_bf16(nmma);
#pragma unroll
            for (int ks = 0; ks < T3_KC / 16; ++ks) {
              const uint32_t off = (uint32_t)ks * 256u;
              mma_bf16(d, sdesc_bf16(a2 + off), sdesc_bf16(b1 + off), id, (kc > 0 || ks > 0) ? 1u : 0u);
            }
          } else {
            const uint32_t id = idesc_tf32(nmma);
#pragma unroll
            for (int ks = 0; ks < T3_KC / 8; ++ks) {
              const uint32_t off = (uint32_t)ks * 256u;
              mma_tf32(d, sdesc(a1 + off), sdesc(b1 + off), id, (kc > 0 || ks > 0) ? 1u : 0u);
              if (MODE == 1) {
                mma_tf32(d, sdesc(a1 + off), sdesc(b2 + off), id, 1u);
                mma_tf32(d, sdesc(a2 + off), sdesc(b1 + off), id, 1u);
              }
            }
          }
          mma_commit(empty + s);
          if (kc == T3_NCH - 1) mma_commit(accf + b);
        }
        last_mma = ch;
        __syncwarp();
      }
      if (!ok) {
        if (lane == 0) { *abort_flag = 1; atomicExch(err, 1); }
        break;
      }
    }
  } else if (warp < T3_CONV_WARP0 + T3_CONV_WARPS) {
    // ------------------------------------------------------------ converters
    const int ct = tid - T3_CONV_WARP0 * 32;
    for (int64_t t = 0; t < my_items && !*abort_flag; ++t) {
      const int64_t item = blockIdx.x + t * gridDim.x;
      const int c0 = (int)(item % ntiles) * TW;
      const int ncol = min(TW, N - c0);
      const int nmma = ((ncol + 15) / 16) * 16;
      bool ok = true;
      for (int kc = 0; kc < T3_NCH; ++kc) {
        const int64_t ch = t * T3_NCH + kc;
        const int s = (int)(ch % T3_STAGES);
        ok = bar_wait(full + s, (uint32_t)((ch / T3_STAGES) & 1));
        if (!ok) break;
        unsigned char* S = sm + s * T3Layout<TW>::STAGE;
        const float* raw = reinterpret_cast<const float*>(S + 2 * T3Layout<TW>::A + 2 * T3Layout<TW>::B);
        unsigned char* B1 = S + 2 * T3Layout<TW>::A;
        unsigned char* B2 = B1 + T3Layout<TW>::B;
        const int nrows = min(T3_KC, NL - kc * T3_KC);
        if (MODE == 2) {
          // BF16 copies: the A chunk (FP32 image, 4-wide K core matrices) into the A2
          // area and the raw rows into the B1 area, both in the 8-wide K layout
          unsigned char* A2 = S + T3Layout<TW>::A;
          const float4* a1 = reinterpret_cast<const float4*>(S);
          for (int v = ct; v < (int)(T3Layout<TW>::A / 16); v += T3_CONV_WARPS * 32) {
            // 16-byte unit v of the FP32 image: row r, K quad kq (cmo layout)
            const int rg = v >> 6, kq = (v >> 3) & 7, ri = v & 7;
            const int r = rg * 8 + ri, k = kq * 4;
            const float4 x = a1[v];
            ushort4 h;
            h.x = bf16r(x.x); h.y = bf16r(x.y); h.z = bf16r(x.z); h.w = bf16r(x.w);
            *reinterpret_cast<ushort4*>(A2 + bmo(r, k)) = h;
          }
          for (int v = ct; v < nmma * 8; v += T3_CONV_WARPS * 32) {
            const int n = v % nmma, kq = v / nmma;
            ushort4 h;
            uint16_t* hp = reinterpret_cast<uint16_t*>(&h);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int kr = kq * 4 + q;
              hp[q] = bf16r((kr < nrows && n < ncol) ? raw[kr * TW + n] : 0.f);
            }
            *reinterpret_cast<ushort4*>(B1 + bmo(n, kq * 4)) = h;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          bar_arrive(conv + s);
          continue;
        }
        {
          // the A chunk in place: A1 = TF32(A), A2 = TF32(A - A1) (elementwise, any layout)
          float4* a1 = reinterpret_cast<float4*>(S);
          float4* a2 = reinterpret_cast<float4*>(S + T3Layout<TW>::A);
          for (int v = ct; v < (int)(T3Layout<TW>::A / 16); v += T3_CONV_WARPS * 32) {
            const float4 x = a1[v];
            float4 h4;
            h4.x = tf32r(x.x); h4.y = tf32r(x.y); h4.z = tf32r(x.z); h4.w = tf32r(x.w);
            a1[v] = h4;
            if (MODE == 1) {
              float4 l4;
              l4.x = tf32r(x.x - h4.x); l4.y = tf32r(x.y - h4.y); l4.z = tf32r(x.z - h4.z); l4.w = tf32r(x.w - h4.w);
              a2[v] = l4;
            }
          }
        }
        for (int v = ct; v < nmma * 8; v += T3_CONV_WARPS * 32) {
          const int n = v % nmma, kq = v / nmma;
          float y[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int kr = kq * 4 + q;
            y[q] = (kr < nrows && n < ncol) ? raw[kr * TW + n] : 0.f;
          }
          float4 h4, l4;
          h4.x = tf32r(y[0]); h4.y = tf32r(y[1]); h4.z = tf32r(y[2]); h4.w = tf32r(y[3]);
          *reinterpret_cast<float4*>(B1 + cmo(n, kq * 4)) = h4;
          if (MODE == 1) {
            l4.x = tf32r(y[0] - h4.x); l4.y = tf32r(y[1] - h4.y); l4.z = tf32r(y[2] - h4.z); l4.w = tf32r(y[3] - h4.w);
            *reinterpret_cast<float4*>(B2 + cmo(n, kq * 4)) = l4;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_arrive(conv + s);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 1);
        break;
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int ew = warp - T3_EPI_WARP0;  // 0..7
    const int quarter = warp & 3;         // TMEM lane quarter accessible to this warp
    const int colgrp = ew >> 2;           // 0..1
    const int r = quarter * 32 + lane;
    for (int64_t t = 0; t < my_items && !*abort_flag; ++t) {
      const int64_t item = blockIdx.x + t * gridDim.x;
      const int64_t e = cells[item / ntiles];
      const int c0 = (int)(item % ntiles) * TW;
      const int ncol = min(TW, N - c0);
      const int b = (int)(t & 1);
      const int64_t g = (r < NL) ? cell_node(m, e, r) : 0;
      float* wr = W + g * ldw + c0;
      if (!bar_wait(accf + b, (uint32_t)((t / 2) & 1))) {
        *abort_flag = 1;
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int cb = colgrp * 16; cb < ncol; cb += 32) {
        const bool full16 = (r < NL) && cb + 16 <= ncol;
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256 + cb))
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        // the products are added in L2 (vector reductions, no read-back): a W value
        // receives one addition per launch (cells of a colour share no node)
        if (r < NL) {
          if (full16) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(wr + cb + 4 * q),
                           "f"(__uint_as_float(v[4 * q])), "f"(__uint_as_float(v[4 * q + 1])),
                           "f"(__uint_as_float(v[4 * q + 2])), "f"(__uint_as_float(v[4 * q + 3]))
                           : "memory");
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (cb + q < ncol) atomicAdd(wr + cb + q, __uint_as_float(v[q]));
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      bar_arrive(acce + b);
    }
  }
  // all roles done.  After an abort, drain before the TMEM and the shared memory
  // are released: every bulk copy issued into the stage ring lands (at most
  // T3_STAGES chunks are in flight: the producer waits for a stage to empty
  // before refilling it), and the last MMA commit (it covers every MMA this CTA
  // issued) arrives; each drain wait is bounded like the pipeline's own.
  __syncthreads();
  if (*abort_flag) {
    if (warp == 0 && lane == 0 && last_copy >= 0) {
      for (int64_t ch = last_copy - T3_STAGES + 1; ch <= last_copy; ++ch)
        if (ch >= 0) bar_wait(full + (int)(ch % T3_STAGES), (uint32_t)((ch / T3_STAGES) & 1));
    }
    if (warp == 1 && lane == 0 && last_mma >= 0)
      bar_wait(empty + (int)(last_mma % T3_STAGES), (uint32_t)((last_mma / T3_STAGES) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T3_TMEM_COLS) : "memory");
  }
}

// TF32 split images of H^cc_e, chunk-major: [cell][chunk][row group][1 KB], each
// chunk a contiguous 16 KB image of the K-major core-matrix layout.
// A1 = tf32(h), A2 = tf32(h - A1) (h in FP64).
__global__ void k_build_aimg(const double* __restrict__ Hcc, int64_t n_cell, float* __restrict__ A) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_cell * T3_M * T3_K) return;
  const int64_t e = idx / (T3_M * T3_K);
  const int rk = (int)(idx % (T3_M * T3_K));
  const int r = rk / T3_K, k = rk % T3_K;
  const double h = (r < NL && k < NL) ? Hcc[e * (int64_t)(NL * NL) + r * NL + k] : 0.0;
  const int kc = k / T3_KC, kl = k % T3_KC;
  const int64_t off = (e * T3_NCH + kc) * (T3_M * T3_KC) + (cmo(r, kl) + (uint32_t)(kl & 3) * 4u) / 4;
  A[off] = (float)h;
}

}  // namespace

int64_t tc3_image_elems(int64_t n_cell) { return n_cell * T3_M * T3_K; }

void launch_build_aimg(const double* Hcc, int64_t n_cell, float* A, cudaStream_t st) {
  const int64_t n = n_cell * T3_M * T3_K;
  if (n <= 0) return;
  k_build_aimg<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Hcc, n_cell, A);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// W += H_e Y_e over the cells of one colour.  Y / W: FP32 rows, ld a multiple of 4
// elements and rows 16-byte aligned (the bulk copies need 16-byte sizes and addresses).
namespace {
template <int TW>
void tc3_launch(const float* A, const int32_t* cells, int64_t ncells, const MeshDev& m,
                const float* Y, int64_t ldy, float* W, int64_t ldw, int N, int mode, int n_sm, int* err,
                cudaStream_t st, int stall) {
  const int ntiles = (N + TW - 1) / TW;
  const int64_t items = ncells * ntiles;
  const unsigned grid = (unsigned)(items < n_sm ? items : n_sm);
  const size_t smem = T3Layout<TW>::TOTAL;
  if (mode == 1) {
    cudaFuncSetAttribute(k_cell_tc3<1, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cell_tc3<1, TW><<<grid, T3_THREADS, smem, st>>>(A, cells, ncells, m, Y, ldy, W, ldw, N, ntiles, err, stall);
  } else if (mode == 2) {
    cudaFuncSetAttribute(k_cell_tc3<2, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cell_tc3<2, TW><<<grid, T3_THREADS, smem, st>>>(A, cells, ncells, m, Y, ldy, W, ldw, N, ntiles, err, stall);
  } else {
    cudaFuncSetAttribute(k_cell_tc3<0, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cell_tc3<0, TW><<<grid, T3_THREADS, smem, st>>>(A, cells, ncells, m, Y, ldy, W, ldw, N, ntiles, err, stall);
  }
}
}  // namespace

const int* tc3_tiles(int* count) {
  static const int tiles[3] = {64, 96, 160};
  *count = 3;
  return tiles;
}

int launch_cell_tc3(const float* A, const int32_t* cells, int64_t ncells, const MeshDev& m,
                    const float* Y, int64_t ldy, float* W, int64_t ldw, int N, int mode, int n_sm, int* err,
                    cudaStream_t st, int tile, int stall) {
  if (ncells <= 0 || N <= 0) return 0;
  if ((ldy & 3) || (ldw & 3)) return 1;
  if (tile == 64)
    tc3_launch<64>(A, cells, ncells, m, Y, ldy, W, ldw, N, mode, n_sm, err, st, stall);
  else if (tile == 96)
    tc3_launch<96>(A, cells, ncells, m, Y, ldy, W, ldw, N, mode, n_sm, err, st, stall);
  else if (tile == 160 || tile == 0)
    tc3_launch<160>(A, cells, ncells, m, Y, ldy, W, ldw, N, mode, n_sm, err, st, stall);
  else
    return 1;
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}

}  // namespace efe
