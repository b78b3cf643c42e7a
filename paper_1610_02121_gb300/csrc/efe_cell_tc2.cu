// Pipelined tensor-core cell products (tcgen05, sm_103a) for the FP32-storage
// Chebyshev filter, with an optional 3-term TF32 split that gives FP32-grade
// products (a*b ~ a1*b1 + a1*b2 + a2*b1 with a = a1 + a2, b = b1 + b2, each
// part TF32-rounded; the dropped a2*b2 term is ~2^-22 relative).
//
// Paper, Sec. V (last paragraph): W_c(e) += H^cc_e Y_c(e) for every cell,
// then assembly.  Per cell one M = 128, K = 128, N = n_mma tensor-core
// product, K streamed in four 32-wide chunks through a 3-stage shared-memory
// ring; the FP32 accumulator lives in one of two TMEM buffers so that the
// epilogue (tcgen05.ld, scatter-add into W) of one cell overlaps the MMAs of
// the next.  CTAs are persistent over the cells of one parity colour (cells of
// a colour share no node: the scatter needs no atomics).  All waits are bounded.
#include <stdint.h>

#include "efe_kernels.h"

namespace efe {

namespace {

constexpr int T2_M = 128, T2_K = 128, T2_KC = 32;   // rows, reduction, K chunk
constexpr int T2_NCH = T2_K / T2_KC;               // chunks per cell
constexpr int T2_STAGES = 3;
constexpr int T2_THREADS = 512;
constexpr long long T2_WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz
constexpr uint32_t T2_TMEM_COLS = 512;             // two accumulators (columns 0 and 256)
constexpr int T2_TW = 160;                          // column tile: 3 stages of 128 x 32 A (x2) and
                                                    // 160 x 32 B (x2) fit in 227 KB of shared memory

__device__ __forceinline__ uint32_t s_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t desc_noswz(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t idesc_tf32(int n_mma) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n_mma >> 3) << 17) | ((uint32_t)(T2_M >> 4) << 24);
}

__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool wait_parity(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  const long long t0 = clock64();
  while (clock64() - t0 < T2_WAIT_CYCLES) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(s_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

struct T2Smem {
  // per stage: A1, A2 (128 x 32 TF32 = 16 KB each), B1, B2 (n_mma x 32 TF32)
  static __host__ __device__ uint32_t a_bytes() { return T2_M * T2_KC * 4; }
  static __host__ __device__ uint32_t b_bytes(int n_mma) { return (uint32_t)n_mma * T2_KC * 4; }
  static __host__ __device__ uint32_t stage_bytes(int n_mma) { return 2 * a_bytes() + 2 * b_bytes(n_mma); }
  static __host__ __device__ size_t total(int n_mma) {
    return (size_t)T2_STAGES * stage_bytes(n_mma) + 2 * 128 * sizeof(int64_t) + 16 * sizeof(uint64_t) + 64;
  }
};

// K-major no-swizzle core-matrix offset within a 32-wide K chunk (SBO = 1024 B, LBO = 128 B)
__device__ __forceinline__ uint32_t cm32(int row, int k) {
  return (uint32_t)(row >> 3) * 1024u + (uint32_t)(k >> 2) * 128u + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

template <bool SPLIT>
__global__ void __launch_bounds__(T2_THREADS, 1) k_cell_tc2(const float* __restrict__ Araw,
                                                            const int32_t* __restrict__ cells, int64_t ncells,
                                                            MeshDev m, const float* __restrict__ Y, int64_t ldy,
                                                            float* __restrict__ W, int64_t ldw, int N, int n_mma,
                                                            int ntiles, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sb = T2Smem::stage_bytes(n_mma);
  unsigned char* stg = smem;
  int64_t* gnode = reinterpret_cast<int64_t*>(smem + T2_STAGES * sb);  // [2][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(gnode + 256);           // stage_free[3], acc_full[2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 8);
  uint64_t* stage_free = bars;
  uint64_t* acc_full = bars + 3;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(tslot)),
                 "r"(T2_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < 5; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(bars + i)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = idesc_tf32(n_mma);
  const int64_t NX = m.nn[0], NY = m.nn[1];

  uint32_t stage_use[T2_STAGES] = {0, 0, 0};  // completed uses per stage (parity source)
  uint32_t acc_use[2] = {0, 0};
  int chunk_it = 0;
  bool ok = true;
  int64_t prev_item = -1;
  int prev_buf = 0, it = 0;

  auto epilogue = [&](int64_t item, int buf) {
    // wait for the accumulator, then scatter-add row r = TMEM lane r
    if (!wait_parity(acc_full + buf, acc_use[buf] & 1u)) ok = false;
    acc_use[buf]++;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int tile = (int)(item % ntiles);
    const int c0 = tile * T2_TW;
    const int ncol = min(n_mma, N - c0);
    const int quarter = warp & 3;           // TMEM lanes 32*quarter .. +31
    const int r = quarter * 32 + lane;
    const int64_t g = (r < NL) ? gnode[buf * 128 + r] : 0;
    for (int cb = (warp >> 2) * 16; cb < ncol; cb += (T2_THREADS / 128) * 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 256 + cb))
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < NL) {
        float* wr = W + g * ldw + c0 + cb;
        if (cb + 16 <= ncol && ((ldw | (int64_t)c0 | cb) & 3) == 0) {
          float4* w4 = reinterpret_cast<float4*>(wr);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float4 o = w4[q];
            o.x += __uint_as_float(v[4 * q]);
            o.y += __uint_as_float(v[4 * q + 1]);
            o.z += __uint_as_float(v[4 * q + 2]);
            o.w += __uint_as_float(v[4 * q + 3]);
            w4[q] = o;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (cb + q < ncol) wr[q] += __uint_as_float(v[q]);
        }
      }
    }
  };

  const int64_t nitems = ncells * ntiles;
  for (int64_t item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++it) {
    const int buf = it & 1;
    const int64_t e = cells[item / ntiles];
    const int tile = (int)(item % ntiles);
    const int c0 = tile * T2_TW;
    const int ncol = min(n_mma, N - c0);
    const int ncol_mma = ((ncol + 15) / 16) * 16;
    // node ids of this cell into slot buf (the epilogue of the cell that used
    // this slot two items ago has finished: program order + barrier below)
    if (tid < NL) {
      const int i = (int)(e % m.nc[0]), j = (int)((e / m.nc[0]) % m.nc[1]),
                k = (int)(e / ((int64_t)m.nc[0] * m.nc[1]));
      const int a = tid % NP1, b = (tid / NP1) % NP1, c = tid / (NP1 * NP1);
      gnode[buf * 128 + tid] = (int64_t)(P * i + a) + NX * ((int64_t)(P * j + b) + NY * (int64_t)(P * k + c));
    }
    __syncthreads();
    for (int kc = 0; kc < T2_NCH; ++kc, ++chunk_it) {
      const int st = chunk_it % T2_STAGES;
      // stage reuse: wait until the MMAs that read it three chunks ago completed
      if (chunk_it >= T2_STAGES) {
        if (!wait_parity(stage_free + st, stage_use[st] & 1u)) ok = false;
        stage_use[st]++;
      }
      unsigned char* S = stg + st * sb;
      float* A1 = reinterpret_cast<float*>(S);
      float* A2 = reinterpret_cast<float*>(S + T2Smem::a_bytes());
      float* B1 = reinterpret_cast<float*>(S + 2 * T2Smem::a_bytes());
      float* B2 = reinterpret_cast<float*>(S + 2 * T2Smem::a_bytes() + T2Smem::b_bytes(n_mma));
      // A chunk: 16 row groups x 1 KB contiguous in the full image (SBO 4096 there)
      const float4* src = reinterpret_cast<const float4*>(Araw + e * (int64_t)(T2_M * T2_K));
      for (int v = tid; v < 16 * 64; v += T2_THREADS) {
        const int grp = v >> 6, x = v & 63;               // 64 float4 per 1 KB piece
        const float4 a = src[grp * 256 + kc * 64 + x];     // (grp*4096 + kc*1024)/16 + x
        float4 h, l;
        h.x = tf32r(a.x); h.y = tf32r(a.y); h.z = tf32r(a.z); h.w = tf32r(a.w);
        reinterpret_cast<float4*>(A1)[grp * 64 + x] = h;
        if (SPLIT) {
          l.x = tf32r(a.x - h.x); l.y = tf32r(a.y - h.y); l.z = tf32r(a.z - h.z); l.w = tf32r(a.w - h.w);
          reinterpret_cast<float4*>(A2)[grp * 64 + x] = l;
        }
      }
      // B chunk: node rows kc*32 .. +31 of the cell, columns c0 .. c0 + ncol_mma, K-major
      for (int v = tid; v < n_mma * 8; v += T2_THREADS) {
        const int n = v % n_mma, kq = v / n_mma;   // 4 consecutive k per thread
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < ncol) {
          const int kb = kc * T2_KC + kq * 4;
          float t4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            t4[q] = (kb + q < NL) ? Y[gnode[buf * 128 + kb + q] * ldy + c0 + n] : 0.f;
          y = make_float4(t4[0], t4[1], t4[2], t4[3]);
        }
        float4 h, l;
        h.x = tf32r(y.x); h.y = tf32r(y.y); h.z = tf32r(y.z); h.w = tf32r(y.w);
        *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(B1) + cm32(n, kq * 4)) = h;
        if (SPLIT) {
          l.x = tf32r(y.x - h.x); l.y = tf32r(y.y - h.y); l.z = tf32r(y.z - h.z); l.w = tf32r(y.w - h.w);
          *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(B2) + cm32(n, kq * 4)) = l;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      ok = __syncthreads_and(ok) != 0;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0 && ok) {
        const uint32_t d = tmem + (uint32_t)(buf * 256);
        const uint32_t id = idesc_tf32(ncol_mma);
        const uint32_t a1 = s_u32(A1), a2 = s_u32(A2), b1 = s_u32(B1), b2 = s_u32(B2);
        for (int ks = 0; ks < T2_KC / 8; ++ks) {
          const uint32_t off = (uint32_t)ks * 256u;
          const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
          mma_tf32(d, desc_noswz(a1 + off, 128u, 1024u), desc_noswz(b1 + off, 128u, 1024u), id, acc);
          if (SPLIT) {
            mma_tf32(d, desc_noswz(a1 + off, 128u, 1024u), desc_noswz(b2 + off, 128u, 1024u), id, 1u);
            mma_tf32(d, desc_noswz(a2 + off, 128u, 1024u), desc_noswz(b1 + off, 128u, 1024u), id, 1u);
          }
        }
        commit(stage_free + st);
        if (kc == T2_NCH - 1) commit(acc_full + buf);
      }
      (void)idesc;
    }
    // epilogue of the previous item overlaps this item's MMAs
    if (prev_item >= 0 && ok) epilogue(prev_item, prev_buf);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;
    prev_item = item;
    prev_buf = buf;
  }
  if (prev_item >= 0 && ok) epilogue(prev_item, prev_buf);
  ok = __syncthreads_and(ok) != 0;
  // drain: every commit issued must have landed before TMEM is released
  for (int st = 0; st < T2_STAGES; ++st) {
    const int issued = chunk_it > st ? (chunk_it - st + T2_STAGES - 1) / T2_STAGES : 0;
    while ((int)stage_use[st] < issued) {
      if (!wait_parity(stage_free + st, stage_use[st] & 1u)) { ok = false; break; }
      stage_use[st]++;
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T2_TMEM_COLS) : "memory");
  }
}

// FP32 image of H^cc_e in the K-major core-matrix layout (full K = 128: SBO = 4096 B).
__global__ void k_build_araw(const double* __restrict__ Hcc, int64_t n_cell, float* __restrict__ img) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_cell * T2_M * T2_K) return;
  const int64_t e = idx / (T2_M * T2_K);
  const int rk = (int)(idx % (T2_M * T2_K));
  const int r = rk / T2_K, k = rk % T2_K;
  const float v = (r < NL && k < NL) ? (float)Hcc[e * (int64_t)(NL * NL) + r * NL + k] : 0.f;
  const uint32_t off = (uint32_t)(r >> 3) * 4096u + (uint32_t)(k >> 2) * 128u + (uint32_t)(r & 7) * 16u +
                       (uint32_t)(k & 3) * 4u;
  img[e * (T2_M * T2_K) + off / 4] = v;
}

}  // namespace

void launch_build_araw(const double* Hcc, int64_t n_cell, float* img, cudaStream_t st) {
  const int64_t n = n_cell * T2_M * T2_K;
  if (n <= 0) return;
  k_build_araw<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Hcc, n_cell, img);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

int launch_cell_tc2(const float* Araw, const int32_t* cells, int64_t ncells, const MeshDev& m, const float* Y,
                    int64_t ldy, float* W, int64_t ldw, int N, bool split, int n_sm, int* err, cudaStream_t st) {
  if (ncells <= 0 || N <= 0) return 0;
  const int ntiles = (N + T2_TW - 1) / T2_TW;
  const int n_mma = N >= T2_TW ? T2_TW : ((N + 15) / 16) * 16;
  const size_t smem = T2Smem::total(n_mma);
  const int64_t items = ncells * ntiles;
  const unsigned grid = (unsigned)(items < n_sm ? items : n_sm);
  if (split) {
    cudaFuncSetAttribute(k_cell_tc2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cell_tc2<true><<<grid, T2_THREADS, smem, st>>>(Araw, cells, ncells, m, Y, ldy, W, ldw, N, n_mma, ntiles, err);
  } else {
    cudaFuncSetAttribute(k_cell_tc2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cell_tc2<false><<<grid, T2_THREADS, smem, st>>>(Araw, cells, ncells, m, Y, ldy, W, ldw, N, n_mma, ntiles, err);
  }
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}

}  // namespace efe
