// Classical cell products on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Paper, Sec. V (last paragraph): the Hamiltonian is applied matrix-free, cell
// by cell -- W_c(e) += H^cc_e Y_c(e) with H^cc_e the 125 x 125 elemental block
// of Eq. Hcc -- followed by assembly.  Here each cell product is one
// M = 128 (125 rows padded), K = 128 (125 padded), N = N_mma tensor-core GEMM:
//
//   A = H^cc_e   TF32 or BF16, pre-arranged once per potential (set_potential)
//                as the exact shared-memory image of the K-major, no-swizzle
//                canonical layout (8-row x 16-byte core matrices), copied in
//                with 16-byte vector loads;
//   B = Y_e      the cell's 125 node rows x N columns, gathered by all threads
//                and written K-major (N rows x K) in the same core-matrix layout;
//   D            FP32 accumulator in tensor memory (TMEM), N_mma columns;
//
// one elected thread issues the K/k_step tcgen05.mma instructions and commits
// them to an mbarrier; every thread waits (bounded spin), reads its TMEM lane
// (one row of D) with tcgen05.ld and adds the row to W.  Cells of one parity
// colour share no node, so the scatter needs no atomics and the result is
// bitwise reproducible.
#include <cuda_bf16.h>
#include <stdint.h>

#include "efe_kernels.h"

namespace efe {

namespace {

constexpr int TC_M = 128;       // MMA rows (125 padded)
constexpr int TC_K = 128;       // reduction length (125 padded)
constexpr uint32_t SPIN_LIMIT = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row, k) in the K-major no-swizzle core-matrix layout
// with 16-byte K chunks of `epc` elements: core matrix = 8 rows x 16 bytes
// (128 contiguous bytes); LBO = 128 (next K chunk), SBO = (K / epc) * 128
// (next 8-row group).
__host__ __device__ __forceinline__ uint32_t cm_offset(int row, int k, int epc, int esize) {
  const uint32_t sbo = (uint32_t)(TC_K / epc) * 128u;
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k / epc) * 128u + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k % epc) * (uint32_t)esize;
}

// tcgen05 shared-memory matrix descriptor: start, LBO, SBO (all >> 4),
// version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D = F32, A/B format code `fmt` (TF32 = 2 under
// kind::tf32, BF16 = 1 under kind::f16), both K-major, N and M fields.
__host__ __device__ __forceinline__ uint32_t make_idesc(int fmt, int n_mma) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n_mma >> 3) << 17) |
         ((uint32_t)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < SPIN_LIMIT; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename T>
struct TcTraits;
template <>
struct TcTraits<float> {
  static constexpr int esize = 4, epc = 4, kstep = 8, fmt = 2;  // kind::tf32
};
template <>
struct TcTraits<__nv_bfloat16> {
  static constexpr int esize = 2, epc = 8, kstep = 16, fmt = 1;  // kind::f16 with BF16 inputs
};

__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <typename T>
__device__ __forceinline__ T to_op(float x);
template <>
__device__ __forceinline__ float to_op<float>(float x) { return round_tf32(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_op<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename T>
__device__ __forceinline__ void issue_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc) {
  if constexpr (sizeof(T) == 4) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  }
}

// One CTA (128 threads) per (cell of one colour, tile of up to 256 columns).
// Vector block Y / W stored in S (float or bf16) with leading dimension ld.
template <typename T, typename S>
__global__ void __launch_bounds__(128, 1) k_cell_tc(const T* __restrict__ Aimg, const int32_t* __restrict__ cells,
                                                    MeshDev m, const S* __restrict__ Y, int64_t ldy,
                                                    S* __restrict__ W, int64_t ldw, int N, int n_mma,
                                                    int tmem_cols, int* __restrict__ err) {
  using TR = TcTraits<T>;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t e = cells[blockIdx.x];
  const int c0 = blockIdx.y * 256;
  const int ncols = min(n_mma, ((N - c0 + 15) / 16) * 16);
  // shared-memory carve-up
  const uint32_t a_bytes = (uint32_t)TC_M * TC_K * TR::esize;
  unsigned char* sA = smem;
  unsigned char* sB = smem + a_bytes;
  const uint32_t b_bytes = (uint32_t)n_mma * TC_K * TR::esize;
  int64_t* gnode = reinterpret_cast<int64_t*>(sB + b_bytes);
  uint64_t* bar = reinterpret_cast<uint64_t*>(gnode + 128);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);

  // TMEM allocation (one warp) and barrier initialisation
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // node ids of the cell
  const int i = (int)(e % m.nc[0]), j = (int)((e / m.nc[0]) % m.nc[1]), k = (int)(e / ((int64_t)m.nc[0] * m.nc[1]));
  const int64_t NX = m.nn[0], NY = m.nn[1];
  if (tid < NL) {
    const int a = tid % NP1, b = (tid / NP1) % NP1, c = tid / (NP1 * NP1);
    gnode[tid] = (int64_t)(P * i + a) + NX * ((int64_t)(P * j + b) + NY * (int64_t)(P * k + c));
  }
  // A: copy the pre-arranged image (16-byte vectors)
  {
    const uint4* src = reinterpret_cast<const uint4*>(Aimg + e * (int64_t)(TC_M * TC_K));
    uint4* dst = reinterpret_cast<uint4*>(sA);
    for (uint32_t v = tid; v < a_bytes / 16; v += blockDim.x) dst[v] = src[v];
  }
  __syncthreads();
  // B: gather Y rows of the cell, column tile [c0, c0 + ncols), written K-major
  {
    T* sBt = reinterpret_cast<T*>(sB);
    const int total = TC_K * n_mma;
    for (int idx = tid; idx < total; idx += blockDim.x) {
      const int kk = idx / n_mma, n = idx % n_mma;  // consecutive threads: consecutive columns
      float v = 0.f;
      if (kk < NL && n < ncols && c0 + n < N) v = (float)Y[gnode[kk] * ldy + c0 + n];
      sBt[cm_offset(n, kk, TR::epc, TR::esize) / TR::esize] = to_op<T>(v);
    }
  }
  // make generic-proxy smem writes visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    const uint32_t sbo = (uint32_t)(TC_K / TR::epc) * 128u;
    const uint32_t idesc = make_idesc(TR::fmt, ncols);
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
    for (int ks = 0; ks < TC_K / TR::kstep; ++ks) {
      // one MMA spans two 16-byte K chunks: advance by 2 core matrices (256 bytes)
      const uint32_t off = (uint32_t)ks * 256u;
      issue_mma<T>(tmem, make_desc(a0 + off, 128u, sbo), make_desc(b0 + off, 128u, sbo), idesc, ks > 0 ? 1u : 0u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
  }
  const bool ok = mbar_wait(bar, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    // epilogue: warp w owns TMEM lanes 32w..32w+31 = rows of D
    const int r = warp * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int cb = 0; cb < ncols; cb += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr + (uint32_t)cb)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < NL) {
        S* wr = W + gnode[r] * ldw + c0 + cb;
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (c0 + cb + q < N) wr[q] = (S)((float)wr[q] + __uint_as_float(v[q]));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

// A images: H^cc_e (FP64, 125 x 125 row-major) -> 128 x 128 TF32/BF16 core-matrix layout.
template <typename T>
__global__ void k_build_aimg(const double* __restrict__ Hcc, int64_t n_cell, T* __restrict__ img) {
  using TR = TcTraits<T>;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_cell * TC_M * TC_K) return;
  const int64_t e = idx / (TC_M * TC_K);
  const int rk = (int)(idx % (TC_M * TC_K));
  const int r = rk / TC_K, kk = rk % TC_K;
  const float v = (r < NL && kk < NL) ? (float)Hcc[e * (int64_t)(NL * NL) + r * NL + kk] : 0.f;
  img[e * (TC_M * TC_K) + cm_offset(r, kk, TR::epc, TR::esize) / TR::esize] = to_op<T>(v);
}

template <typename T, typename S>
size_t tc_smem_bytes(int n_mma) {
  return (size_t)TC_M * TC_K * TcTraits<T>::esize + (size_t)n_mma * TC_K * TcTraits<T>::esize + 128 * 8 + 64;
}

}  // namespace

int64_t tc_image_elems(int64_t n_cell) { return n_cell * TC_M * TC_K; }

void launch_build_aimg_tf32(const double* Hcc, int64_t n_cell, float* img, cudaStream_t st) {
  const int64_t n = n_cell * TC_M * TC_K;
  k_build_aimg<float><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Hcc, n_cell, img);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

void launch_build_aimg_bf16(const double* Hcc, int64_t n_cell, void* img, cudaStream_t st) {
  const int64_t n = n_cell * TC_M * TC_K;
  k_build_aimg<__nv_bfloat16><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(Hcc, n_cell, (__nv_bfloat16*)img);
  g_launches.fetch_add(1, std::memory_order_relaxed);
}

// W += H_e Y_e on tcgen05, TF32 operands, FP32 vectors.
int launch_cell_tc_tf32(const float* Aimg, const int32_t* cells, int64_t ncells, const MeshDev& m, const float* Y,
                        int64_t ldy, float* W, int64_t ldw, int N, int* err, cudaStream_t st) {
  if (ncells <= 0 || N <= 0) return 0;
  const int n_mma = N >= 256 ? 256 : ((N + 15) / 16) * 16;
  const int tmem_cols = n_mma <= 32 ? 32 : (n_mma <= 64 ? 64 : (n_mma <= 128 ? 128 : 256));
  const size_t smem = tc_smem_bytes<float, float>(n_mma);
  cudaFuncSetAttribute(k_cell_tc<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 g((unsigned)ncells, (unsigned)((N + 255) / 256));
  k_cell_tc<float, float><<<g, 128, smem, st>>>(Aimg, cells, m, Y, ldy, W, ldw, N, n_mma, tmem_cols, err);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}

// W += H_e Y_e on tcgen05, BF16 operands, BF16 vectors, FP32 accumulation.
int launch_cell_tc_bf16(const void* Aimg, const int32_t* cells, int64_t ncells, const MeshDev& m, const void* Y,
                        int64_t ldy, void* W, int64_t ldw, int N, int* err, cudaStream_t st) {
  if (ncells <= 0 || N <= 0) return 0;
  const int n_mma = N >= 256 ? 256 : ((N + 15) / 16) * 16;
  const int tmem_cols = n_mma <= 32 ? 32 : (n_mma <= 64 ? 64 : (n_mma <= 128 ? 128 : 256));
  const size_t smem = tc_smem_bytes<__nv_bfloat16, __nv_bfloat16>(n_mma);
  cudaFuncSetAttribute(k_cell_tc<__nv_bfloat16, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  dim3 g((unsigned)ncells, (unsigned)((N + 255) / 256));
  k_cell_tc<__nv_bfloat16, __nv_bfloat16><<<g, 128, smem, st>>>(
      (const __nv_bfloat16*)Aimg, cells, m, (const __nv_bfloat16*)Y, ldy, (__nv_bfloat16*)W, ldw, N, n_mma, tmem_cols,
      err);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return 0;
}

}  // namespace efe
