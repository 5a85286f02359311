// Tensor-core Galerkin assembly: G_a = U^T diag(Omega_a) U for every injection
// a (the coefficient matrices of the data term of Eq. Proj_Sylv), with BF16
// operands and float32 accumulation in tensor memory (tcgen05).
//
// U (n x j, j <= 128) is kept as two BF16 shadows, U = U_hi + U_lo + O(2^-17 |U|).
// Each CTA owns one injection a and a range of 64-voxel K-blocks:
//   * TMA loads the 128 x 64 tiles of U_hi and U_lo (128-byte swizzled,
//     K-major: the canonical tcgen05 operand layout) into shared memory;
//   * A = diag(Omega_a)-masked copy of the tiles.  Omega_a is 1 except on the
//     injection site, so most K-blocks need no mask and A reuses the B tiles;
//     blocks that hold masked voxels get a masked copy written in shared memory
//     (swizzle-aware) and published to the tensor core with fence.proxy.async;
//   * one thread issues, per 16-wide K step, three MMAs hi*hi + hi*lo + lo*hi
//     (M = N = 128) into one float32 accumulator in tensor memory, and commits
//     them to an mbarrier;
//   * the epilogue reads the accumulator with tcgen05.ld (each warp its 32
//     lanes) and writes the CTA's partial sum; a second kernel adds the
//     K-range partials in a fixed order.
// Every mbarrier wait is bounded; on timeout the kernel records an error word,
// waits (bounded) for its own MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstring>

#include "cr_common.cuh"

namespace cr {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTileRows = 128;  // M = N
constexpr int kKBlock = 64;     // voxels per K-block (128 bytes of BF16)
constexpr int kTileBytes = kTileRows * kKBlock * 2;  // 16 KB
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr uint64_t kWaitNs = 500000000ull;  // 0.5 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row
// groups 1024 bytes apart; start address in 16-byte units.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);        // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)2 << 61;                        // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 A and B (K-major), float32 D, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase with parity `parity` to complete; false on timeout.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// at most kSpinLimit polls and kWaitNs of wall-clock time (a poll may suspend the thread)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t spin = 0; spin < kSpinLimit; ++spin) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) break;
  }
  return false;
}

// The first timeout wins: site (1 = tiles loaded, 2 = MMAs done) * 100000 + K-block + 1.
__device__ __forceinline__ void record_timeout(int* err, int site, int kb) {
  atomicCAS(err, 0, site * 100000 + kb + 1);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// byte offset of element (row, k) in a 128 x 64 BF16 tile, 128-byte swizzle
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ (row & 7)) << 4) | ((k & 7) << 1)));
}

struct TcArgs {
  int n, j, m, kb_per_cta, nkb;
  const uint8_t* Om;  // n x m (ld ldo)
  int64_t ldo;
  float* part;        // [splits][m][128][128]
  int* err;
};

__global__ void __launch_bounds__(kTcThreads, 1)
    galerkin_assemble_tc_kernel(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                                const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  // 1024-byte aligned tiles: B_hi, B_lo, A_hi, A_lo
  unsigned char* base = (unsigned char*)(((uintptr_t)tsm + 1023) & ~(uintptr_t)1023);
  unsigned char* Bhi = base;
  unsigned char* Blo = base + kTileBytes;
  unsigned char* Ahi = base + 2 * kTileBytes;
  unsigned char* Alo = base + 3 * kTileBytes;
  __shared__ __align__(8) uint64_t bar_full, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int masked_block;
  __shared__ int failed;

  const int alpha = blockIdx.x;
  const int split = blockIdx.y;
  const int kb0 = split * a.kb_per_cta;
  const int kb1 = min(a.nkb, kb0 + a.kb_per_cta);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bfull = smem_u32(&bar_full), bmma = smem_u32(&bar_mma);

  if (threadIdx.x == 0) {
    mbar_init(bfull, 1);
    mbar_init(bmma, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(128u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t dtm = tmem_base;
  const uint32_t idesc = idesc_bf16_f32(kTileRows, kTileRows);
  uint32_t phase = 0;
  bool issued = false;

  for (int kb = kb0; kb < kb1 && !failed; ++kb) {
    const int v0 = kb * kKBlock;
    if (threadIdx.x == 0) {
      mbar_expect_tx(bfull, 2u * kTileBytes);
      tma_load_2d(smem_u32(Bhi), &map_hi, v0, 0, bfull);
      tma_load_2d(smem_u32(Blo), &map_lo, v0, 0, bfull);
    }
    // does this K-block hold a voxel outside Omega_a?
    if (threadIdx.x == 0) masked_block = 0;
    __syncthreads();
    if (threadIdx.x < kKBlock) {
      const int i = v0 + threadIdx.x;
      if (i < a.n && a.Om[i + (int64_t)alpha * a.ldo] == 0) masked_block = 1;
    }
    if (!mbar_wait(bfull, phase)) {
      record_timeout(a.err, 1, kb);
      failed = 1;
    }
    __syncthreads();
    if (failed) break;
    const int mb = masked_block;
    if (mb) {
      // A = B with the masked voxels' K-columns zeroed (every row)
      for (int t = threadIdx.x; t < kTileRows * kKBlock; t += blockDim.x) {
        const int row = t >> 6, k = t & 63;
        const int i = v0 + k;
        const bool keep = i < a.n && a.Om[i + (int64_t)alpha * a.ldo] != 0;
        const uint32_t off = sw128_off(row, k);
        const __nv_bfloat16 zero = __float2bfloat16(0.f);
        *(__nv_bfloat16*)(Ahi + off) = keep ? *(const __nv_bfloat16*)(Bhi + off) : zero;
        *(__nv_bfloat16*)(Alo + off) = keep ? *(const __nv_bfloat16*)(Blo + off) : zero;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ahi = smem_u32(mb ? Ahi : Bhi), alo = smem_u32(mb ? Alo : Blo);
      const uint32_t bhi = smem_u32(Bhi), blo = smem_u32(Blo);
#pragma unroll
      for (int ks = 0; ks < kKBlock / 16; ++ks) {
        const uint32_t koff = ks * 32;  // 16 BF16 = 32 bytes along K inside the swizzle atom
        const uint32_t acc = (kb > kb0 || ks > 0) ? 1u : 0u;
        mma_bf16(dtm, smem_desc_sw128(ahi + koff), smem_desc_sw128(bhi + koff), idesc, acc);
        mma_bf16(dtm, smem_desc_sw128(ahi + koff), smem_desc_sw128(blo + koff), idesc, 1u);
        mma_bf16(dtm, smem_desc_sw128(alo + koff), smem_desc_sw128(bhi + koff), idesc, 1u);
      }
      mma_commit(bmma);
    }
    issued = true;
    // the next TMA / masked copy overwrites the tiles: wait for these MMAs
    if (!mbar_wait(bmma, phase)) {
      record_timeout(a.err, 2, kb);
      failed = 1;
    }
    __syncthreads();
    phase ^= 1;
  }

  // epilogue: warp w owns accumulator lanes [32w, 32w + 32)
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float* out = a.part + ((int64_t)split * a.m + alpha) * kTileRows * kTileRows;
  const int row = warp * 32 + lane;
  if (!failed && issued) {
#pragma unroll
    for (int c0 = 0; c0 < kTileRows; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = dtm + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int q = 0; q < 32; ++q) out[(int64_t)row + (int64_t)(c0 + q) * kTileRows] = __uint_as_float(r[q]);
    }
  } else {
    for (int q = 0; q < kTileRows; ++q) out[(int64_t)row + (int64_t)q * kTileRows] = 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtm), "r"(128u) : "memory");
  }
}

// fG[a](p, q) = sum_s part[s][a](p, q), p, q < j (fixed order)
__global__ void assemble_reduce_kernel(int splits, int j, int m, const float* __restrict__ part, float* __restrict__ G,
                                       int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)m * j * j;
  if (t >= tot) return;
  const int a = (int)(t / ((int64_t)j * j));
  const int r = (int)(t % ((int64_t)j * j));
  const int p = r % j, q = r / j;
  float s = 0.f;
  for (int sp = 0; sp < splits; ++sp) s += part[(((int64_t)sp * m + a) * kTileRows + q) * kTileRows + p];
  G[(int64_t)a * ld * ld + p + (int64_t)q * ld] = s;
}

__global__ void split_bf16_kernel(int n, int cols, const double* __restrict__ U, int64_t ldu, __nv_bfloat16* hi,
                                  __nv_bfloat16* lo, int64_t ldb) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * cols) return;
  const int64_t i = t % n, c = t / n;
  const float u = (float)U[i + c * ldu];
  const __nv_bfloat16 h = __float2bfloat16_rn(u);
  hi[i + c * ldb] = h;
  lo[i + c * ldb] = __float2bfloat16_rn(u - __bfloat162float(h));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn lookup_encode() {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  EncodeTiledFn fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    fn = (EncodeTiledFn)p;
  cudaGetLastError();
  return fn;
}

// looked up once (thread-safe static initialisation: problems may be driven from several threads)
EncodeTiledFn get_encode() {
  static const EncodeTiledFn fn = lookup_encode();
  return fn;
}

}  // namespace

size_t tc_part_elems(int splits, int m) { return (size_t)splits * m * kTileRows * kTileRows; }

// BF16 hi/lo shadows of U's first `cols` columns (U with column stride ldu).
void bf16_split(int n, int cols, const double* U, int64_t ldu, void* hi, void* lo, int64_t ldb, cudaStream_t st) {
  const int64_t tot = (int64_t)n * cols;
  if (tot <= 0) return;
  count_launch();
  split_bf16_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, cols, U, ldu, (__nv_bfloat16*)hi,
                                                                      (__nv_bfloat16*)lo, ldb);
}

// G(float32, m blocks of ld x ld) = U^T diag(Omega_a) U for j <= 128 from the
// BF16 shadows hi/lo (n x 128, column stride ldb elements, ldb a multiple of
// 64, columns >= j zero).  part must hold tc_part_elems(splits, m) floats.
cudaError_t galerkin_assemble_tc(int n, int j, int m, const void* hi, const void* lo, int64_t ldb, const uint8_t* Om,
                                 int64_t ldo, int splits, float* part, float* G, int64_t ld, int* err, cudaStream_t st) {
  if (j < 1 || j > kTileRows || (ldb % 64) != 0) return cudaErrorNotSupported;
  EncodeTiledFn enc = get_encode();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap mh, ml;
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)kTileRows};
  const cuuint64_t strides[1] = {(cuuint64_t)ldb * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kKBlock, (cuuint32_t)kTileRows};
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(hi), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  if (enc(&ml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(lo), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int nkb = (n + kKBlock - 1) / kKBlock;
  if (splits < 1) splits = 1;
  if (splits > nkb) splits = nkb;
  TcArgs a{};
  a.n = n;
  a.j = j;
  a.m = m;
  a.nkb = nkb;
  a.kb_per_cta = (nkb + splits - 1) / splits;
  splits = (nkb + a.kb_per_cta - 1) / a.kb_per_cta;
  a.Om = Om;
  a.ldo = ldo;
  a.part = part;
  a.err = err;
  const size_t smem = 4 * (size_t)kTileBytes + 1024;
  cudaError_t e = cudaFuncSetAttribute(galerkin_assemble_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  count_launch();
  galerkin_assemble_tc_kernel<<<dim3(m, splits), kTcThreads, smem, st>>>(mh, ml, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tot = (int64_t)m * j * j;
  count_launch();
  assemble_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(splits, j, m, part, G, ld);
  return cudaGetLastError();
}

}  // namespace cr
