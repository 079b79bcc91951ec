// tcgen05 (5th-generation tensor core) GEMM for the Kronecker-form product.
//
//   acc[m][n] = sum_k A[m][k] * B[n][k]        (A: M x K, B: N x K, both K-contiguous)
//
// computed with tcgen05.mma kind::tf32 and FP32 accumulation in tensor memory,
// in the 3xTF32 form: each FP32 operand is split into x = hi + lo with hi the
// TF32 truncation of x, and acc = A_hi B_hi + A_hi B_lo + A_lo B_hi, which
// keeps the product at FP32 accuracy (the dropped lo*lo term is ~2^-22
// relative).  One CTA of 128 threads owns 128 rows of A (one M = 128 MMA
// tile) and the whole N (<= 256 columns of tensor memory).  B (hi and lo) is
// resident in shared memory for the CTA's lifetime; A streams through in groups
// of 32-column (128-byte) chunks.  Operands are written to shared memory by
// coalesced loads in the canonical K-major 128-byte-swizzled layout (rows of
// 128 B, the 16-byte granule index XOR-ed with row % 8, 1024-byte atoms), so any
// M, N, K and any row pitch work (ragged tails are zero-filled).  The epilogue
// reads the accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31,
// i.e. tile rows) and hands each (m, n, value) to an epilogue functor.
//
// Every wait is bounded: an MMA that does not complete within the spin budget
// sets *err and the CTA still frees its tensor memory before returning.
#pragma once

#include "common.cuh"

namespace rmc {
namespace umma {

constexpr int kRows = 128;        // M tile
constexpr int kChunk = 32;        // TF32 elements per 128-byte row chunk
constexpr int kThreads = 128;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (row, k) (k < 32) inside one K-major SW128 chunk tile.
__device__ __forceinline__ uint32_t sw128_offset(int row, int k) {
  const uint32_t byte = (uint32_t)k * 4u;
  return (uint32_t)row * 128u + ((((byte >> 4) ^ (uint32_t)(row & 7)) & 7u) << 4) + (byte & 15u);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (unused for swizzled K-major; 16 B), stride byte offset (1024 B
// between 8-row atoms), descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}

// Bounded wait for the mbarrier phase `parity` to complete: true on success.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t max_spins) {
  const uint32_t a = smem_u32(mbar);
  for (uint32_t i = 0; i < max_spins; ++i) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

// Load rows [r0, r0 + nrows) x columns [32c, 32c + 32) of a K-contiguous FP32
// matrix (leading dimension ld, valid extent rows_valid x K) into hi/lo
// SW128 chunk tiles: a warp reads 8 rows at a time, one lane per element, so
// each lane keeps 8 independent coalesced loads in flight.
__device__ __forceinline__ void load_chunk_split(const float* __restrict__ src, long ld, int r0, int rows_valid,
                                                 int K, int c, int nrows, unsigned char* hi_tile,
                                                 unsigned char* lo_tile) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int k = c * kChunk + lane;
  for (int rb = warp * 8; rb < nrows; rb += nw * 8) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = rb + i, gr = r0 + r;
      x[i] = (r < nrows && gr < rows_valid && k < K) ? __ldg(src + (long)gr * ld + k) : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = rb + i;
      if (r < nrows) {
        float h, l;
        split_tf32(x[i], h, l);
        const uint32_t off = sw128_offset(r, lane);
        *(float*)(hi_tile + off) = h;
        *(float*)(lo_tile + off) = l;
      }
    }
  }
}

struct GemmArgs {
  const float* A;
  long lda;
  int M;
  const float* B;
  long ldb;
  int N;      // valid columns
  int Npad;   // multiple of 16, <= 256
  int K;
  int group;  // A chunks per shared-memory group
  int* err;
};

__host__ __device__ inline int tmem_cols_for(int Npad) {
  int c = 32;
  while (c < Npad) c <<= 1;
  return c;
}

inline size_t smem_bytes_for(int Npad, int K, int group) {
  const int kc = (K + kChunk - 1) / kChunk;
  return 1024 /* alignment slack */ + 2 * (size_t)kc * Npad * 128 + 2 * (size_t)group * kRows * 128;
}

constexpr size_t kSmemLimit = 232448 - 256;  // opt-in shared memory per CTA, less the static part

// Launch plan for acc = A B^T with N columns and K contraction: false when the
// shape does not fit one CTA's tensor memory / shared memory (then the caller
// uses the SIMT path).
inline bool plan(int N, int K, int* Npad, int* group, size_t* smem) {
  *Npad = (N + 15) / 16 * 16;
  if (*Npad > 256 || K < 1) return false;
  const int kc = (K + kChunk - 1) / kChunk;
  const size_t bbytes = 2 * (size_t)kc * (*Npad) * 128;
  if (1024 + bbytes + 2 * (size_t)kRows * 128 > kSmemLimit) return false;
  int g = (int)((kSmemLimit - 1024 - bbytes) / (2 * (size_t)kRows * 128));
  *group = g < kc ? g : kc;
  *smem = smem_bytes_for(*Npad, K, *group);
  return true;
}

template <class Epi>
__global__ void __launch_bounds__(kThreads, 1) gemm_tf32x3_kernel(GemmArgs g, Epi epi) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int kc = (g.K + kChunk - 1) / kChunk;
  const size_t btile = (size_t)g.Npad * 128;
  unsigned char* Bhi = base;
  unsigned char* Blo = base + kc * btile;
  unsigned char* Ahi = base + 2 * kc * btile;
  unsigned char* Alo = Ahi + (size_t)g.group * kRows * 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t ncols = (uint32_t)tmem_cols_for(g.Npad);

  if (warp == 0) tmem_alloc(&tmem_base, ncols);
  if (threadIdx.x == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B: resident hi/lo chunk tiles
  for (int c = 0; c < kc; ++c) load_chunk_split(g.B, g.ldb, 0, g.N, g.K, c, g.Npad, Bhi + c * btile, Blo + c * btile);
  fence_proxy_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_tf32(kRows, g.Npad);
  uint32_t phase = 0;
  bool ok = true;
  const int tiles = (g.M + kRows - 1) / kRows;

  for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
    const int m0 = t * kRows;
    for (int c0 = 0; c0 < kc && ok; c0 += g.group) {
      const int cn = min(g.group, kc - c0);
      for (int c = 0; c < cn; ++c)
        load_chunk_split(g.A, g.lda, m0, g.M, g.K, c0 + c, kRows, Ahi + (size_t)c * kRows * 128,
                         Alo + (size_t)c * kRows * 128);
      fence_proxy_async_smem();
      fence_before_sync();
      __syncthreads();
      fence_after_sync();
      if (threadIdx.x == 0) {
        for (int c = 0; c < cn; ++c) {
          const uint32_t ah = smem_u32(Ahi + (size_t)c * kRows * 128), al = smem_u32(Alo + (size_t)c * kRows * 128);
          const uint32_t bh = smem_u32(Bhi + (size_t)(c0 + c) * btile), bl = smem_u32(Blo + (size_t)(c0 + c) * btile);
#pragma unroll
          for (int kk = 0; kk < kChunk / 8; ++kk) {  // K = 8 per tf32 MMA: 32 bytes
            const uint32_t o = kk * 32;
            const uint32_t first = (c0 == 0 && c == 0 && kk == 0) ? 0u : 1u;
            mma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, first ? 1u : 0u);
            mma_tf32(tmem, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
            mma_tf32(tmem, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
          }
        }
        mma_commit(&mbar);
      }
      // every thread waits for the MMAs (they read this group's A tiles); the
      // threads start waiting at different times, so the outcome is combined
      // over the block before anyone acts on it: every thread then takes the
      // same branch and meets the same barriers
      const bool done = mbar_wait(&mbar, phase, 1u << 24);
      phase ^= 1u;
      fence_after_sync();
      if (!__syncthreads_and(done ? 1 : 0)) {
        if (threadIdx.x == 0 && g.err) atomicExch(g.err, 1);
        ok = false;
      }
    }
    if (!ok) break;
    // epilogue: warp w reads accumulator lanes 32w .. 32w + 31
    const int row = m0 + warp * 32 + lane;
    for (int cc = 0; cc < g.Npad; cc += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cc, v);
      if (row < g.M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = cc + j;
          if (n < g.N) epi(0, 0, row, n, v[j]);
        }
      }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  // a timed-out MMA may still write tensor memory: give it a last bounded
  // chance to land before the allocation is released
  if (!ok) mbar_wait(&mbar, phase ^ 1u, 1u << 20);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

}  // namespace umma
}  // namespace rmc
