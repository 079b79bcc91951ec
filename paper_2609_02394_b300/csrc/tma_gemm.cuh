// TMA-fed, pipelined tcgen05 GEMM for the two stages of the Kronecker-form
// product (Eq. (7)) in 3xTF32:
//
//   acc[m][n] = sum_k A[m][k] * B[n][k]        (A: M x K, B: N x K, K-contiguous)
//
// Each FP32 operand x is used as x_hi = the TF32 truncation the tensor core
// applies to the raw FP32 word, plus x_lo = x - x_hi (exact in FP32), and
// acc = A_hi B_hi + A_hi B_lo + A_lo B_hi on tcgen05.mma kind::tf32 with FP32
// accumulation in tensor memory (the dropped lo*lo term is ~2^-22 relative).
//
// One persistent CTA per SM walks output tiles of 128 x BN (BN <= 256, a
// multiple of 16) with warp-specialised roles:
//   warp 0     TMA producer: cp.async.bulk.tensor.2d loads of the raw A and B
//              row chunks (32 floats = 128 B of K per row) into a stage,
//              completing on the stage's `full` mbarrier (expect_tx bytes);
//   warp 1     tensor-memory allocation and the MMA issuer (one thread): three
//              MMAs per K = 8 step, tcgen05.commit to the stage's `empty`
//              barrier and, after a tile's last chunk, to the accumulator's
//              `accf` barrier;
//   warps 2-5  converters: form the lo parts of both tiles of a stage in
//              shared memory (same swizzled layout, elementwise), fence them
//              to the async proxy and arrive on the stage's `conv` barrier;
//   warps 6-9  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//              lanes 32 (w % 4) .. + 31, i.e. tile rows), then free the
//              accumulator buffer (`acce`).  Where the functor maps the warp's
//              32 rows x 32 columns onto a 32 x 32 block of a 2-D output
//              (block_xy), the final values (values) go transposed into a
//              shared-memory staging block and out with one TMA tensor store
//              (two staging blocks a warp, bulk groups waited on before a
//              block is reused and before exit); otherwise each run of 32
//              consecutive columns of a row goes to the functor's
//              run(m, n0, values, count).
// The accumulator is double-buffered (2 x 256 TMEM columns), so the epilogue of
// one tile overlaps the MMAs of the next; the K chunks run through a ring of
// kStages stages (2 for 256-column tiles, 3 for tiles of <= 128 columns, the
// most that fit shared memory), so the TMA loads and conversions of the next
// chunks overlap the MMAs of the current one.
//
// Shared-memory layout: the TMA writes each box in the canonical K-major
// 128-byte-swizzled layout (rows of 128 B, 16-byte granule index XOR row % 8,
// 1024-byte atoms), which is the layout the sdesc_sw128 descriptors describe.
// Ragged M, N and K tails are zero-filled by the TMA (out-of-bounds box
// elements), and the epilogue skips rows >= M and columns >= N.
//
// Requirements (checked by the host): A and B 16-byte aligned, row pitches
// (in floats) multiples of 4 (TMA strides are multiples of 16 bytes), K >= 1.
// Every K-chunk coordinate is a multiple of 32 floats, so each TMA box starts
// on a 16-byte boundary.
//
// Every wait is bounded (kSpin polls).  A role that gives up raises the
// kernel's error flag and leaves its loop; the others then give up too at
// their own bounded waits (the whole-warp roles decide as a warp).  Before the tensor memory is released the MMA
// thread waits (bounded) for its last MMAs and the producer for its last
// loads, so no asynchronous write outlives the CTA.
#pragma once

#include <cuda.h>

#include "umma.cuh"

namespace rmc {
namespace tmag {

using umma::fence_after_sync;
using umma::fence_before_sync;
using umma::fence_proxy_async_smem;
using umma::idesc_tf32;
using umma::mbar_init;
using umma::mbar_wait;
using umma::mma_commit;
using umma::mma_tf32;
using umma::sdesc_sw128;
using umma::smem_u32;
using umma::tmem_ld32;

constexpr int kBM = 128;        // rows of an output tile (one M = 128 MMA)
constexpr int kMaxStages = 3;   // K-chunk pipeline depth: 3 for N tiles <= 128, else 2
constexpr int kWarps = 10;
constexpr int kThreads = kWarps * 32;
constexpr int kConvWarp0 = 2;   // warps 2..5
constexpr int kEpiWarp0 = 6;    // warps 6..9
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kSpin = 1u << 22;
constexpr uint32_t kABytes = kBM * 128;  // one A stage tile (hi or lo)

struct Args {
  int M, N, K;
  int BN;        // N tile, multiple of 16, <= 256
  int m_tiles, n_tiles;
  int* err;
  int tma_store;  // 1: the epilogue writes 32 x 32 output blocks with TMA stores (mapO)
  int k_splits;   // K split into k_splits ranges of kc_split 32-wide chunks (split-K);
  int kc_split;   // each (tile, split) accumulates one range and hands the split index on
};

constexpr uint32_t kStageBlock = 32 * 32 * 4;    // one 32 x 32 FP32 output block
constexpr uint32_t kStoreBytes = 4 * 2 * kStageBlock;  // 4 epilogue warps x 2 buffers

// stages that fit 227 KB of shared memory with the hi and lo tiles of A and B
__host__ __device__ inline int stages_for(int BN) { return BN <= 128 ? 3 : 2; }

__host__ __device__ inline size_t smem_bytes(int BN, int stages) {
  return 1024 + (size_t)stages * 2 * (kABytes + (size_t)BN * 128) + kStoreBytes;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 2-D tiled TMA load of the box at (x = K offset, y = row offset) into dst,
// completing `bytes` on bar.  x is always a multiple of 32 floats.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 2-D tiled TMA store of a 32 x 32 FP32 block from shared memory (bulk group).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"((uint64_t)map),
               "r"(x), "r"(y), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one bulk group of this thread still reading shared memory
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)map) : "memory");
}

__device__ __forceinline__ float lo_part(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

__device__ __forceinline__ void lo_tile(const unsigned char* hi, unsigned char* lo, uint32_t bytes, int t) {
  const float4* h = (const float4*)hi;
  float4* l = (float4*)lo;
  for (uint32_t i = t; i < bytes / 16; i += 128) {
    const float4 v = h[i];
    l[i] = make_float4(lo_part(v.x), lo_part(v.y), lo_part(v.z), lo_part(v.w));
  }
}

template <int kStages, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tma_tf32x3_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                           const __grid_constant__ CUtensorMap mapO, Args g, Epi epi) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full[kStages], conv[kStages], empty[kStages], accf[2], acce[2], last;
  __shared__ uint32_t tmem_base;
  __shared__ int aborted;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t b_bytes = (uint32_t)g.BN * 128;
  const uint32_t stage_bytes = 2 * (kABytes + b_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles = g.m_tiles * g.n_tiles * g.k_splits;
  const int kcs_all = (g.K + 31) / 32;
  // work item t: output tile (mt, nt) and K range ks (chunks kc0 .. kc0 + count - 1)
  auto decode = [&](int t, int* mt, int* nt, int* ks, int* kc0, int* count) {
    const int mn = t / g.k_splits;
    *ks = t % g.k_splits;
    *mt = mn / g.n_tiles;
    *nt = mn % g.n_tiles;
    *kc0 = *ks * g.kc_split;
    *count = max(0, min(kcs_all - *kc0, g.kc_split));
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 4);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 4);
    }
    mbar_init(&last, 1);
    aborted = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) umma::tmem_alloc(&tmem_base, kTmemCols);
  if (warp == 0 && lane == 0) {
    prefetch_map(&mapA);
    prefetch_map(&mapB);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = tmem_base;
  auto give_up = [&]() {
    if (g.err) atomicExch(g.err, 1);
    *(volatile int*)&aborted = 1;
  };
  auto stopped = [&]() { return *(volatile int*)&aborted != 0; };
  // the whole-warp roles (converters, epilogue) take every wait decision as a
  // warp: their loops hold __syncwarp and warp-collective tcgen05.ld, so the
  // lanes must leave a loop together
  auto warp_stopped = [&]() { return __any_sync(0xffffffffu, stopped()) != 0; };
  auto warp_wait = [&](uint64_t* bar, uint32_t parity) {
    const bool ok = mbar_wait(bar, parity, kSpin) && !stopped();
    return __all_sync(0xffffffffu, ok) != 0;
  };

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      int it = 0;
      for (int t = blockIdx.x; t < tiles && !stopped(); t += gridDim.x) {
        int mt, nt, ks, kc0, kcs;
        decode(t, &mt, &nt, &ks, &kc0, &kcs);
        for (int kc = 0; kc < kcs; ++kc, ++it) {
          const int s = it % kStages;
          const uint32_t ph = (uint32_t)(it / kStages) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, kSpin) || stopped()) {
            give_up();
            break;
          }
          unsigned char* st = base + (size_t)s * stage_bytes;
          mbar_arrive_expect_tx(&full[s], kABytes + b_bytes);
          tma_load_2d(st, &mapA, (kc0 + kc) * 32, mt * kBM, &full[s]);
          tma_load_2d(st + kABytes, &mapB, (kc0 + kc) * 32, nt * g.BN, &full[s]);
        }
      }
      // the last loads of every stage have landed before the CTA may exit
      for (int j = 0; j < kStages && j < it; ++j) {
        const int i2 = it - 1 - j;
        mbar_wait(&full[i2 % kStages], (uint32_t)(i2 / kStages) & 1u, kSpin);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(kBM, g.BN);
      int it = 0, tc = 0;
      for (int t = blockIdx.x; t < tiles && !stopped(); t += gridDim.x, ++tc) {
        int mt, nt, ks, kc0, kcs;
        decode(t, &mt, &nt, &ks, &kc0, &kcs);
        const int ab = tc & 1;
        if (!mbar_wait(&acce[ab], ((uint32_t)(tc >> 1) & 1u) ^ 1u, kSpin)) {
          give_up();
          break;
        }
        fence_after_sync();
        const uint32_t d = tmem + (uint32_t)ab * 256u;
        bool ok = true;
        for (int kc = 0; kc < kcs; ++kc, ++it) {
          const int s = it % kStages;
          if (!mbar_wait(&conv[s], (uint32_t)(it / kStages) & 1u, kSpin) || stopped()) {
            ok = false;
            break;
          }
          fence_after_sync();
          unsigned char* st = base + (size_t)s * stage_bytes;
          const uint32_t ah = smem_u32(st), bh = smem_u32(st + kABytes);
          const uint32_t al = smem_u32(st + kABytes + b_bytes), bl = smem_u32(st + 2 * kABytes + b_bytes);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // K = 8 per tf32 MMA: 32 bytes of the 128-byte row
            const uint32_t o = kk * 32;
            const uint32_t acc = (kc == 0 && kk == 0) ? 0u : 1u;
            mma_tf32(d, sdesc_sw128(ah + o), sdesc_sw128(bh + o), idesc, acc);
            mma_tf32(d, sdesc_sw128(ah + o), sdesc_sw128(bl + o), idesc, 1u);
            mma_tf32(d, sdesc_sw128(al + o), sdesc_sw128(bh + o), idesc, 1u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) {
          give_up();
          break;
        }
        mma_commit(&accf[ab]);
      }
      // every MMA issued has completed before the tensor memory is freed
      mma_commit(&last);
      mbar_wait(&last, 0u, kSpin);
    }
  } else if (warp < kEpiWarp0) {
    // ---- converters: lo parts of the stage's tiles ----
    const int ct = threadIdx.x - kConvWarp0 * 32;
    int it = 0;
    for (int t = blockIdx.x; t < tiles && !warp_stopped(); t += gridDim.x) {
      int mt, nt, ks, kc0, kcs;
      decode(t, &mt, &nt, &ks, &kc0, &kcs);
      bool ok = true;
      for (int kc = 0; kc < kcs; ++kc, ++it) {
        const int s = it % kStages;
        if (!warp_wait(&full[s], (uint32_t)(it / kStages) & 1u)) {
          ok = false;
          break;
        }
        unsigned char* st = base + (size_t)s * stage_bytes;
        lo_tile(st, st + kABytes + b_bytes, kABytes, ct);
        lo_tile(st + kABytes, st + 2 * kABytes + b_bytes, b_bytes, ct);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[s]);
      }
      if (!ok) {
        give_up();
        break;
      }
    }
  } else {
    // ---- epilogue ----
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    // two 32 x 32 staging blocks of this warp for the TMA stores
    float* stg0 = (float*)(base + (size_t)kStages * stage_bytes + (size_t)(warp - kEpiWarp0) * 2 * kStageBlock);
    int sbuf = 0;
    int tc = 0;
    for (int t = blockIdx.x; t < tiles && !warp_stopped(); t += gridDim.x, ++tc) {
      const int ab = tc & 1;
      if (!warp_wait(&accf[ab], (uint32_t)(tc >> 1) & 1u)) {
        give_up();
        break;
      }
      fence_after_sync();
      int mt, nt, ks, kc0, kcs;
      decode(t, &mt, &nt, &ks, &kc0, &kcs);
      const int row = mt * kBM + q * 32 + lane;
      const int n0 = nt * g.BN;
      for (int cc = 0; cc < g.BN; cc += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)ab * 256u + (uint32_t)cc, v);
        const int cnt = min(32, min(g.BN - cc, g.N - (n0 + cc)));
        int bx = 0, by = 0;
        const int row0 = mt * kBM + q * 32;
        if (g.tma_store && cnt == 32 && row0 + 31 < g.M && epi.block_xy(ks, row0, n0 + cc, &bx, &by)) {
          // the warp's 32 x 32 block: final values, transposed into shared
          // memory (row r of the block = output column n0 + cc + r, lanes
          // along the block's inner dimension), one TMA store
          float o[32];
          epi.values(ks, row, n0 + cc, v, o);
          float* stg = stg0 + sbuf * 1024;
          if (lane == 0) bulk_wait_read_1();  // the store that used this buffer has read it
          __syncwarp();
#pragma unroll
          for (int r = 0; r < 32; ++r) stg[r * 32 + lane] = o[r];
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&mapO, bx, by, stg);
            bulk_commit();
          }
          sbuf ^= 1;
        } else if (row < g.M && cnt > 0) {
          epi.run(ks, row, n0 + cc, v, cnt);
        }
      }
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[ab]);
    }
    if (lane == 0) bulk_wait_all();  // every TMA store of this warp has completed
    __syncwarp();
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 1) umma::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace tmag
}  // namespace rmc
