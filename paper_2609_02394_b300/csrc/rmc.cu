// Host driver and C ABI of the recursive module-coupling eigensolver.
//
// Algorithm 1 of the paper, B300-native:
//   * rmc_build_leaf[_pauli]  leaf module: dense H on the device, FP64-accurate
//                             small eigensolve, projected carried operators.
//   * rmc_couple              one merge: diagonal + start block, Chebyshev-
//                             filtered subspace iteration on the Kronecker-form
//                             product (working precision FP64 or FP32), FP64
//                             finalisation (Cholesky-QR, Rayleigh-Ritz with
//                             refined eigenvectors), degenerate cut, gauge,
//                             rotation of the carried operators.
//   * rmc_solve_chain         the recursion loop with homogeneous reuse.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <memory>
#include <set>
#include <string>
#include <tuple>
#include <thread>
#include <vector>

#include "../../include/rmc.h"
#include "common.cuh"
#include "gemm.cuh"
#include "cheb_fused.cuh"
#include "kernels.cuh"
#include "umma.cuh"
#include "tma_gemm.cuh"
#include "bounds.cuh"

using namespace rmc;

// Concurrent solves (server slots, merge lanes) each own a CUDA stream; the
// driver serves streams through CUDA_DEVICE_MAX_CONNECTIONS hardware queues
// (8 unless set) and streams that share a queue run their kernels in order, so
// a long one-CTA kernel of one solve would hold back another.  The driver
// reads the variable when the CUDA context is created: when the library is
// loaded before that, it asks for 32 queues, unless the caller set a value.
__attribute__((constructor)) static void rmc_default_connections() {
  setenv("CUDA_DEVICE_MAX_CONNECTIONS", "32", 0);
}

struct rmc_block {
  int k = 0;          // kept states
  int n_ops = 0;      // carried operators
  int rows = 0;       // basis rows (D for a leaf, kA*kB for a merge; 0 = none)
  double* E = nullptr;      // k
  double* ops = nullptr;    // n_ops * k * k
  double* basis = nullptr;  // k vectors of `rows` (vector-major)
  std::vector<rmc_op_tag> tags;
  std::vector<double> opnorm;  // upper bound of each operator's 2-norm
  size_t bytes = 0;
};

struct rmc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaMemPool_t pool = nullptr;
  bool own_pool = true;
  size_t budget = 0;
  size_t in_use = 0;
  std::map<void*, size_t> live;
  // lanes: child contexts that run merges of one level concurrently
  // (rmc_couple_batch); each has its own stream, status words and pinned
  // staging, shares this context's pool, and charges its bytes to `acct`
  rmc_ctx* acct = nullptr;  // context whose budget this one draws on (null: itself)
  std::mutex acct_mu;       // guards in_use of an accounting context
  std::vector<rmc_ctx*> lanes;
  bool native64 = false;  // set while a kernel-level entry point runs (Native64Scope)
  rmc_config cfg{};
  std::string err;
  uint64_t launches = 0, iterations = 0;
  int* d_status = nullptr;      // device scratch ints
  double* h_pinned = nullptr;   // pinned host staging (status + thetas)
  std::set<rmc_block*> blocks;
  int trace = 0;  // RMC_TRACE=1 in the environment: per-iteration convergence lines on stderr
  // opt-in per-kind timing (rmc_profile)
  unsigned prof = 0;  // bit k set: launch groups of kind k are timed
  struct Pending { cudaEvent_t a, b; int kind; uint64_t launches; double flops; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  uint64_t prof_groups[RMC_PROF_KINDS] = {};
  uint64_t prof_launches[RMC_PROF_KINDS] = {};
  double prof_ms[RMC_PROF_KINDS] = {};
  double prof_flops[RMC_PROF_KINDS] = {};
};

namespace {

constexpr size_t kPinnedDoubles = 4096;

rmc_status fail(rmc_ctx* ctx, rmc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return st;
}

#define CK(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail(ctx, RMC_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,  \
                                       cudaGetErrorString(e_));                                       \
  } while (0)
#define CKL()                                                                                         \
  do {                                                                                                \
    ctx->launches++;                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                              \
    if (e_ != cudaSuccess) return fail(ctx, RMC_ERR_CUDA, "%s:%d launch: %s", __FILE__, __LINE__,     \
                                       cudaGetErrorString(e_));                                       \
  } while (0)
#define TRY(x)                          \
  do {                                  \
    rmc_status s_ = (x);                \
    if (s_ != RMC_OK) return s_;        \
  } while (0)

rmc_status dalloc(rmc_ctx* ctx, void** p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  rmc_ctx* a = ctx->acct ? ctx->acct : ctx;
  {
    std::lock_guard<std::mutex> lk(a->acct_mu);
    if (a->in_use + bytes > a->budget)
      return fail(ctx, RMC_ERR_NOMEM, "device-memory budget exceeded: need %zu more bytes, %zu of %zu in use",
                  bytes, a->in_use, a->budget);
    a->in_use += bytes;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(a->acct_mu);
    a->in_use -= bytes;
    return fail(ctx, RMC_ERR_NOMEM, "cudaMallocFromPoolAsync(%zu): %s", bytes, cudaGetErrorString(e));
  }
  ctx->live[*p] = bytes;
  return RMC_OK;
}

void dfree(rmc_ctx* ctx, void* p) {
  if (!p) return;
  auto it = ctx->live.find(p);
  if (it != ctx->live.end()) {
    rmc_ctx* a = ctx->acct ? ctx->acct : ctx;
    std::lock_guard<std::mutex> lk(a->acct_mu);
    a->in_use -= it->second;
    ctx->live.erase(it);
  }
  cudaFreeAsync(p, ctx->stream);
}

// Scoped workspace: every allocation is released when it goes out of scope.
struct Workspace {
  rmc_ctx* ctx;
  std::vector<void*> ptrs;
  explicit Workspace(rmc_ctx* c) : ctx(c) {}
  ~Workspace() {
    for (void* p : ptrs) dfree(ctx, p);
  }
  template <typename T>
  rmc_status get(T** p, size_t count) {
    void* q = nullptr;
    TRY(dalloc(ctx, &q, count * sizeof(T)));
    ptrs.push_back(q);
    *p = (T*)q;
    return RMC_OK;
  }
};

inline unsigned grid1d(long n, int threads = 256) { return (unsigned)std::min<long>(std::max<long>(1, (n + threads - 1) / threads), 148 * 16); }

// ---------------------------------------------------------------------------
// Opt-in timing: a Scope records an event pair around a launch group.
// ---------------------------------------------------------------------------
cudaEvent_t take_event(rmc_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void harvest(rmc_ctx* ctx) {  // call after a stream synchronisation
  for (auto& p : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      ctx->prof_groups[p.kind] += 1;
      ctx->prof_launches[p.kind] += p.launches;
      ctx->prof_ms[p.kind] += ms;
      ctx->prof_flops[p.kind] += p.flops;
    }
    ctx->event_pool.push_back(p.a);
    ctx->event_pool.push_back(p.b);
  }
  ctx->pending.clear();
  cudaGetLastError();
}

struct ProfScope {
  rmc_ctx* ctx;
  int kind;
  double flops;
  uint64_t l0;
  cudaEvent_t a = nullptr;
  ProfScope(rmc_ctx* c, int k, double f) : ctx(c), kind(k), flops(f), l0(c->launches) {
    if (ctx->prof & (1u << kind)) {
      a = take_event(ctx);
      cudaEventRecord(a, ctx->stream);
    }
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = take_event(ctx);
    cudaEventRecord(b, ctx->stream);
    ctx->pending.push_back({a, b, kind, ctx->launches - l0, flops});
  }
};

// ---------------------------------------------------------------------------
// GEMM front ends on vector-major blocks (a block of nv vectors of length n is
// a row-major nv x n matrix).
// ---------------------------------------------------------------------------
template <typename T, bool TA, bool TB, class Epi>
void gemm_big(const T* A, const T* B, const GemmShape& s, int batches, const Epi& epi, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) launch_gemm<T, 64, 64, 16, 4, 4, TA, TB>(A, B, s, batches, epi, st);
  else launch_gemm<T, 64, 64, 8, 4, 4, TA, TB>(A, B, s, batches, epi, st);
}
template <typename T, bool TA, bool TB, class Epi>
void gemm_small(const T* A, const T* B, const GemmShape& s, int batches, const Epi& epi, cudaStream_t st) {
  launch_gemm<T, 16, 16, 16, 1, 1, TA, TB>(A, B, s, batches, epi, st);
}
// FP64 data, double-float products on the FP32 pipe (64 x 64 x 8 tiles)
template <bool TA, bool TB, class Epi>
void gemm_df(const double* A, const double* B, const GemmShape& s, int batches, const Epi& epi, cudaStream_t st) {
  launch_gemm<double, 64, 64, 8, 4, 4, TA, TB, Epi, true>(A, B, s, batches, epi, st);
}
// The mixed paths form their FP64-accurate block products (Gram matrices and
// basis combinations of the refinement and the rotations) in double-float;
// the FP64 path keeps native FP64.
inline bool fp64_by_df(const rmc_ctx* ctx) { return ctx->cfg.precision != RMC_PREC_FP64 && !ctx->native64; }

// Kernel-level entry points promise native FP64 for FP64 data whatever the
// context's precision: this guard holds that for the duration of a call.
struct Native64Scope {
  rmc_ctx* ctx;
  bool prev;
  explicit Native64Scope(rmc_ctx* c) : ctx(c), prev(c->native64) { c->native64 = true; }
  ~Native64Scope() { ctx->native64 = prev; }
};

// ---------------------------------------------------------------------------
// Autotuned tile shapes.  The block products of the solver (Gram matrices
// X1 X2^T over long vectors, basis combinations op(W) X) come in a handful of
// shapes per workload (b x b outputs with b = k_ret + guard, vectors of
// k_A k_B), and the best tile and split-K factor depend on them: a 64 x 64
// tile wastes 78 % of its work on a 96 x 96 Gram matrix's ragged edge, a
// 48 x 48 tile none.  Every tunable product has a short list of candidate
// launch configurations; outside tuning the table's choice for the product's
// shape bin is used (the first candidate, the untuned default, when the bin
// has no entry).  rmc_autotune runs a solve with tuning on: each product whose
// bin has no entry yet times every candidate on its own operands (CUDA events
// on the context's stream, one warm-up and three timed runs each, a
// synchronisation per candidate) and stores the fastest.  All candidates
// compute the same product; they differ in summation order only (rounding).
// The table is process-wide (every context and server slot reads it) and can
// be saved and restored as text (rmc_tune_dump / rmc_tune_load).
// ---------------------------------------------------------------------------
struct TuneTable {
  std::mutex mu;
  std::map<std::string, int> choice;
  std::atomic<int> tuning{0};  // > 0 while rmc_autotune runs
};
TuneTable& tune_table() {
  static TuneTable t;
  return t;
}

// Shape bin of a dimension: exact up to 64, then multiples of 16 up to 512,
// then the power of two above (keys stay few for the ragged k_eff of the cut).
std::string tune_bin(long d) {
  long b = d;
  if (d > 64 && d <= 512) b = (d + 15) / 16 * 16;
  else if (d > 512) { b = 1; while (b < d) b <<= 1; }
  return std::to_string(b);
}

// Runs candidate `c` (0 <= c < ncand) of a product through `run(c)`; picks c
// from the table, or by timing when tuning is on and the bin is new.
template <class Run>
rmc_status tuned_launch(rmc_ctx* ctx, const std::string& key, int ncand, Run&& run, bool may_time = true) {
  TuneTable& tt = tune_table();
  int c = -1;
  {
    std::lock_guard<std::mutex> lk(tt.mu);
    auto it = tt.choice.find(key);
    if (it != tt.choice.end() && it->second >= 0 && it->second < ncand) c = it->second;
  }
  if (c < 0 && may_time && tt.tuning.load() > 0 && ncand > 1) {
    struct Events {  // returned to the context's pool on every exit path
      rmc_ctx* ctx;
      cudaEvent_t a, b;
      ~Events() {
        ctx->event_pool.push_back(a);
        ctx->event_pool.push_back(b);
      }
    } ev{ctx, take_event(ctx), take_event(ctx)};
    cudaEvent_t e0 = ev.a, e1 = ev.b;
    float best = INFINITY;
    int arg = 0;
    for (int i = 0; i < ncand; ++i) {
      TRY(run(i));  // warm-up (and a first launch of the configuration)
      CK(cudaEventRecord(e0, ctx->stream));
      for (int r = 0; r < 3; ++r) TRY(run(i));
      CK(cudaEventRecord(e1, ctx->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; arg = i; }
    }
    std::lock_guard<std::mutex> lk(tt.mu);
    tt.choice[key] = arg;
    c = arg;
  }
  return run(c < 0 ? 0 : c);
}

// Tile presets of the SIMT GEMM, 256 threads each: 64 x 64 (4 x 4 a thread),
// 48 x 48 (3 x 3), 32 x 32 (2 x 2); K steps of 16 (FP32) or 8 (FP64 and
// double-float).
template <typename T, bool TA, bool TB, class Epi, bool DF>
void gemm_tile(int tile, const T* A, const T* B, const GemmShape& s, int batches, const Epi& epi, cudaStream_t st) {
  constexpr int BK = sizeof(T) == 4 ? 16 : 8;
  if (tile == 1) launch_gemm<T, 48, 48, BK, 3, 3, TA, TB, Epi, DF>(A, B, s, batches, epi, st);
  else if (tile == 2) launch_gemm<T, 32, 32, BK, 2, 2, TA, TB, Epi, DF>(A, B, s, batches, epi, st);
  else launch_gemm<T, 64, 64, BK, 4, 4, TA, TB, Epi, DF>(A, B, s, batches, epi, st);
}

// G (nv1 x nv2) = X1 X2^T, contraction over n, deterministic split-K.
// Candidates: tile in {64, 48, 32} x split-K in {s, s/2, 2s}, s the default
// split count (about two CTA waves of the 64 x 64 tiling, >= 128 terms a split).
// Tensor-core Gram products (FP32 data, 3xTF32) for the long contractions of
// the wide merges (n >= kTcGramMinN): split-K over about two waves of CTAs,
// partial 128 x BN tiles to P, then the deterministic split reduction.
constexpr long kTcGramMinN = 16384;

bool tc_gram(const rmc_ctx* ctx, const float* X1, const float* X2, long n);
rmc_status gram_tc(rmc_ctx* ctx, Workspace& ws, const float* X1, int nv1, const float* X2, int nv2, long n, float* G,
                   bool symmetrize);

// tensor_ok: the caller accepts 3xTF32 accuracy (~5e-7 relative a product,
// against ~6e-8 for FP32), e.g. projections whose coefficients are applied
// again, or Gram products of small corrections; Gram matrices that are
// factorised (Cholesky-QR of a filtered block, conditioned up to ~1e6: 3xTF32
// made the factorisation fail) or diagonalised must stay on the FP32 pipe.  No
// solver call sets it: at the 256-state merges' shapes (M, N <= 288,
// K = 65536) the split-K tensor-core form measured 2.6 ms against 0.14-0.57 ms
// on the FP32 pipe (each of its TMA boxes reads 128 bytes from each of up to
// 288 rows 256 KB apart, from 148 CTAs at once); rmc_gram exposes both forms.
template <typename T>
rmc_status gram(rmc_ctx* ctx, Workspace& ws, const T* X1, int nv1, const T* X2, int nv2, long n, T* G,
                bool symmetrize, bool tensor_ok = false) {
  ProfScope ps(ctx, 4, 2.0 * nv1 * nv2 * (double)n);
  if constexpr (sizeof(T) == 4) {
    if (tensor_ok && tc_gram(ctx, X1, X2, n)) return gram_tc(ctx, ws, X1, nv1, X2, nv2, n, G, symmetrize);
  }
  bool df = false;
  if constexpr (sizeof(T) == 8) df = fp64_by_df(ctx);
  const int tiles64 = (int)(ceil_div(nv1, 64) * ceil_div(nv2, 64));
  const int base = std::min(64, (int)std::min<long>(std::max<long>(1, n / 128), std::max(1, 296 / tiles64)));
  const int max_split = (int)std::min<long>(std::max<long>(1, n / 64), 128);
  auto splits_of = [&](int c) {
    const int m = c % 3;
    const int sp = m == 0 ? base : m == 1 ? std::max(1, base / 2) : 2 * base;
    return std::max(1, std::min(sp, max_split));
  };
  T* P = nullptr;
  TRY(ws.get(&P, (size_t)std::max(base, std::min(2 * base, max_split)) * nv1 * nv2));
  // the untuned default keeps the historical choice: 16 x 16 tiles for small
  // native outputs, else 64 x 64, with the base split
  const bool small = !df && nv1 <= 32 && nv2 <= 32;
  auto run = [&](int c) -> rmc_status {
    const int sp = splits_of(c);
    GemmShape s{nv1, nv2, (int)n, n, n, 0, 0, sp};
    EpiStore<T> epi{P, nv2, 0, (long)nv1 * nv2, T(1), T(0)};
    const int tile = c / 3;
    if constexpr (sizeof(T) == 8) {
      if (df) gemm_tile<T, false, true, EpiStore<T>, true>(tile, X1, X2, s, 1, epi, ctx->stream);
      else if (small && c == 0) gemm_small<T, false, true>(X1, X2, s, 1, epi, ctx->stream);
      else gemm_tile<T, false, true, EpiStore<T>, false>(tile, X1, X2, s, 1, epi, ctx->stream);
    } else {
      if (small && c == 0) gemm_small<T, false, true>(X1, X2, s, 1, epi, ctx->stream);
      else gemm_tile<T, false, true, EpiStore<T>, false>(tile, X1, X2, s, 1, epi, ctx->stream);
    }
    CKL();
    reduce_splits_kernel<T><<<grid1d((long)nv1 * nv2), 256, 0, ctx->stream>>>(
        P, sp, (long)nv1 * nv2, nv1, nv2, G, nv2, T(1), T(0), symmetrize ? 1 : 0);
    CKL();
    return RMC_OK;
  };
  const std::string key = std::string("gram|") + (df ? "df" : sizeof(T) == 8 ? "f64" : "f32") + "|" +
                          tune_bin(nv1) + "x" + tune_bin(nv2) + "|" + tune_bin(n);
  return tuned_launch(ctx, key, 9, run);
}

// Out (nvo x n) = alpha * op(W) X + beta * Src; op(W) = W (nvo x nvi) or W^T
// (W stored nvi x nvo).  Candidates: tile in {64, 48, 32}; tuning is skipped
// (default tile) when Out aliases an input, since every timed run must leave
// the same result.
template <typename T>
rmc_status combine(rmc_ctx* ctx, const T* W, bool transW, int nvo, int nvi, const T* X, long n, T* Out, T alpha,
                   T beta, const T* Src) {
  ProfScope ps(ctx, 5, 2.0 * nvo * nvi * (double)n);
  GemmShape s{nvo, (int)n, nvi, transW ? nvo : nvi, n, 0, 0, 1};
  EpiAxpby<T> epi{Out, Src, n, n, 0, 0, alpha, beta};
  bool df = false;
  if constexpr (sizeof(T) == 8) df = fp64_by_df(ctx);
  auto run = [&](int tile) -> rmc_status {
    if constexpr (sizeof(T) == 8) {
      if (df) {
        if (transW) gemm_tile<T, true, false, EpiAxpby<T>, true>(tile, W, X, s, 1, epi, ctx->stream);
        else gemm_tile<T, false, false, EpiAxpby<T>, true>(tile, W, X, s, 1, epi, ctx->stream);
        CKL();
        return RMC_OK;
      }
    }
    if (transW) gemm_tile<T, true, false, EpiAxpby<T>, false>(tile, W, X, s, 1, epi, ctx->stream);
    else gemm_tile<T, false, false, EpiAxpby<T>, false>(tile, W, X, s, 1, epi, ctx->stream);
    CKL();
    return RMC_OK;
  };
  const bool aliased = Out == X || Out == W || (beta != T(0) && Out == Src);
  const std::string key = std::string("comb|") + (df ? "df" : sizeof(T) == 8 ? "f64" : "f32") +
                          (transW ? "|t|" : "|n|") + tune_bin(nvo) + "x" + tune_bin(nvi) + "|" + tune_bin(n);
  return tuned_launch(ctx, key, 3, run, !aliased);
}

// C (m x m) = alpha op(A) op(B) + beta Src for the small Rayleigh-Ritz products.
template <typename T, bool TA, bool TB>
rmc_status small_mm(rmc_ctx* ctx, const T* A, const T* B, int m, T* C, T alpha, T beta, const T* Src) {
  GemmShape s{m, m, m, m, m, 0, 0, 1};
  EpiAxpby<T> epi{C, Src, m, m, 0, 0, alpha, beta};
  gemm_small<T, TA, TB>(A, B, s, 1, epi, ctx->stream);
  CKL();
  return RMC_OK;
}

// ---------------------------------------------------------------------------
// Kronecker-form product with the effective Hamiltonian (Eq. (7)).
// ---------------------------------------------------------------------------
template <typename T>
struct KronOp {
  int kA = 0, kB = 0, n_ops = 0;
  const T* EA = nullptr;
  const T* EB = nullptr;
  const T* Acat = nullptr;  // kA x (n_ops kA), coefficients folded in
  const T* Bcat = nullptr;  // (n_ops kB) x kB
  long n() const { return (long)kA * kB; }
};

template <typename T>
rmc_status kron_apply(rmc_ctx* ctx, const KronOp<T>& H, const T* X, int nv, T* Y, T alpha, T beta, T gamma,
                      const T* Z, T* Tbuf) {
  const int kA = H.kA, kB = H.kB, no = H.n_ops;
  // algorithmic FLOPs: 2 n_ops kA kB (kA + kB) per vector for the two
  // contractions plus 3 kA kB for the diagonal term and the scaling
  ProfScope ps(ctx, sizeof(T) == 8 ? 1 : 0,
               (double)nv * ((double)2 * no * kA * kB * (kA + kB) + 3.0 * kA * kB));
  bool df = false;  // the mixed paths form FP64-accurate products in double-FP32
  if constexpr (sizeof(T) == 8) df = fp64_by_df(ctx);
  if (no > 0) {
    GemmShape s1{nv * kA, no * kB, kB, kB, kB, 0, 0, 1};
    EpiKron1<T> e1{Tbuf, kA, kB, nv};
    if constexpr (sizeof(T) == 8) {
      if (df) gemm_df<false, true>(X, H.Bcat, s1, 1, e1, ctx->stream);
      else gemm_big<T, false, true>(X, H.Bcat, s1, 1, e1, ctx->stream);
    } else {
      gemm_big<T, false, true>(X, H.Bcat, s1, 1, e1, ctx->stream);
    }
    CKL();
  }
  GemmShape s2{kA, nv * kB, no * kA, (long)no * kA, (long)nv * kB, 0, 0, 1};
  EpiKron2<T> e2{X, Z, H.EA, H.EB, Y, kA, kB, alpha, beta, gamma};
  if (no > 0) {
    if constexpr (sizeof(T) == 8) {
      if (df) gemm_df<false, false>(H.Acat, Tbuf, s2, 1, e2, ctx->stream);
      else gemm_big<T, false, false>(H.Acat, Tbuf, s2, 1, e2, ctx->stream);
    } else {
      gemm_big<T, false, false>(H.Acat, Tbuf, s2, 1, e2, ctx->stream);
    }
  } else {
    // no coupling: K = 0, the GEMM loop is empty and only the epilogue runs
    GemmShape s0{kA, nv * kB, 0, 1, (long)nv * kB, 0, 0, 1};
    gemm_big<T, false, false>(H.EA, X, s0, 1, e2, ctx->stream);
  }
  CKL();
  return RMC_OK;
}

// Kronecker-form product on the tcgen05 tensor cores (3xTF32, FP32 data).
// Returns false (and launches nothing) when a stage's shape does not fit the
// tensor-core kernel; the caller then runs the SIMT product.
bool tma_fits(long lda, long ldb, int K);
bool tc_fits(int kA, int kB, int n_ops) {
  int np, g;
  size_t sm;
  if (n_ops <= 0) return false;
  // each stage on the TMA-fed kernel (any N) or the plain-load one (N <= 256)
  const bool s1 = tma_fits(kB, kB, kB) || umma::plan(n_ops * kB, kB, &np, &g, &sm);
  const bool s2 = tma_fits((long)n_ops * kA, (long)n_ops * kA, n_ops * kA) || umma::plan(kA, n_ops * kA, &np, &g, &sm);
  return s1 && s2;
}

template <class Epi>
rmc_status launch_tc(rmc_ctx* ctx, const float* A, long lda, int M, const float* B, long ldb, int N, int K,
                     const Epi& epi) {
  int Npad, group;
  size_t sm;
  if (!umma::plan(N, K, &Npad, &group, &sm)) return fail(ctx, RMC_ERR_INVAL, "tensor-core plan failed");
  // process-wide attribute: raise to the limit once, never lower it
  CK(cudaFuncSetAttribute(umma::gemm_tf32x3_kernel<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)umma::kSmemLimit));
  umma::GemmArgs g{A, lda, M, B, ldb, N, Npad, K, group, ctx->d_status + 3};
  const int tiles = (M + umma::kRows - 1) / umma::kRows;
  umma::gemm_tf32x3_kernel<Epi><<<std::min(tiles, 148), umma::kThreads, sm, ctx->stream>>>(g, epi);
  CKL();
  return RMC_OK;
}

// TMA-fed pipelined form (tma_gemm.cuh).  The tensor-map encoder is a
// driver entry point, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return (EncodeTiledFn)p;
  }();
  return fn;
}

// Tensor map of a K-contiguous FP32 matrix (rows x K, row pitch ld floats),
// box 32 x box_rows, 128-byte swizzle, zero fill out of bounds.  False when
// the TMA cannot address it (pitch not a multiple of 16 bytes, base not
// 16-byte aligned).
bool make_map(CUtensorMap* m, const float* ptr, long rows, long K, long ld, int box_rows, bool swizzle = true) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc || ((uintptr_t)ptr & 15) || (ld % 4) != 0 || K < 1 || rows < 1 || ld < K) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Output of the TMA kernel's block stores: a row-major rows x cols FP32 matrix
// written in 32 x 32 blocks (no swizzle: the staging block is plain row-major).
struct TmaOut {
  float* ptr = nullptr;
  long rows = 0, cols = 0;
};

int sm_count() {
  static int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      v = 148;
    return v > 0 ? v : 148;
  }();
  return n;
}

// N tiling of the TMA kernel: at most max_bn (256, or 128 for the deeper
// pipeline) columns a tile, the columns dealt evenly over the tiles, rounded
// up to the MMA's multiple of 16.
int tma_max_bn() {
  static int v = [] {
    const char* e = std::getenv("RMC_TMA_BN");
    const int b = e ? std::atoi(e) : 256;
    return b == 128 ? 128 : 256;
  }();
  return v;
}

void tma_n_tiles(int N, int* n_tiles, int* BN) {
  const int mx = tma_max_bn();
  *n_tiles = (N + mx - 1) / mx;
  *BN = ((N + *n_tiles - 1) / *n_tiles + 15) / 16 * 16;
}

bool tma_fits(long lda, long ldb, int K) { return encode_tiled() && K >= 1 && lda % 4 == 0 && ldb % 4 == 0; }

template <class Epi>
rmc_status launch_tma(rmc_ctx* ctx, const float* A, long lda, int M, const float* B, long ldb, int N, int K,
                      const Epi& epi, bool* launched, const TmaOut& out = TmaOut{}, int k_splits = 1,
                      int kc_split = 0) {
  *launched = false;
  int n_tiles, BN;
  tma_n_tiles(N, &n_tiles, &BN);
  CUtensorMap ma, mb, mo;
  if (!make_map(&ma, A, M, K, lda, tmag::kBM) || !make_map(&mb, B, N, K, ldb, BN)) return RMC_OK;
  // block stores when the output can be addressed (otherwise mo is an unused copy)
  const bool store = out.ptr && make_map(&mo, out.ptr, out.rows, out.cols, out.cols, 32, false);
  if (!store) mo = mb;
  const int kcs = (K + 31) / 32;
  tmag::Args g{M, N, K, BN, (M + tmag::kBM - 1) / tmag::kBM, n_tiles, ctx->d_status + 3, store ? 1 : 0,
               std::max(1, k_splits), kc_split > 0 ? kc_split : kcs};
  const int tiles = g.m_tiles * g.n_tiles;
  const int grid = std::min(tiles, sm_count());
  // the attribute is process-wide: always the largest size any launch needs
  if (tmag::stages_for(BN) == 3) {
    CK(cudaFuncSetAttribute(tmag::gemm_tma_tf32x3_kernel<3, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)tmag::smem_bytes(128, 3)));
    tmag::gemm_tma_tf32x3_kernel<3, Epi><<<grid, tmag::kThreads, tmag::smem_bytes(BN, 3), ctx->stream>>>(ma, mb, mo, g,
                                                                                                   epi);
  } else {
    CK(cudaFuncSetAttribute(tmag::gemm_tma_tf32x3_kernel<2, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)tmag::smem_bytes(256, 2)));
    tmag::gemm_tma_tf32x3_kernel<2, Epi><<<grid, tmag::kThreads, tmag::smem_bytes(BN, 2), ctx->stream>>>(ma, mb, mo, g,
                                                                                                   epi);
  }
  CKL();
  *launched = true;
  return RMC_OK;
}

bool tc_gram(const rmc_ctx* ctx, const float* X1, const float* X2, long n) {
  return ctx->cfg.precision != RMC_PREC_FP64 && n >= kTcGramMinN && n % 4 == 0 && !((uintptr_t)X1 & 15) &&
         !((uintptr_t)X2 & 15) && encode_tiled();
}

rmc_status gram_tc(rmc_ctx* ctx, Workspace& ws, const float* X1, int nv1, const float* X2, int nv2, long n, float* G,
                   bool symmetrize) {
  const int kcs = (int)((n + 31) / 32);
  int n_tiles, BN;
  tma_n_tiles(nv2, &n_tiles, &BN);
  const int mn = (nv1 + tmag::kBM - 1) / tmag::kBM * n_tiles;
  int ks = std::max(1, std::min(kcs, (2 * sm_count() + mn - 1) / mn));
  const int kc_split = (kcs + ks - 1) / ks;
  ks = (kcs + kc_split - 1) / kc_split;
  float* P = nullptr;
  TRY(ws.get(&P, (size_t)ks * nv1 * nv2));
  bool done = false;
  TRY(launch_tma(ctx, X1, n, nv1, X2, n, nv2, (int)n, EpiSplitT{P, nv1, nv2}, &done,
                 TmaOut{P, (long)ks * nv2, (long)nv1}, ks, kc_split));
  if (!done) return fail(ctx, RMC_ERR_INVAL, "tensor-core Gram product: operands not addressable by the TMA");
  reduce_splits_t_kernel<<<grid1d((long)nv1 * nv2), 256, 0, ctx->stream>>>(P, ks, nv1, nv2, G);
  CKL();
  if (symmetrize && nv1 == nv2) {
    symmetrize_kernel<<<grid1d((long)nv1 * nv1), 256, 0, ctx->stream>>>(G, nv1);
    CKL();
  }
  return RMC_OK;
}

rmc_status kron_apply_tc(rmc_ctx* ctx, const KronOp<float>& H, const float* X, int nv, float* Y, float alpha,
                         float beta, float gamma, const float* Z, float* Tbuf) {
  const int kA = H.kA, kB = H.kB, no = H.n_ops;
  ProfScope ps(ctx, 0, (double)nv * ((double)2 * no * kA * kB * (kA + kB) + 3.0 * kA * kB));
  // stage 1: T'[(v, b)][(j, a)] = sum_b' X[v][a][b'] B_j[b][b']; stage 2:
  // Y^T rows (v, b) = T' Acat^T.  Each stage on the TMA-fed kernel when the
  // TMA can address its operands, else on the plain-load kernel.
  bool done = false;
  const EpiKron1T<float> e1{Tbuf, kA, kB, no};
  TRY(launch_tma(ctx, X, kB, nv * kA, H.Bcat, kB, no * kB, kB, e1, &done,
                 TmaOut{Tbuf, (long)nv * kB, (long)no * kA}));
  if (!done) TRY(launch_tc(ctx, X, kB, nv * kA, H.Bcat, kB, no * kB, kB, e1));
  const EpiKron2T<float> e2{X, Z, H.EA, H.EB, Y, kA, kB, alpha, beta, gamma};
  TRY(launch_tma(ctx, Tbuf, (long)no * kA, nv * kB, H.Acat, (long)no * kA, kA, no * kA, e2, &done,
                 TmaOut{Y, (long)nv * kA, (long)kB}));
  if (!done) TRY(launch_tc(ctx, Tbuf, (long)no * kA, nv * kB, H.Acat, (long)no * kA, kA, no * kA, e2));
  return RMC_OK;
}

// The working-precision product of the subspace iteration: tensor cores for
// the TF32 mixed path when the shape fits, SIMT otherwise.
// RMC_PREC_MIXED_TF32 takes the tensor cores wherever a stage fits; the
// default mixed path takes them for wide merges whose both stages the TMA-fed
// kernel can address (k_A k_B >= 16384 and 16-byte row pitches), where they
// are 2-4x faster than the FP32 pipe (measured at k = 128 and 256); smaller
// products stay on the FP32 pipe, where the tensor-core form is not faster.
bool tc_wide(int kA, int kB, int n_ops) {
  return n_ops > 0 && (long)kA * kB >= 16384 && tma_fits(kB, kB, kB) &&
         tma_fits((long)n_ops * kA, (long)n_ops * kA, n_ops * kA);
}

template <typename T>
rmc_status kron_work(rmc_ctx* ctx, const KronOp<T>& H, const T* X, int nv, T* Y, T alpha, T beta, T gamma,
                     const T* Z, T* Tbuf) {
  if constexpr (sizeof(T) == 4) {
    const bool tc = ctx->cfg.precision == RMC_PREC_MIXED_TF32 ? tc_fits(H.kA, H.kB, H.n_ops)
                    : ctx->cfg.precision == RMC_PREC_MIXED  ? tc_wide(H.kA, H.kB, H.n_ops)
                                                             : false;
    if (tc) return kron_apply_tc(ctx, H, X, nv, Y, alpha, beta, gamma, Z, Tbuf);
  }
  return kron_apply<T>(ctx, H, X, nv, Y, alpha, beta, gamma, Z, Tbuf);
}

// Fused forms (one launch, vectors held in shared memory; see cheb_fused.cuh).
// Plan: vectors per CTA (enough that a CTA has >= 2048 outputs per product,
// within the shared-memory limit) and whether the operators are staged in
// shared memory (FP32 only).  False when one vector does not fit.
template <typename T>
bool fused_plan(const KronOp<T>& H, int nv, FusedArgs* p, size_t* smem) {
  const long n = H.n();
  const int no = H.n_ops;
  if (nv <= 0 || n <= 0) return false;
  const size_t per_vec = (size_t)(2 + no) * n * sizeof(T);
  const size_t red = 32 * sizeof(T);
  size_t ops = (size_t)no * ((size_t)H.kA * H.kA + (size_t)H.kB * H.kB) * sizeof(T);
  const bool ops_sm = sizeof(T) == 4 && no > 0 && ops + per_vec + red <= kFusedSmemLimit;
  if (!ops_sm) ops = 0;
  if (per_vec + ops + red > kFusedSmemLimit) return false;
  const int fit = (int)((kFusedSmemLimit - ops - red) / per_vec);
  const int vpc = (int)std::min<long>({(2048 + n - 1) / n, (long)fit, (long)nv});
  *p = FusedArgs{H.kA, H.kB, no, nv, std::max(1, vpc), 0, 0, ops_sm ? 1 : 0, 0.0, 0.0, 0.0};
  *smem = (size_t)p->vpc * per_vec + ops + red;
  return true;
}

template <typename T>
rmc_status launch_fused(rmc_ctx* ctx, const KronOp<T>& H, const T* X, const T* HX, T* Out, const FusedArgs& p,
                        size_t smem, double flops) {
  ProfScope ps(ctx, sizeof(T) == 8 ? 1 : 7, flops);
  if constexpr (sizeof(T) == 4) {
    // the k-major float4 kernel whenever its (padded) layout fits: at most
    // the planned vectors per CTA, fewer if the padding needs the room
    if (p.n_ops > 0 && p.ops_in_smem) {
      FusedArgs q = p;
      while (q.vpc > 1 && v4_layout(q.kA, q.kB, q.n_ops, q.vpc).bytes > kFusedSmemLimit) --q.vpc;
      const size_t bytes = v4_layout(q.kA, q.kB, q.n_ops, q.vpc).bytes;
      if (bytes <= kFusedSmemLimit) {
        CK(cudaFuncSetAttribute(cheb_fused_v4_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kFusedSmemLimit));
        cheb_fused_v4_kernel<<<ceil_div(q.nv, q.vpc), kV4Threads, bytes, ctx->stream>>>(
            (const float*)X, (const float*)HX, (const float*)H.EA, (const float*)H.EB, (const float*)H.Acat,
            (const float*)H.Bcat, (float*)Out, q);
        CKL();
        return RMC_OK;
      }
    }
  }
  // process-wide attribute: raise to the limit once, never lower it
  CK(cudaFuncSetAttribute(cheb_fused_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemLimit));
  cheb_fused_kernel<T><<<ceil_div(p.nv, p.vpc), kFusedThreads, smem, ctx->stream>>>(X, HX, H.EA, H.EB, H.Acat,
                                                                                       H.Bcat, Out, p);
  CKL();
  return RMC_OK;
}

inline double kron_flops_per_vector(int kA, int kB, int no) {
  return (double)2 * no * kA * kB * (kA + kB) + 3.0 * kA * kB;
}

// Out = normalised p(H) X, p the degree-deg filter damping [a, ub] scaled at
// theta0 (as cheb_filter, followed by column normalisation).  With hx_given
// the product H X is read from HX, else formed in the kernel.  *done = false
// when the block does not fit (nothing launched).
template <typename T>
rmc_status cheb_fused(rmc_ctx* ctx, const KronOp<T>& H, const T* X, const T* HX, int nv, int deg, double theta0,
                      double a, double ub, T* Out, bool* done) {
  *done = false;
  FusedArgs p;
  size_t smem;
  if (sizeof(T) == 4 && ctx->cfg.precision == RMC_PREC_MIXED_TF32) return RMC_OK;  // tensor-core product
  if (!fused_plan<T>(H, nv, &p, &smem)) return RMC_OK;
  p.deg = std::max(1, deg);
  p.compute_hx = HX ? 0 : 1;
  p.e = (ub - a) / 2;
  p.c = (ub + a) / 2;
  p.sigma1 = p.e / (theta0 - p.c);
  const double products = (double)(p.deg - 1 + p.compute_hx);
  TRY(launch_fused<T>(ctx, H, X, HX, Out, p, smem, nv * products * kron_flops_per_vector(H.kA, H.kB, H.n_ops)));
  *done = true;
  return RMC_OK;
}

// The fused filter / product on FP64 data in double-FP32 arithmetic
// (cheb_fused_df_kernel): deg >= 1 gives the normalised filter output with
// H X formed in the kernel, deg == 0 the plain product.  *done = false when
// the block does not fit (nothing launched).
rmc_status cheb_fused_df(rmc_ctx* ctx, const KronOp<double>& H, const double* X, int nv, int deg, double theta0,
                         double a, double ub, double* Out, bool* done) {
  *done = false;
  FusedArgs p;
  size_t smem;
  if (!fused_plan<double>(H, nv, &p, &smem)) return RMC_OK;  // same shared-memory layout size as FP64
  Workspace ws(ctx);
  const int no = H.n_ops;
  float2 *Ahl = nullptr, *Bhl = nullptr;
  if (no > 0) {
    TRY(ws.get(&Ahl, (size_t)H.kA * no * H.kA));
    TRY(ws.get(&Bhl, (size_t)no * H.kB * H.kB));
    df_split_kernel<<<grid1d((long)H.kA * no * H.kA), 256, 0, ctx->stream>>>(H.Acat, (long)H.kA * no * H.kA, Ahl);
    CKL();
    df_split_kernel<<<grid1d((long)no * H.kB * H.kB), 256, 0, ctx->stream>>>(H.Bcat, (long)no * H.kB * H.kB, Bhl);
    CKL();
  }
  p.deg = std::max(0, deg);
  p.compute_hx = 1;
  if (p.deg > 0) {
    p.e = (ub - a) / 2;
    p.c = (ub + a) / 2;
    p.sigma1 = p.e / (theta0 - p.c);
  }
  ProfScope ps(ctx, 1, nv * (double)std::max(1, p.deg) * kron_flops_per_vector(H.kA, H.kB, no));
  CK(cudaFuncSetAttribute(cheb_fused_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemLimit));
  cheb_fused_df_kernel<<<ceil_div(p.nv, p.vpc), kDfThreads, smem, ctx->stream>>>(X, H.EA, H.EB, Ahl, Bhl, Out, p);
  CKL();
  *done = true;
  return RMC_OK;
}

// Y = H X: the fused single-launch product when the block fits, else the
// two-stage product (tensor cores for the TF32 working precision).
template <typename T>
rmc_status kron_product(rmc_ctx* ctx, const KronOp<T>& H, const T* X, int nv, T* Y, T* Tbuf) {
  FusedArgs p;
  size_t smem;
  if (!(sizeof(T) == 4 && ctx->cfg.precision == RMC_PREC_MIXED_TF32) && fused_plan<T>(H, nv, &p, &smem))
    return launch_fused<T>(ctx, H, X, nullptr, Y, p, smem, nv * kron_flops_per_vector(H.kA, H.kB, H.n_ops));
  return kron_work<T>(ctx, H, X, nv, Y, T(1), T(0), T(0), nullptr, Tbuf);
}

// ---------------------------------------------------------------------------
// Small symmetric eigensolvers.
// ---------------------------------------------------------------------------
template <typename TI, typename TO>
rmc_status jacobi(rmc_ctx* ctx, const TI* S, int m, TO* w, TO* V) {
  if (m > kMaxSmallDim) return fail(ctx, RMC_ERR_INVAL, "small eigensolver: m=%d exceeds %d", m, kMaxSmallDim);
  ProfScope ps(ctx, 2, 0.0);
  const size_t sm = jacobi_smem_bytes(m);
  // The attribute is process-wide and other threads launch this kernel too:
  // always raise it to the largest size any call can need, never lower it.
  CK(cudaFuncSetAttribute(jacobi_kernel<TI, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)jacobi_smem_bytes(kMaxSmallDim)));
  jacobi_kernel<TI, TO><<<1, jacobi_threads(m), sm, ctx->stream>>>(S, m, w, V, ctx->d_status + 1, 30);
  CKL();
  return RMC_OK;
}

// FP64-accurate: FP32 Jacobi, then Ogita-Aishima refinement steps (at most
// kOASteps; each step is quadratically convergent, and once a correction is at
// the FP64 rounding level a device flag makes the remaining launches return
// at once).
constexpr int kOASteps = 8;
constexpr int kOAParts = 148;  // CTAs of an Ogita-Aishima step (rows dealt to them)

// The m x m products of the refinement: in the mixed paths in double-float on
// the FP32 pipe (like their block products), in the FP64 path native FP64.
template <bool TA, bool TB>
rmc_status small_mm_skip(rmc_ctx* ctx, const double* A, const double* B, int m, double* C, double beta,
                         const double* Src, const int* skip, double alpha = 1.0) {
  GemmShape s{m, m, m, m, m, 0, 0, 1};
  s.skip = skip;
  EpiAxpby<double> epi{C, Src, m, m, 0, 0, alpha, beta};
  if (fp64_by_df(ctx)) launch_gemm<double, 16, 16, 8, 1, 1, TA, TB, EpiAxpby<double>, true>(A, B, s, 1, epi, ctx->stream);
  else gemm_small<double, TA, TB>(A, B, s, 1, epi, ctx->stream);
  CKL();
  return RMC_OK;
}

// With from_identity the Jacobi start is skipped and the refinement starts
// from the identity: used when S is already nearly diagonal (the Rayleigh-
// Ritz matrix of a block whose chunks were each diagonalised), and for any
// size (no shared-memory bound).
rmc_status syev64(rmc_ctx* ctx, Workspace& ws, const double* S, int m, double* w, double* V,
                  bool from_identity = false) {
  if (m < 1 || m > 1024) return fail(ctx, RMC_ERR_INVAL, "small eigensolver: m=%d outside [1, 1024]", m);
  double *V0, *V1, *R, *AV, *Sp, *lam, *pe, *part;
  int* done;
  const int nparts = std::min(m, kOAParts);
  TRY(ws.get(&pe, 1));
  TRY(ws.get(&part, (size_t)4 * nparts));
  TRY(ws.get(&V0, (size_t)m * m));
  TRY(ws.get(&V1, (size_t)m * m));
  TRY(ws.get(&R, (size_t)m * m));
  TRY(ws.get(&AV, (size_t)m * m));
  TRY(ws.get(&Sp, (size_t)m * m));
  TRY(ws.get(&lam, (size_t)m));
  TRY(ws.get(&done, 1));
  CK(cudaMemsetAsync(done, 0, sizeof(int), ctx->stream));
  CK(cudaMemsetAsync(pe, 0x7f, sizeof(double), ctx->stream));  // a huge previous correction
  if (from_identity || m > kMaxSmallDim) {
    identity_fill_kernel<<<grid1d((long)m * m), 256, 0, ctx->stream>>>(V0, m);
    CKL();
  } else {
    TRY((jacobi<double, double>(ctx, S, m, lam, V0)));
  }
  const int steps = (from_identity || m > kMaxSmallDim) ? 2 * kOASteps : kOASteps;
  for (int it = 0; it < steps; ++it) {
    TRY((small_mm_skip<true, false>(ctx, V0, V0, m, R, 0.0, nullptr, done)));
    identity_minus_kernel<<<grid1d((long)m * m), 256, 0, ctx->stream>>>(R, m, done);
    CKL();
    TRY((small_mm_skip<false, false>(ctx, S, V0, m, AV, 0.0, nullptr, done)));
    TRY((small_mm_skip<true, false>(ctx, V0, AV, m, Sp, 0.0, nullptr, done)));
    oa_sums_kernel<<<nparts, 256, 0, ctx->stream>>>(R, Sp, S, m, lam, part, done);
    CKL();
    oa_update_kernel<<<nparts, 256, 0, ctx->stream>>>(R, Sp, lam, m, part, nparts, part + 3 * nparts, done);
    CKL();
    oa_finish_kernel<<<1, 256, 0, ctx->stream>>>(part + 3 * nparts, nparts, done, pe);
    CKL();
    TRY((small_mm_skip<false, false>(ctx, V0, R, m, V1, 1.0, V0, done)));
    copy_unless_kernel<<<grid1d((long)m * m), 256, 0, ctx->stream>>>(V1, V0, m * m, done);
    CKL();
  }
  // one Newton-Schulz step: exact orthonormality whatever the refinement left
  TRY((small_mm_skip<true, false>(ctx, V0, V0, m, R, 0.0, nullptr, nullptr)));
  half_identity_minus_kernel<<<grid1d((long)m * m), 256, 0, ctx->stream>>>(R, m, AV);
  CKL();
  TRY((small_mm_skip<false, false>(ctx, V0, AV, m, V1, 1.0, V0, nullptr)));
  // exact rotations for the pairs the refinement left coupled (near-degenerate
  // pairs whose gap is below its coupling bound): on Sp = V^T S V in FP64
  if (m <= kMaxSmallDim) {
    TRY((small_mm_skip<false, false>(ctx, S, V1, m, AV, 0.0, nullptr, nullptr)));
    TRY((small_mm_skip<true, false>(ctx, V1, AV, m, Sp, 0.0, nullptr, nullptr)));
    CK(cudaFuncSetAttribute(jacobi_cleanup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(double) * kMaxSmallDim * kMaxSmallDim)));
    jacobi_cleanup_kernel<<<1, 1024, sizeof(double) * m * m, ctx->stream>>>(Sp, m, V1, lam, 1e-14);
    CKL();
  } else {
    // the same for a matrix too large for shared memory (V0 is free here and
    // holds the working copy of Sp)
    TRY((small_mm_skip<false, false>(ctx, S, V1, m, AV, 0.0, nullptr, nullptr)));
    TRY((small_mm_skip<true, false>(ctx, V1, AV, m, Sp, 0.0, nullptr, nullptr)));
    jacobi_cleanup_global_kernel<<<1, 512, 0, ctx->stream>>>(Sp, m, V0, V1, lam, 1e-14);
    CKL();
  }
  sort_pairs_kernel<<<1, 256, 0, ctx->stream>>>(lam, V1, m, w, V);
  CKL();
  return RMC_OK;
}

// Cholesky-QR of a vector-major block in place: a Cholesky pass with a small
// relative diagonal shift (robust for the ill-conditioned filter output), then
// a second pass that is the first-order correction X <- (I - F^T) X whenever
// the first left X X^T within 1e-3 of the identity (error O(||E||^2), no
// second factorisation), else a full second Cholesky pass.
template <typename T>
rmc_status cholqr(rmc_ctx* ctx, Workspace& ws, T* X, int nv, long n, T* tmp, double shift) {
  ProfScope ps(ctx, 3, 0.0);
  T *G, *Li;
  TRY(ws.get(&G, (size_t)nv * nv));
  TRY(ws.get(&Li, (size_t)nv * nv));
  CK(cudaFuncSetAttribute(cholinv_kernel<T, T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          (int)cholinv_smem_bytes(kMaxSmallDim, sizeof(T))));
  const size_t sm = cholinv_smem_bytes(nv, sizeof(T));
  for (int pass = 0; pass < 2; ++pass) {
    TRY(gram<T>(ctx, ws, X, nv, X, nv, n, G, true));
    cholinv_kernel<T, T, T><<<1, cholinv_threads<T>(), sm, ctx->stream>>>(G, nv, pass == 0 ? shift : 0.0, Li, ctx->d_status + 2,
                                                          pass == 0 ? 0 : 1);
    CKL();
    TRY(combine<T>(ctx, Li, false, nv, nv, X, n, tmp, T(1), T(0), nullptr));
    CK(cudaMemcpyAsync(X, tmp, sizeof(T) * nv * n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return RMC_OK;
}

// FP64 Cholesky-QR for a nearly orthonormal block: FP32 Cholesky of the FP64
// Gram matrix, then two first-order FP64 passes (X <- X - F^T X).
rmc_status cholqr64_refine(rmc_ctx* ctx, Workspace& ws, double* X, int nv, long n, double* tmp,
                           int first_order_passes = 2) {
  ProfScope ps(ctx, 3, 0.0);
  double *G, *Li;
  TRY(ws.get(&G, (size_t)nv * nv));
  TRY(ws.get(&Li, (size_t)nv * nv));
  const bool wide = nv > kMaxSmallDim;  // too wide for the one-CTA factorisation: the block is
                                        // then orthonormal to working precision, first order suffices
  if (!wide) {
    // an FP64 factorisation of the Gram matrix, and a second one (first order
    // when the first left it within 1e-3 of the identity): blocks conditioned
    // up to ~1e6, as left by the refinement filter, come out orthonormal
    const size_t sm = cholinv_smem_bytes(nv, sizeof(double));
    CK(cudaFuncSetAttribute(cholinv_kernel<double, double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)cholinv_smem_bytes(kMaxSmallDim, sizeof(double))));
    for (int pass = 0; pass < 2; ++pass) {
      TRY(gram<double>(ctx, ws, X, nv, X, nv, n, G, true));
      cholinv_kernel<double, double, double><<<1, cholinv_threads<double>(), sm, ctx->stream>>>(G, nv, 0.0, Li, ctx->d_status + 2, pass);
      CKL();
      TRY(combine<double>(ctx, Li, false, nv, nv, X, n, tmp, 1.0, 0.0, nullptr));
      CK(cudaMemcpyAsync(X, tmp, sizeof(double) * nv * n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
  }
  // first-order passes square the deviation from orthonormality: two take a
  // block within 1e-3 of orthonormal (a wide block from the FP32 phase is
  // within ~1e-6) to rounding level, one suffices for a block within ~1e-8
  // (the refinement leaves ~1e-11)
  for (int pass = 0; pass < first_order_passes; ++pass) {
    TRY(gram<double>(ctx, ws, X, nv, X, nv, n, G, true));
    cholqr_first_order_kernel<<<grid1d((long)nv * nv), 256, 0, ctx->stream>>>(G, nv, Li);
    CKL();
    TRY(combine<double>(ctx, Li, false, nv, nv, X, n, tmp, -1.0, 1.0, X));
    CK(cudaMemcpyAsync(X, tmp, sizeof(double) * nv * n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return RMC_OK;
}

rmc_status read_status(rmc_ctx* ctx, int* vals, int count) {
  CK(cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(int) * count, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  harvest(ctx);
  std::memcpy(vals, ctx->h_pinned, sizeof(int) * count);
  return RMC_OK;
}

template <typename T>
rmc_status to_host(rmc_ctx* ctx, const T* d, double* h, int count) {
  if (count <= 0) return RMC_OK;
  if (sizeof(T) * count > kPinnedDoubles * sizeof(double)) return fail(ctx, RMC_ERR_INVAL, "staging too small");
  CK(cudaMemcpyAsync(ctx->h_pinned, d, sizeof(T) * count, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  harvest(ctx);
  const T* src = (const T*)ctx->h_pinned;
  for (int i = 0; i < count; ++i) h[i] = (double)src[i];
  return RMC_OK;
}

int cut_rule(const std::vector<double>& th, int k_ret, double tau) {
  const int n = (int)th.size();
  if (k_ret >= n) return n;
  for (int kp = k_ret; kp > 0; --kp)
    if (th[kp] - th[kp - 1] > tau * std::max(1.0, std::fabs(th[kp]))) return kp;
  return k_ret;
}

// ---------------------------------------------------------------------------
// Block construction helpers.
// ---------------------------------------------------------------------------
rmc_status new_block(rmc_ctx* ctx, int k, int n_ops, int rows, rmc_block** out) {
  std::unique_ptr<rmc_block> b(new rmc_block);
  b->k = k;
  b->n_ops = n_ops;
  b->rows = rows;
  void* p = nullptr;
  TRY(dalloc(ctx, &p, sizeof(double) * k));
  b->E = (double*)p;
  if (n_ops > 0) {
    rmc_status st = dalloc(ctx, &p, sizeof(double) * (size_t)n_ops * k * k);
    if (st != RMC_OK) { dfree(ctx, b->E); return st; }
    b->ops = (double*)p;
  }
  if (rows > 0) {
    rmc_status st = dalloc(ctx, &p, sizeof(double) * (size_t)rows * k);
    if (st != RMC_OK) { dfree(ctx, b->E); dfree(ctx, b->ops); return st; }
    b->basis = (double*)p;
  }
  b->tags.resize(n_ops);
  b->opnorm.assign(n_ops, 1.0);
  *out = b.release();
  ctx->blocks.insert(*out);
  return RMC_OK;
}

void free_block(rmc_ctx* ctx, rmc_block* b) {
  dfree(ctx, b->E);
  dfree(ctx, b->ops);
  dfree(ctx, b->basis);
  ctx->blocks.erase(b);
  delete b;
}

// Leaf from a dense device H (D x D) and dense device operators.
rmc_status leaf_from_device(rmc_ctx* ctx, Workspace& ws, const double* dH, int D, int k, bool cut,
                            const std::vector<const double*>& dops, const std::vector<rmc_op_tag>& tags,
                            const std::vector<double>& norms, rmc_block** out) {
  if (D > kMaxSmallDim) return fail(ctx, RMC_ERR_INVAL, "leaf dimension %d exceeds %d", D, kMaxSmallDim);
  double *w, *V;
  TRY(ws.get(&w, D));
  TRY(ws.get(&V, (size_t)D * D));
  TRY(syev64(ctx, ws, dH, D, w, V));
  std::vector<double> hw(D);
  TRY(to_host(ctx, w, hw.data(), D));
  const int kr = std::min(k, D);
  const int keff = cut ? cut_rule(hw, kr, ctx->cfg.tau_deg) : kr;
  const int n_ops = (int)dops.size();
  rmc_block* b = nullptr;
  TRY(new_block(ctx, keff, n_ops, D, &b));
  CK(cudaMemcpyAsync(b->E, w, sizeof(double) * keff, cudaMemcpyDeviceToDevice, ctx->stream));
  // basis[i][r] = V[r][i]: vector-major copy of the first keff columns
  columns_to_vectors_kernel<double><<<grid1d((long)keff * D), 256, 0, ctx->stream>>>(V, D, keff, b->basis);
  CKL();
  gauge_kernel<<<keff, 128, 0, ctx->stream>>>(b->basis, D);
  CKL();
  double* Tm;
  TRY(ws.get(&Tm, (size_t)keff * D));
  for (int j = 0; j < n_ops; ++j) {
    // T = U^T O (keff x D), o = T U (keff x keff)
    GemmShape s1{keff, D, D, D, D, 0, 0, 1};
    EpiStore<double> e1{Tm, D, 0, 0, 1.0, 0.0};
    gemm_small<double, false, false>(b->basis, dops[j], s1, 1, e1, ctx->stream);
    CKL();
    GemmShape s2{keff, keff, D, D, D, 0, 0, 1};
    EpiStore<double> e2{b->ops + (size_t)j * keff * keff, keff, 0, 0, 1.0, 0.0};
    gemm_small<double, false, true>(Tm, b->basis, s2, 1, e2, ctx->stream);
    CKL();
    b->tags[j] = tags[j];
    b->opnorm[j] = norms[j];
  }
  *out = b;
  return RMC_OK;
}

double host_opnorm2(const double* O, int k) {
  // power iteration on O^T O for an upper bound of ||O||_2 (k <= 256), then a
  // 1% margin; exact enough for the filter's spectral bound.
  std::vector<double> x(k, 1.0 / std::sqrt((double)k)), y(k), z(k);
  double lam = 0;
  for (int it = 0; it < 60; ++it) {
    for (int i = 0; i < k; ++i) { double s = 0; for (int j = 0; j < k; ++j) s += O[i * k + j] * x[j]; y[i] = s; }
    for (int i = 0; i < k; ++i) { double s = 0; for (int j = 0; j < k; ++j) s += O[j * k + i] * y[j]; z[i] = s; }
    double nz = 0;
    for (double v : z) nz += v * v;
    nz = std::sqrt(nz);
    if (nz == 0) return 0;
    lam = nz;
    for (int i = 0; i < k; ++i) x[i] = z[i] / nz;
  }
  double fro = 0;
  for (int i = 0; i < k * k; ++i) fro += O[i] * O[i];
  return std::min(std::sqrt(fro), 1.01 * std::sqrt(lam) + 1e-12);
}

// ---------------------------------------------------------------------------
// One merge.
// ---------------------------------------------------------------------------
struct MergeInput {
  const rmc_block* A;
  const rmc_block* B;
  std::vector<rmc_term> terms;
  int k_keep;
  std::vector<rmc_carry> carry;
  bool top;
};

template <typename W>
rmc_status project_out(rmc_ctx* ctx, const W* Xl, int nl, W* Xa, int na, long n, W* C, int passes = 2);

// Chebyshev filter (Zhou and Saad's scaled three-term recurrence) of degree
// deg >= 2 applied to the block X with H X given: damps [a, ub], scaled at
// theta0.  Uses Y0, Y1, Y2 (b x n each) and leaves the result in *out (one of
// them); X and HX are left unchanged.
//
// With nl > 0 locked vectors Ql (orthonormal, below theta0) the filter runs on
// the deflated operator P H P, P = I - Ql^T Ql: each new term has the locked
// span removed (one Gram-Schmidt pass, Cbuf holds nl x b coefficients).  The
// polynomial is largest below the damped interval, so without this the
// rounding-level locked components of X would grow by T_deg at the locked
// eigenvalues, far faster than the wanted ones, and swamp them in working
// precision.
//
// The locked span need not be removed after every product: a rounding-level
// locked component grows, relative to the scaled wanted ones, by the scalar
// recurrence evaluated at the lowest locked eigenvalue theta_lock (which has
// the fastest growth below the damped interval).  With theta_lock given, a
// term is deflated once that growth since the last deflation exceeds
// kDeflateGrowth, and the last term is left to the caller's orthonormalisation
// (which removes the locked span twice); with theta_lock NaN every term is
// deflated.
constexpr double kDeflateGrowth = 10.0;

template <typename W>
rmc_status cheb_filter(rmc_ctx* ctx, const KronOp<W>& H, const W* X, const W* HX, int b, double theta0, double a,
                       double ub, int deg, W* Y0, W* Y1, W* Y2, W* Tbuf, W** out, const W* Ql = nullptr,
                       int nl = 0, W* Cbuf = nullptr, double theta_lock = NAN) {
  const long n = H.n();
  const double e = (ub - a) / 2, c = (ub + a) / 2;
  double sigma = e / (theta0 - c);
  const double tau = 2.0 / sigma;
  const bool every = std::isnan(theta_lock);
  // the scalar recurrence at theta_lock, and its value at the last deflation
  double yl_prev = 1.0, yl = sigma / e * (theta_lock - c), yl_ref = 1.0;
  auto due = [&](int d, double y) {
    if (nl <= 0) return false;
    if (every) return true;
    if (d == deg) return false;
    if (std::fabs(y) > kDeflateGrowth * std::fabs(yl_ref)) {
      yl_ref = y;
      return true;
    }
    return false;
  };
  // Y1 = (sigma/e) (H X - c X), from the stored H X
  axpby_kernel<W><<<grid1d((long)b * n), 256, 0, ctx->stream>>>(HX, X, (long)b * n, W(sigma / e),
                                                                 W(-c * sigma / e), Y1);
  CKL();
  if (due(1, yl)) TRY(project_out<W>(ctx, Ql, nl, Y1, b, n, Cbuf, 1));
  const W* Yprev = X;
  W* Ycur = Y1;
  W* Ynext = Y2;
  W* spare = Y0;
  for (int d = 2; d <= deg; ++d) {
    const double s1 = 1.0 / (tau - sigma);
    TRY(kron_work<W>(ctx, H, Ycur, b, Ynext, W(2 * s1 / e), W(-2 * s1 * c / e), W(-sigma * s1), Yprev, Tbuf));
    const double yl_next = 2 * s1 / e * (theta_lock - c) * yl - sigma * s1 * yl_prev;
    yl_prev = yl;
    yl = yl_next;
    if (due(d, yl)) TRY(project_out<W>(ctx, Ql, nl, Ynext, b, n, Cbuf, 1));
    // rotate: the buffer two steps back is free unless it is X itself
    W* old_prev = const_cast<W*>(Yprev);
    Yprev = Ycur;
    Ycur = Ynext;
    Ynext = (old_prev == X) ? spare : old_prev;
    sigma = s1;
  }
  *out = Ycur;
  return RMC_OK;
}

// Norm of the pseudo-random part of each start vector (per element amplitude
// kStartAmp / sqrt(n), uniform, so the norm is about kStartAmp / sqrt(3)).
constexpr double kStartAmp = 1e-2;

// Rounding floor of the FP32 iterations (mixed paths): the worst relative
// residual of the wanted vectors has not halved in kStallIters iterations and
// is within kStallFactor of the tolerance.  The iteration then stops as
// converged and the FP64 refinement that follows sets the final accuracy (its
// own residual test decides).  Wide blocks of large merges reach a floor of a
// few 1e-6 relative in FP32.
constexpr int kStallIters = 8;
constexpr double kStallFactor = 20.0;
struct StallGuard {
  double best = 1e300;
  int since = 0;
  bool at_floor(double worst, double tol) {
    if (worst < 0.5 * best) {
      best = worst;
      since = 0;
      return false;
    }
    return ++since >= kStallIters && worst < kStallFactor * tol;
  }
};

// Worst relative residual r_i / max(1, |theta_i|) over the first m vectors.
inline double worst_relative(const std::vector<double>& r, const std::vector<double>& th, int m, int* at) {
  double w = 0;
  *at = 0;
  for (int i = 0; i < m; ++i) {
    const double v = r[i] / std::max(1.0, std::fabs(th[i]));
    if (v > w) { w = v; *at = i; }
  }
  return w;
}

template <typename W>
rmc_status chfsi(rmc_ctx* ctx, Workspace& ws, const KronOp<W>& H, int b, int k_conv, const int* d_idx,
                 double ub, double tol, int max_iter, W* X, W* HX, W* theta, int* iters_out, bool* converged,
                 bool value_only = false) {
  const long n = H.n();
  W *Y0, *Y1, *Y2, *Tbuf, *G, *Z, *tmp;
  double* rn;
  TRY(ws.get(&Y0, (size_t)b * n));
  TRY(ws.get(&Y1, (size_t)b * n));
  TRY(ws.get(&Y2, (size_t)b * n));
  TRY(ws.get(&tmp, (size_t)b * n));
  TRY(ws.get(&Tbuf, (size_t)std::max(1, H.n_ops) * b * n));
  TRY(ws.get(&G, (size_t)b * b));
  TRY(ws.get(&Z, (size_t)b * b));
  TRY(ws.get(&rn, (size_t)b));
  const bool fp64 = sizeof(W) == 8;
  const double rho = fp64 ? 1e6 : 1e3;  // cap on the filter's amplification ratio
  const int dmax = 40;

  start_vectors_kernel<W><<<grid1d((long)b * n), 256, 0, ctx->stream>>>(d_idx, b, n, kStartAmp / std::sqrt((double)n), X);
  CKL();
  auto rayleigh_ritz = [&]() -> rmc_status {
    Workspace wl(ctx);
    TRY(kron_product<W>(ctx, H, X, b, HX, Tbuf));
    TRY(gram<W>(ctx, wl, X, b, HX, b, n, G, true));
    if (fp64) {
      double* w64 = (double*)(void*)theta;
      TRY(syev64(ctx, wl, (const double*)(const void*)G, b, w64, (double*)(void*)Z));
    } else {
      TRY((jacobi<W, W>(ctx, G, b, theta, Z)));
    }
    TRY(combine<W>(ctx, Z, true, b, b, X, n, tmp, W(1), W(0), nullptr));
    std::swap(X, tmp);
    TRY(combine<W>(ctx, Z, true, b, b, HX, n, tmp, W(1), W(0), nullptr));
    std::swap(HX, tmp);
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    residual_kernel<W><<<b, 256, 0, ctx->stream>>>(X, HX, theta, n, k_conv, tol, rn, ctx->d_status);
    CKL();
    return RMC_OK;
  };
  W* X_orig = X;
  W* HX_orig = HX;
  TRY(rayleigh_ritz());
  std::vector<double> th(b), r(b);
  StallGuard stall;
  int it = 0, steady = 0;
  double th0_prev = NAN;
  *converged = false;
  for (;; ++it) {
    int fails = 0;
    TRY(read_status(ctx, &fails, 1));
    TRY(to_host<W>(ctx, theta, th.data(), b));
    // value_only: the caller needs the lowest Ritz value alone, which
    // converges quadratically in the residual; inside a tight cluster the
    // Ritz vectors (and their residuals) settle much later than the value,
    // so a value unchanged to 1e-13 over three iterations counts as converged
    if (value_only) {
      steady = std::fabs(th[0] - th0_prev) <= 1e-13 * std::max(1.0, std::fabs(th[0])) ? steady + 1 : 0;
      th0_prev = th[0];
      if (steady >= 3) fails = 0;
    }
    double worst = 0;
    int wi = 0;
    if (ctx->trace || (!fp64 && fails > 0)) {
      TRY(to_host<double>(ctx, rn, r.data(), b));
      worst = worst_relative(r, th, k_conv, &wi);
    }
    if (ctx->trace)
      fprintf(stderr, "[rmc] n=%ld b=%d it=%d fails=%d worst i=%d res=%.3e theta=%.12g th0=%.12g thb=%.12g\n", n, b, it,
              fails, wi, worst, th[wi], th[0], th[b - 1]);
    if (fails == 0) { *converged = true; break; }
    if (!fp64 && stall.at_floor(worst, tol)) { *converged = true; break; }
    if (it >= max_iter) break;
    ctx->iterations++;
    const double a = th[b - 1];
    const double e = (ub - a) / 2, c = (ub + a) / 2;
    if (!(e > 0)) break;
    const double x0 = std::fabs((th[0] - c) / e);
    int deg = (int)std::floor(std::acosh(rho) / std::acosh(std::max(x0, 1.0 + 1e-12)));
    deg = std::max(2, std::min(dmax, deg));
    // X <- normalised filter output (one fused launch when the block fits),
    // then orthonormalised
    bool fused = false;
    TRY(cheb_fused<W>(ctx, H, X, HX, b, deg, th[0], a, ub, X, &fused));
    if (!fused) {
      W* Yout = nullptr;
      TRY((cheb_filter<W>(ctx, H, X, HX, b, th[0], a, ub, deg, Y0, Y1, Y2, Tbuf, &Yout)));
      CK(cudaMemcpyAsync(X, Yout, sizeof(W) * b * n, cudaMemcpyDeviceToDevice, ctx->stream));
      normalize_kernel<W><<<b, 256, 0, ctx->stream>>>(X, n, nullptr);
      CKL();
    }
    {
      Workspace wl(ctx);
      TRY(cholqr<W>(ctx, wl, X, b, n, tmp, fp64 ? 1e-14 : 1e-6));
    }
    TRY(rayleigh_ritz());
  }
  // results must end up in the caller's buffers
  if (X != X_orig) CK(cudaMemcpyAsync(X_orig, X, sizeof(W) * b * n, cudaMemcpyDeviceToDevice, ctx->stream));
  if (HX != HX_orig) CK(cudaMemcpyAsync(HX_orig, HX, sizeof(W) * b * n, cudaMemcpyDeviceToDevice, ctx->stream));
  *iters_out = it;
  return RMC_OK;
}


// X_a <- X_a - X_l^T (X_l X_a^T)^T, `passes` times: remove the span of the nl
// locked vectors X_l from the na vectors X_a (classical Gram-Schmidt; two
// passes unless the caller repeats it anyway).
template <typename W>
rmc_status project_out(rmc_ctx* ctx, const W* Xl, int nl, W* Xa, int na, long n, W* C, int passes) {
  if (nl <= 0) return RMC_OK;
  for (int pass = 0; pass < passes; ++pass) {
    Workspace wl(ctx);
    TRY(gram<W>(ctx, wl, Xl, nl, Xa, na, n, C, false));   // C[i][j] = <x_l_i, x_a_j>
    TRY(combine<W>(ctx, C, true, na, nl, Xl, n, Xa, W(-1), W(1), Xa));
  }
  return RMC_OK;
}

// Chebyshev-filtered subspace iteration with locking, for blocks wider than
// the small eigensolver: the lowest k_conv eigenpairs are found `chunk` at a
// time, each chunk in the orthogonal complement of the pairs already locked,
// with an active block of at most kMaxSmallDim vectors (chunk + 48 guard: on
// the 65536-row merges of k = 256 a 112 + 48 split took 11 % fewer
// iterations than 128 + 32, and 96 + 64 no fewer than 112 + 48).
// On return the first k_conv rows of X are the locked Ritz vectors and the
// rest (up to b_total) the last chunk's guard vectors; theta holds all b_total
// Ritz values.
template <typename W>
rmc_status chfsi_locked(rmc_ctx* ctx, Workspace& ws, const KronOp<W>& H, int b_total, int k_conv, const int* d_idx,
                        double ub, double tol, int max_iter, W* X, W* HX, W* theta, int* iters_out, bool* converged) {
  const long n = H.n();
  constexpr int kGuard = 48;
  const int chunk = kMaxSmallDim - kGuard;
  const int bmax = kMaxSmallDim;
  W *Y0, *Y1, *Y2, *Tbuf, *G, *Z, *tmp, *C;
  double* rn;
  TRY(ws.get(&Y0, (size_t)bmax * n));
  TRY(ws.get(&Y1, (size_t)bmax * n));
  TRY(ws.get(&Y2, (size_t)bmax * n));
  TRY(ws.get(&tmp, (size_t)bmax * n));
  TRY(ws.get(&Tbuf, (size_t)std::max(1, H.n_ops) * bmax * n));
  TRY(ws.get(&G, (size_t)bmax * bmax));
  TRY(ws.get(&Z, (size_t)bmax * bmax));
  TRY(ws.get(&C, (size_t)b_total * bmax));
  TRY(ws.get(&rn, (size_t)bmax));
  const bool fp64 = sizeof(W) == 8;
  const double rho = fp64 ? 1e6 : 1e3;
  const int dmax = 40;
  start_vectors_kernel<W><<<grid1d((long)b_total * n), 256, 0, ctx->stream>>>(d_idx, b_total, n,
                                                                               kStartAmp / std::sqrt((double)n), X);
  CKL();
  *converged = true;
  int total_it = 0;
  double theta_lock = NAN;  // lowest locked Ritz value (the first chunk's first)
  for (int L = 0; L < k_conv;) {
    const int c = std::min(chunk, k_conv - L);
    const int ba = std::min(b_total - L, c + kGuard);
    W* Xa = X + (size_t)L * n;
    W* HXa = HX + (size_t)L * n;
    W* tha = theta + L;
    auto orthonormalise = [&]() -> rmc_status {
      TRY(project_out<W>(ctx, X, L, Xa, ba, n, C));
      normalize_kernel<W><<<ba, 256, 0, ctx->stream>>>(Xa, n, nullptr);
      CKL();
      Workspace wl(ctx);
      return cholqr<W>(ctx, wl, Xa, ba, n, tmp, fp64 ? 1e-14 : 1e-6);
    };
    auto rayleigh_ritz = [&]() -> rmc_status {
      Workspace wl(ctx);
      TRY(kron_work<W>(ctx, H, Xa, ba, HXa, W(1), W(0), W(0), nullptr, Tbuf));
      TRY(gram<W>(ctx, wl, Xa, ba, HXa, ba, n, G, true));
      if (fp64) {
        TRY(syev64(ctx, wl, (const double*)(const void*)G, ba, (double*)(void*)tha, (double*)(void*)Z));
      } else {
        TRY((jacobi<W, W>(ctx, G, ba, tha, Z)));
      }
      TRY(combine<W>(ctx, Z, true, ba, ba, Xa, n, tmp, W(1), W(0), nullptr));
      CK(cudaMemcpyAsync(Xa, tmp, sizeof(W) * ba * n, cudaMemcpyDeviceToDevice, ctx->stream));
      TRY(combine<W>(ctx, Z, true, ba, ba, HXa, n, tmp, W(1), W(0), nullptr));
      CK(cudaMemcpyAsync(HXa, tmp, sizeof(W) * ba * n, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
      residual_kernel<W><<<ba, 256, 0, ctx->stream>>>(Xa, HXa, tha, n, c, tol, rn, ctx->d_status);
      CKL();
      return RMC_OK;
    };
    TRY(orthonormalise());
    TRY(rayleigh_ritz());
    std::vector<double> th(ba), r(ba);
    StallGuard stall;
    for (int it = 0;; ++it) {
      int fails = 0;
      TRY(read_status(ctx, &fails, 1));
      TRY(to_host<W>(ctx, tha, th.data(), ba));
      double worst = 0;
      int wi = 0;
      if (ctx->trace || (!fp64 && fails > 0)) {
        TRY(to_host<double>(ctx, rn, r.data(), ba));
        worst = worst_relative(r, th, c, &wi);
      }
      if (ctx->trace)
        fprintf(stderr, "[rmc locked] n=%ld L=%d c=%d ba=%d it=%d fails=%d worst i=%d res=%.3e theta=%.12g\n", n, L, c,
                ba, it, fails, wi, worst, th[wi]);
      if (fails == 0) break;
      if (!fp64 && stall.at_floor(worst, tol)) break;
      if (it >= max_iter) { *converged = false; break; }
      ctx->iterations++;
      total_it++;
      const double a = th[ba - 1];
      const double e = (ub - a) / 2, cc = (ub + a) / 2;
      if (!(e > 0)) { *converged = false; break; }
      const double x0 = std::fabs((th[0] - cc) / e);
      int deg = (int)std::floor(std::acosh(rho) / std::acosh(std::max(x0, 1.0 + 1e-12)));
      deg = std::max(2, std::min(dmax, deg));
      W* Yout = nullptr;
      TRY((cheb_filter<W>(ctx, H, Xa, HXa, ba, th[0], a, ub, deg, Y0, Y1, Y2, Tbuf, &Yout, X, L, C,
                          L > 0 ? theta_lock : NAN)));
      CK(cudaMemcpyAsync(Xa, Yout, sizeof(W) * ba * n, cudaMemcpyDeviceToDevice, ctx->stream));
      TRY(orthonormalise());
      TRY(rayleigh_ritz());
    }
    if (!*converged) break;
    if (L == 0) theta_lock = th[0];
    L += c;
  }
  *iters_out = total_it;
  return RMC_OK;
}

template <typename W>
rmc_status prepare_kron(rmc_ctx* ctx, Workspace& ws, const MergeInput& in, KronOp<W>* H) {
  const rmc_block* A = in.A;
  const rmc_block* B = in.B;
  const int kA = A->k, kB = B->k, no = (int)in.terms.size();
  H->kA = kA;
  H->kB = kB;
  H->n_ops = no;
  W *EA, *EB, *Araw, *Acat, *Bcat;
  TRY(ws.get(&EA, kA));
  TRY(ws.get(&EB, kB));
  TRY(ws.get(&Araw, (size_t)std::max(1, no) * kA * kA));
  TRY(ws.get(&Acat, (size_t)std::max(1, no) * kA * kA));
  TRY(ws.get(&Bcat, (size_t)std::max(1, no) * kB * kB));
  convert_kernel<W, double><<<grid1d(kA), 256, 0, ctx->stream>>>(A->E, EA, kA);
  CKL();
  convert_kernel<W, double><<<grid1d(kB), 256, 0, ctx->stream>>>(B->E, EB, kB);
  CKL();
  Coefs cf{};
  for (int j = 0; j < no; ++j) {
    const rmc_term& t = in.terms[j];
    cf.c[j] = t.coef;
    convert_kernel<W, double><<<grid1d((long)kA * kA), 256, 0, ctx->stream>>>(
        A->ops + (size_t)t.op_a * kA * kA, Araw + (size_t)j * kA * kA, (long)kA * kA);
    CKL();
    convert_kernel<W, double><<<grid1d((long)kB * kB), 256, 0, ctx->stream>>>(
        B->ops + (size_t)t.op_b * kB * kB, Bcat + (size_t)j * kB * kB, (long)kB * kB);
    CKL();
  }
  if (no > 0) {
    build_acat_kernel<W><<<grid1d((long)kA * kA * no), 256, 0, ctx->stream>>>(Araw, cf, kA, no, Acat);
    CKL();
  }
  H->EA = EA;
  H->EB = EB;
  H->Acat = Acat;
  H->Bcat = Bcat;
  return RMC_OK;
}

// FP64 refinement of a wide block (more vectors than the small eigensolver
// takes) in defect form, for the mixed paths.
//
// The iterate is C (FP64, orthonormal Ritz vectors, Ritz values theta)
// together with its FP64-accurate product HC.  A Chebyshev filter pass (the
// scaled recurrence of cheb_filter, bounds from the current Ritz values)
// applied to C splits exactly into
//     p(H) C = C diag(y(theta)) + D,
// where y_d is the same three-term recurrence evaluated at the Ritz values and
// the defect D obeys
//     D_1 = (s_1/e) R,
//     D_d = (2 s_d/e)(H - c) D_{d-1} - s_{d-1} s_d D_{d-2} + (2 s_d/e) R diag(y_{d-1})
// with R = HC - C diag(theta) the Ritz residuals.  D is as small as R, so its
// products run in FP32 (an FP32 rounding relative to D is ~1e-7 of R, far
// below the FP64 target).
//
// The new basis is Q = C + E with E = D_perp diag(1/y), where D = C G1 + D_perp
// (G1 = C^T D, D_perp outside span C): each column gains the part of its
// filtered image outside the current span, relative to its own amplification
// -- the subspace-iteration step, with the in-span mixing of the filtered
// columns left to the Rayleigh-Ritz step.  (Forming span(X) exactly would
// need A^{-1} for A = diag(y) + G1, which is ill-conditioned for the guard
// columns at the bottom of the filter, where y ~ 1/kDefectRho; a
// Newton-Schulz inverse diverged there and stalled two merges.)  E is as small
// as the subspace still moves, up to ~2x a guard column's current error.  Then,
// with H E an FP32 product,
//     Q^T Q = I + C^T E + E^T C + E^T E,
//     Q^T H Q = diag(theta) + C^T R + C^T HE + E^T HC + E^T HE,
// and C^T HE = (HC)^T E = R^T E + diag(theta) C^T E.  C^T E is the one
// FP64-accurate Gram product of the pass: E is stored in FP32, and for the
// unconverged guard columns it is large (up to ~0.4), so its rounding has
// components along C of ~2e-8 that theta would magnify into the Rayleigh-Ritz
// matrix (measured: a residual floor of 2e-8 - 1.4e-7 on half the 65536-row
// merges when all Gram products were FP32).  C^T R, R^T E, E^T E and E^T HE
// involve a small factor, or carry a large error only in guard-guard entries,
// and stay FP32.  The generalised
// Rayleigh-Ritz problem is solved as W Q^T H Q W with W = (Q^T Q)^{-1/2}
// (a coupled Newton-Schulz iteration); its matrix is nearly diagonal, so the
// FP64 eigensolver starts from the identity.  With Z the
// combined rotation W Z~, the new iterate is C Z + E Z and its product
// HC Z + HE Z: C Z and HC Z are FP64-accurate combinations, E Z and HE Z FP32.
// A pass therefore costs FP32 Kronecker products on small data (tensor-core for
// the 256-state merges' filter; H E on the FP32 pipe, since it enters H C
// directly), FP32 Gram products, one FP64-accurate Gram product and two
// FP64-accurate combinations, where the earlier form of the pass took twelve
// FP64-accurate Gram and combination products; the merge's only FP64-accurate
// Kronecker product is the first one, of the working-precision block.
//
// After the first pass a pass works on the active columns only: the kept
// vectors that still fail the residual test and the guard columns.  Their
// defects are projected against the whole basis, so the active block Q_S is
// orthogonal to the fixed columns, whose coupling to it through H is second
// order (E_S^T R_fixed); the Rayleigh-Ritz step runs on span Q_S alone, and
// every product of the pass is sized by the active count (on the 65536-row
// merges about a third of the block on the second pass and an eighth after).
//
// The passes stop when the kept vectors pass the residual test, after
// max_passes, or after two passes in a row that did not halve the worst
// residual.
//
// The filter covers the whole block at once (no chunks); its amplification
// ratio is capped (kDefectRho) so that the guard columns' corrections stay
// moderate.  Each pass leaves C orthonormal to ~1e-11 (the FP32 parts of its
// corrections), so a last FP64 Cholesky-QR pass makes the returned basis
// orthonormal to FP64 rounding.
//
// On return C holds the Ritz vectors and w their values (ascending).  X, HX and HC are scratch (b x n FP64 each, HC also n_ops wide
// for the first product).
constexpr double kDefectRho = 1e5;
constexpr int kDefectMaxDeg = 40;
constexpr int kInvSqrtSteps = 10;
constexpr double kDefectBlowup = 100.0;  // a pass this much worse than the last is undone

rmc_status refine_wide_defect(rmc_ctx* ctx, Workspace& ws, const KronOp<double>& H64, const KronOp<float>& Hf, int b,
                              int k_acc, double ub, double tol, int max_passes, double* X, double* HX, double* C,
                              double* HC, double* G, double* w, double* Z, double* rn) {
  const long n = H64.n();
  const long tot = (long)b * n;
  const size_t bb = (size_t)b * b;
  float *Rf, *D0, *D1, *D2, *Tf, *sdev, *Cf, *E, *HE, *g32, *Af;
  double *ydev, *X1, *Tm, *S, *S2, *Wm, *Gm, *Gt, *Zt, *Zs;
  TRY(ws.get(&Rf, (size_t)tot));
  TRY(ws.get(&D0, (size_t)tot));
  TRY(ws.get(&D1, (size_t)tot));
  TRY(ws.get(&D2, (size_t)tot));
  TRY(ws.get(&Cf, (size_t)tot));
  TRY(ws.get(&E, (size_t)tot));
  TRY(ws.get(&HE, (size_t)tot));
  TRY(ws.get(&Tf, (size_t)std::max(1, Hf.n_ops) * tot));
  TRY(ws.get(&sdev, (size_t)kDefectMaxDeg * b));
  TRY(ws.get(&g32, 5 * bb));
  TRY(ws.get(&Af, bb));
  TRY(ws.get(&ydev, (size_t)b));
  double* cdev;
  TRY(ws.get(&cdev, 1));
  for (double** m : {&X1, &Tm, &S, &S2, &Wm, &Gm, &Gt, &Zt, &Zs}) TRY(ws.get(m, bb));
  float *G1 = g32, *SEE = g32 + bb, *CR = g32 + 2 * bb, *RE = g32 + 3 * bb, *EHE = g32 + 4 * bb;
  double* SCE;
  TRY(ws.get(&SCE, bb));
  double* const C_out = C;
  // FP64 Rayleigh-Ritz of the working-precision block: the one FP64-accurate
  // Kronecker product (HC serves as its scratch before it holds H C)
  TRY(cholqr64_refine(ctx, ws, X, b, n, C));
  TRY(kron_product<double>(ctx, H64, X, b, HX, HC));
  TRY(gram<double>(ctx, ws, X, b, HX, b, n, G, true));
  TRY(syev64(ctx, ws, G, b, w, Z, true));
  TRY(combine<double>(ctx, Z, true, b, b, X, n, C, 1.0, 0.0, nullptr));
  TRY(combine<double>(ctx, Z, true, b, b, HX, n, HC, 1.0, 0.0, nullptr));
  // A pass refines only the active columns: the kept vectors that still fail
  // the residual test and the guard columns (the rest stay as they are).
  // Their corrections are projected against the whole basis C, so Q_S =
  // C_S + E_S is orthogonal to the fixed columns, which are Ritz vectors with
  // residuals below tol: the coupling Q_S^T H C_fixed = E_S^T R_fixed is
  // second order, and the Rayleigh-Ritz step is taken on span Q_S alone.
  // Columns keep their physical slots; the order by Ritz value is taken on
  // the host each pass and made physical at the end.
  std::vector<double> th(b), y0(b), y1(b), y2(b), r(b), tha(b);
  std::vector<float> sc((size_t)kDefectMaxDeg * b);
  std::vector<int> order(b), act;
  int* act_dev;
  double *Cs, *HCs, *wa;
  TRY(ws.get(&act_dev, (size_t)b));
  TRY(ws.get(&Cs, (size_t)tot));
  TRY(ws.get(&HCs, (size_t)tot));
  TRY(ws.get(&wa, (size_t)b));
  float* Cfs;
  TRY(ws.get(&Cfs, (size_t)tot));
  auto sorted_order = [&]() {
    for (int i = 0; i < b; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return th[x] < th[y]; });
  };
  auto failing = [&](int i) { return !(r[i] <= tol * std::max(1.0, std::fabs(th[i]))); };
  double prev_worst = 1e300;
  int stalled = 0;
  for (int pass = 0;; ++pass) {
    residual_kernel<double><<<b, 256, 0, ctx->stream>>>(C, HC, w, n, 0, tol, rn, ctx->d_status);
    CKL();
    TRY(to_host<double>(ctx, w, th.data(), b));
    TRY(to_host<double>(ctx, rn, r.data(), b));
    sorted_order();
    int fails = 0, wi = order[0];
    double worst = 0.0;
    for (int pos = 0; pos < k_acc; ++pos) {
      const int i = order[pos];
      const double v = r[i] / std::max(1.0, std::fabs(th[i]));
      if (failing(i)) ++fails;
      if (v > worst) { worst = v; wi = i; }
    }
    if (ctx->trace)
      fprintf(stderr, "[rmc refine defect] n=%ld b=%d pass=%d fails=%d worst res=%.3e theta=%.12g thb=%.12g\n", n, b,
              pass, fails, worst, th[wi], th[order[b - 1]]);
    // a pass that made the worst residual far larger (its Rayleigh-Ritz
    // basis lost a direction: seen once on a 65280-row merge whose guard
    // columns' corrections were large) is undone: the previous active
    // columns, their products and Ritz values go back to their slots
    // (they are still in Cs, HCs, tha and act_dev), and the refinement ends
    if (pass > 0 && worst > kDefectBlowup * prev_worst) {
      const int na = (int)act.size();
      scatter_rows_kernel<double><<<rows_grid(n, na), 256, 0, ctx->stream>>>(Cs, act_dev, n, C);
      CKL();
      scatter_rows_kernel<double><<<rows_grid(n, na), 256, 0, ctx->stream>>>(HCs, act_dev, n, HC);
      CKL();
      CK(cudaMemcpyAsync(wa, tha.data(), sizeof(double) * na, cudaMemcpyHostToDevice, ctx->stream));
      scatter_values_kernel<<<ceil_div(na, 256), 256, 0, ctx->stream>>>(wa, act_dev, na, w);
      CKL();
      CK(cudaStreamSynchronize(ctx->stream));  // tha is pageable host memory
      if (ctx->trace) fprintf(stderr, "[rmc refine defect] n=%ld pass=%d undone (worst %.3e)\n", n, pass, worst);
      break;
    }
    if (fails == 0 || pass >= max_passes) break;
    // two passes in a row without halving the worst residual: the remaining
    // vectors converge too slowly to be worth more passes (the energies they
    // feed into are second order in their residual)
    stalled = (pass > 0 && worst > 0.5 * prev_worst) ? stalled + 1 : 0;
    if (stalled >= 2) break;
    prev_worst = worst;
    act.clear();
    for (int pos = 0; pos < b; ++pos)
      if (pos >= k_acc || failing(order[pos])) act.push_back(order[pos]);
    std::sort(act.begin(), act.end());
    const int na = (int)act.size();
    const long tota = (long)na * n;
    const double a = th[order[b - 1]], e = (ub - a) / 2, c = (ub + a) / 2;
    if (!(e > 0)) break;
    const double tlo = th[order[0]];
    const double x0 = std::fabs((tlo - c) / e);
    int deg = (int)std::floor(std::acosh(kDefectRho) / std::acosh(std::max(x0, 1.0 + 1e-12)));
    deg = std::max(2, std::min(kDefectMaxDeg, deg));
    // scalar recurrence at the active Ritz values and their source scales
    double sigma = e / (tlo - c);
    const double tau = 2.0 / sigma;
    for (int j = 0; j < na; ++j) {
      tha[j] = th[act[j]];
      y0[j] = 1.0;
      y1[j] = sigma / e * (tha[j] - c);
    }
    std::vector<double> s_of(deg + 1);
    for (int d = 2; d <= deg; ++d) {
      const double s1 = 1.0 / (tau - sigma);
      for (int j = 0; j < na; ++j) {
        sc[(size_t)(d - 2) * na + j] = (float)(2 * s1 / e * y1[j]);
        y2[j] = 2 * s1 / e * (tha[j] - c) * y1[j] - sigma * s1 * y0[j];
      }
      std::swap(y0, y1);
      std::swap(y1, y2);
      s_of[d] = s1;
      sigma = s1;
    }
    // (pageable sources: the copies are staged before the calls return)
    CK(cudaMemcpyAsync(sdev, sc.data(), sizeof(float) * (size_t)(deg - 1) * na, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ydev, y1.data(), sizeof(double) * na, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(wa, tha.data(), sizeof(double) * na, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(act_dev, act.data(), sizeof(int) * na, cudaMemcpyHostToDevice, ctx->stream));
    // the active columns, FP32 copies, residuals and the defect recurrence
    gather_rows_kernel<double><<<rows_grid(n, na), 256, 0, ctx->stream>>>(C, act_dev, n, Cs);
    CKL();
    gather_rows_kernel<double><<<rows_grid(n, na), 256, 0, ctx->stream>>>(HC, act_dev, n, HCs);
    CKL();
    convert_kernel<float, double><<<grid1d(tot), 256, 0, ctx->stream>>>(C, Cf, tot);
    CKL();
    convert_kernel<float, double><<<grid1d(tota), 256, 0, ctx->stream>>>(Cs, Cfs, tota);
    CKL();
    ritz_residual_kernel<<<rows_grid(n, na), 256, 0, ctx->stream>>>(Cs, HCs, wa, n, Rf);
    CKL();
    CK(cudaMemsetAsync(D0, 0, sizeof(float) * tota, ctx->stream));
    sigma = e / (tlo - c);
    axpby_kernel<float><<<grid1d(tota), 256, 0, ctx->stream>>>(Rf, Rf, tota, (float)(sigma / e), 0.0f, D1);
    CKL();
    float *Dp = D0, *Dc = D1, *Dn = D2;
    for (int d = 2; d <= deg; ++d) {
      const double s1 = s_of[d];
      TRY(kron_work<float>(ctx, Hf, Dc, na, Dn, (float)(2 * s1 / e), (float)(-2 * s1 * c / e), (float)(-sigma * s1), Dp,
                           Tf));
      add_scaled_columns_kernel<<<rows_grid(n, na), 256, 0, ctx->stream>>>(Dn, Rf, sdev + (size_t)(d - 2) * na, n);
      CKL();
      float* t = Dp;
      Dp = Dc;
      Dc = Dn;
      Dn = t;
      sigma = s1;
    }
    // D = C G1 + D_perp (in place, against the whole basis), E = D_perp diag(1/y)
    {
      Workspace wl(ctx);
      TRY(gram<float>(ctx, wl, Cf, b, Dc, na, n, G1, false));
      TRY(combine<float>(ctx, G1, true, na, b, Cf, n, Dc, -1.0f, 1.0f, Dc));
      TRY(gram<float>(ctx, wl, Cfs, na, Rf, na, n, CR, false));
    }
    scale_columns_inv_kernel<<<rows_grid(n, na), 256, 0, ctx->stream>>>(Dc, ydev, n, E);
    CKL();
    // H E on the FP32 pipe, not in 3xTF32: it enters the new H C directly, and
    // the large corrections of the guard columns would carry the tensor-core
    // form's ~5e-7 relative error into the kept vectors through the rotation
    TRY(kron_apply<float>(ctx, Hf, E, na, HE, 1.0f, 0.0f, 0.0f, nullptr, Tf));
    {
      Workspace wl(ctx);
      convert_kernel<double, float><<<grid1d(tota), 256, 0, ctx->stream>>>(E, X, tota);  // E exactly, in FP64
      CKL();
      TRY(gram<double>(ctx, wl, Cs, na, X, na, n, SCE, false));
      TRY(gram<float>(ctx, wl, E, na, E, na, n, SEE, true));
      TRY(gram<float>(ctx, wl, Rf, na, E, na, n, RE, false));
      TRY(gram<float>(ctx, wl, E, na, HE, na, n, EHE, false));
    }
    const size_t aa = (size_t)na * na;
    defect_gram_kernel<<<grid1d((long)aa), 256, 0, ctx->stream>>>(SCE, SEE, CR, RE, EHE, wa, na, S, Gm);
    CKL();
    // W = (I + S)^{-1/2} by the coupled Newton-Schulz iteration on (I + S)/c
    // (Y -> its square root, W -> its inverse square root; the corrections of
    // unconverged guard columns make S far from small, so the spectrum is
    // first scaled into [1/c, 1]); Gt = W Gm W; its eigenpairs; Z = W Zt
    ns_start_kernel<<<1, 1024, 0, ctx->stream>>>(S, SEE, na, Gt, cdev);   // Y0 = (I + S) / c
    CKL();
    shifted_identity_kernel<<<grid1d((long)aa), 256, 0, ctx->stream>>>(nullptr, na, 1.0, 0.0, Wm);  // W0 = I
    CKL();
    for (int it = 0; it < kInvSqrtSteps; ++it) {
      TRY((small_mm_skip<false, false>(ctx, Wm, Gt, na, S2, 0.0, nullptr, nullptr, -0.5)));  // -W Y / 2
      shifted_identity_kernel<<<grid1d((long)aa), 256, 0, ctx->stream>>>(S2, na, 1.5, 1.0, S2);  // T = 3/2 I - W Y / 2
      CKL();
      TRY((small_mm_skip<false, false>(ctx, Gt, S2, na, Tm, 0.0, nullptr, nullptr, 1.0)));  // Y T
      TRY((small_mm_skip<false, false>(ctx, S2, Wm, na, X1, 0.0, nullptr, nullptr, 1.0)));  // T W
      std::swap(Gt, Tm);
      std::swap(Wm, X1);
    }
    scale_inv_sqrt_kernel<<<grid1d((long)aa), 256, 0, ctx->stream>>>(Wm, na, cdev);
    CKL();
    TRY((small_mm_skip<false, false>(ctx, Wm, Gm, na, Tm, 0.0, nullptr, nullptr, 1.0)));
    TRY((small_mm_skip<false, false>(ctx, Tm, Wm, na, Gt, 0.0, nullptr, nullptr, 1.0)));
    TRY(syev64(ctx, ws, Gt, na, wa, Zt, true));
    TRY((small_mm_skip<false, false>(ctx, Wm, Zt, na, Zs, 0.0, nullptr, nullptr, 1.0)));
    // new active columns: C_S Z + E Z and HC_S Z + HE Z (FP64-accurate
    // combinations of the O(1) parts, FP32 of the small ones), back to their slots
    TRY(combine<double>(ctx, Zs, true, na, na, Cs, n, X, 1.0, 0.0, nullptr));
    TRY(combine<double>(ctx, Zs, true, na, na, HCs, n, HX, 1.0, 0.0, nullptr));
    convert_kernel<float, double><<<grid1d((long)aa), 256, 0, ctx->stream>>>(Zs, Af, (long)aa);
    CKL();
    TRY(combine<float>(ctx, Af, true, na, na, E, n, D0, 1.0f, 0.0f, nullptr));
    TRY(combine<float>(ctx, Af, true, na, na, HE, n, D1, 1.0f, 0.0f, nullptr));
    add_f32_kernel<<<grid1d(tota), 256, 0, ctx->stream>>>(X, D0, tota);
    CKL();
    add_f32_kernel<<<grid1d(tota), 256, 0, ctx->stream>>>(HX, D1, tota);
    CKL();
    scatter_rows_kernel<double><<<rows_grid(n, na), 256, 0, ctx->stream>>>(X, act_dev, n, C);
    CKL();
    scatter_rows_kernel<double><<<rows_grid(n, na), 256, 0, ctx->stream>>>(HX, act_dev, n, HC);
    CKL();
    scatter_values_kernel<<<ceil_div(na, 256), 256, 0, ctx->stream>>>(wa, act_dev, na, w);
    CKL();
  }
  // the Ritz pairs in ascending order
  TRY(to_host<double>(ctx, w, th.data(), b));
  sorted_order();
  bool permuted = false;
  for (int i = 0; i < b; ++i) permuted |= order[i] != i;
  if (permuted) {
    for (int i = 0; i < b; ++i) tha[i] = th[order[i]];
    CK(cudaMemcpyAsync(act_dev, order.data(), sizeof(int) * b, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(w, tha.data(), sizeof(double) * b, cudaMemcpyHostToDevice, ctx->stream));
    gather_rows_kernel<double><<<rows_grid(n, b), 256, 0, ctx->stream>>>(C, act_dev, n, X);
    CKL();
    CK(cudaMemcpyAsync(C, X, sizeof(double) * tot, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  // the basis to FP64 orthonormality (each pass left it within ~1e-11)
  TRY(cholqr64_refine(ctx, ws, C, b, n, X, 1));
  if (C != C_out) CK(cudaMemcpyAsync(C_out, C, sizeof(double) * tot, cudaMemcpyDeviceToDevice, ctx->stream));
  return RMC_OK;
}

template <typename W>
rmc_status couple_impl(rmc_ctx* ctx, const MergeInput& in, rmc_block** out, rmc_status* soft) {
  Workspace ws(ctx);
  const rmc_block* A = in.A;
  const rmc_block* B = in.B;
  const int kA = A->k, kB = B->k, no = (int)in.terms.size();
  const long n = (long)kA * kB;
  const int k_ret = (int)std::min<long>(in.k_keep, n);
  int g = ctx->cfg.guard > 0 ? ctx->cfg.guard : std::max(16, k_ret / 2);
  int b = (int)std::min<long>(n, (long)k_ret + g);
  // Blocks wider than the small eigensolver are solved with locking, chunk by
  // chunk, with a 32-vector guard after the wanted ones.
  // Single block whenever the wanted vectors and a guard of at least 16 fit
  // (the guard shrinks to what is left); otherwise locking, chunk by chunk.
  const int want = in.top ? k_ret : k_ret + 1;
  const bool chunked = b > kMaxSmallDim && (long)want + 16 > kMaxSmallDim && n > kMaxSmallDim;
  if (chunked) b = (int)std::min<long>(n, (long)k_ret + 1 + 31);
  else b = std::min(b, kMaxSmallDim);
  if (!chunked && b < want && b < n)
    return fail(ctx, RMC_ERR_INVAL, "kept count %d does not fit the solver block", k_ret);
  if (b > 1024) return fail(ctx, RMC_ERR_INVAL, "kept count %d exceeds the solver limit of 992", k_ret);
  const int k_conv = std::min(b, in.top ? k_ret : k_ret + 1);

  // FP64 operator copies for the diagonal, the finalisation and the rotation
  KronOp<double> H64;
  TRY(prepare_kron<double>(ctx, ws, in, &H64));
  double* D;
  int* idx;
  double* dmm;
  TRY(ws.get(&D, n));
  TRY(ws.get(&idx, b));
  TRY(ws.get(&dmm, 2));
  {
    Coefs cf{};
    double *Ad, *Bd;
    TRY(ws.get(&Ad, (size_t)std::max(1, no) * kA * kA));
    TRY(ws.get(&Bd, (size_t)std::max(1, no) * kB * kB));
    for (int j = 0; j < no; ++j) {
      cf.c[j] = in.terms[j].coef;
      CK(cudaMemcpyAsync(Ad + (size_t)j * kA * kA, A->ops + (size_t)in.terms[j].op_a * kA * kA,
                         sizeof(double) * kA * kA, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(cudaMemcpyAsync(Bd + (size_t)j * kB * kB, B->ops + (size_t)in.terms[j].op_b * kB * kB,
                         sizeof(double) * kB * kB, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    diag_kernel<<<grid1d(n), 256, 0, ctx->stream>>>(A->E, B->E, Ad, Bd, cf, no, kA, kB, D);
    CKL();
    select_smallest_kernel<<<1, 1024, 0, ctx->stream>>>(D, n, b, idx, dmm);
    CKL();
  }
  double hdmm[2];
  TRY(to_host<double>(ctx, dmm, hdmm, 2));
  double ub = hdmm[1];
  for (int j = 0; j < no; ++j) {
    const rmc_term& t = in.terms[j];
    ub += std::fabs(t.coef) * A->opnorm[t.op_a] * B->opnorm[t.op_b];
  }
  ub += 1e-12 * std::max(1.0, std::fabs(ub));

  double *X64, *HX64, *tmp64, *Tb64;
  TRY(ws.get(&X64, (size_t)b * n));
  TRY(ws.get(&HX64, (size_t)b * n));
  TRY(ws.get(&tmp64, (size_t)b * n));
  TRY(ws.get(&Tb64, (size_t)std::max(1, no) * b * n));
  bool converged = true;
  int iters = 0;
  std::vector<double> th_work;  // working-precision Ritz values (mixed paths)
  KronOp<W> Hw;                 // working-precision operator (mixed paths)
  const bool dense = (b == n) && !chunked;
  if (dense) {
    CK(cudaMemsetAsync(X64, 0, sizeof(double) * b * n, ctx->stream));
    unit_vectors_kernel<double><<<ceil_div(b, 128), 128, 0, ctx->stream>>>(idx, b, n, X64);
    CKL();
  } else {
    const double tol = ctx->cfg.tol;
    if (sizeof(W) == 8) {
      double* th;
      TRY(ws.get(&th, b));
      if (chunked)
        TRY((chfsi_locked<double>(ctx, ws, H64, b, k_conv, idx, ub, tol, ctx->cfg.max_iter, X64, HX64, th, &iters,
                                  &converged)));
      else
        TRY((chfsi<double>(ctx, ws, H64, b, k_conv, idx, ub, tol, ctx->cfg.max_iter, X64, HX64, th, &iters,
                           &converged)));
    } else {
      TRY(prepare_kron<W>(ctx, ws, in, &Hw));
      W *Xw, *HXw, *thw;
      TRY(ws.get(&Xw, (size_t)b * n));
      TRY(ws.get(&HXw, (size_t)b * n));
      TRY(ws.get(&thw, b));
      const double tolw = ctx->cfg.precision == RMC_PREC_FP64 ? tol : std::max(tol, 2e-6);
      if (chunked)
        TRY((chfsi_locked<W>(ctx, ws, Hw, b, k_conv, idx, ub, tolw, ctx->cfg.max_iter, Xw, HXw, thw, &iters,
                             &converged)));
      else
        TRY((chfsi<W>(ctx, ws, Hw, b, k_conv, idx, ub, tolw, ctx->cfg.max_iter, Xw, HXw, thw, &iters, &converged)));
      convert_kernel<double, W><<<grid1d((long)b * n), 256, 0, ctx->stream>>>(Xw, X64, (long)b * n);
      CKL();
      th_work.resize(b);
      TRY(to_host<W>(ctx, thw, th_work.data(), b));
    }
  }
  // FP64 finalisation: orthonormalise, project, refined small eigensolve, on
  // the whole block (the guard vectors improve the Rayleigh-Ritz extraction of
  // the wanted subspace: restricting it to the wanted vectors cost accuracy).
  //
  // Mixed paths: FP64 refinement of the working-precision subspace, repeated
  // until the FP64 residuals of the wanted vectors are below kRefineTol
  // relative (at most kRefinePasses passes).  A pass is one FP64 Chebyshev
  // filter pass (bounds from the current Ritz values), the FP64 Cholesky-QR
  // and the FP64 Rayleigh-Ritz.  A single block is filtered whole, with the
  // degree for an amplification ratio of 1e6 (at most 16): the wanted vectors
  // nearest the guard then gain ~1e3 over the damped interval in one pass,
  // and the FP64 factorisation of cholqr64_refine absorbs the conditioning
  // this leaves in the guard columns.  A locked block is filtered chunk by chunk (at most 128
  // vectors, degree for 1e6, at most 12) on the operator deflated by the
  // earlier chunks, and each chunk is orthonormalised against them and
  // rotated to its own Ritz vectors, so the global Rayleigh-Ritz is nearly
  // diagonal and its eigensolver starts from the identity.  The FP64 path of
  // a locked block takes the chunk orthonormalisation once, without filter.
  const int bf = b;
  constexpr int kRefinePasses = 4;
  constexpr int kDefectPasses = 8;
  constexpr double kRefineTol = 1e-8;
  const bool refine = sizeof(W) == 4 && !dense && th_work.size() == (size_t)bf;
  std::vector<double> th_cur = th_work;
  double *Gs, *w, *Zs, *rn64;
  TRY(ws.get(&Gs, (size_t)bf * bf));
  TRY(ws.get(&w, bf));
  TRY(ws.get(&Zs, (size_t)bf * bf));
  TRY(ws.get(&rn64, bf));
  double* C = tmp64;
  const int k_acc = std::min(k_conv, k_ret);
  bool defect_done = false;
  if constexpr (sizeof(W) == 4) {
    if (chunked && refine) {
      // wide block: refinement in defect form (FP32 products on the small
      // defect, FP64-accurate Gram and combination GEMMs)
      TRY(refine_wide_defect(ctx, ws, H64, Hw, bf, k_acc, ub, kRefineTol, kDefectPasses, X64, HX64, C, Tb64, Gs, w,
                             Zs, rn64));
      defect_done = true;
    }
  }
  for (int pass = 0; !defect_done; ++pass) {
    if (chunked) {
      const int cw = 128;
      Workspace wc(ctx);
      double *Y0, *Y1, *Y2, *Cp, *Gc, *Zc, *wcv;
      TRY(wc.get(&Y0, (size_t)cw * n));
      TRY(wc.get(&Y1, (size_t)cw * n));
      TRY(wc.get(&Y2, (size_t)cw * n));
      TRY(wc.get(&Cp, (size_t)bf * cw));
      TRY(wc.get(&Gc, (size_t)cw * cw));
      TRY(wc.get(&Zc, (size_t)cw * cw));
      TRY(wc.get(&wcv, cw));
      for (int s0 = 0; s0 < bf; s0 += cw) {
        const int nc = std::min(cw, bf - s0);
        double* Xc = X64 + (size_t)s0 * n;
        if (refine && nc >= 2) {
          const double a = th_cur[s0 + nc - 1], e = (ub - a) / 2, cc = (ub + a) / 2;
          if (e > 0) {
            const double x0 = std::fabs((th_cur[s0] - cc) / e);
            int deg = (int)std::floor(std::acosh(1e6) / std::acosh(std::max(x0, 1.0 + 1e-12)));
            deg = std::max(2, std::min(12, deg));
            double* Yout = nullptr;
            TRY(kron_apply<double>(ctx, H64, Xc, nc, HX64, 1.0, 0.0, 0.0, nullptr, Tb64));
            TRY((cheb_filter<double>(ctx, H64, Xc, HX64, nc, th_cur[s0], a, ub, deg, Y0, Y1, Y2, Tb64, &Yout, X64,
                                     s0, Cp)));
            CK(cudaMemcpyAsync(Xc, Yout, sizeof(double) * nc * n, cudaMemcpyDeviceToDevice, ctx->stream));
          }
        }
        if (refine || pass == 0) {
          TRY(project_out<double>(ctx, X64, s0, Xc, nc, n, Cp));
          normalize_kernel<double><<<nc, 256, 0, ctx->stream>>>(Xc, n, nullptr);
          CKL();
          TRY(cholqr<double>(ctx, wc, Xc, nc, n, tmp64, 1e-14));
          TRY(kron_product<double>(ctx, H64, Xc, nc, HX64, Tb64));
          TRY(gram<double>(ctx, wc, Xc, nc, HX64, nc, n, Gc, true));
          TRY(syev64(ctx, wc, Gc, nc, wcv, Zc));
          TRY(combine<double>(ctx, Zc, true, nc, nc, Xc, n, tmp64, 1.0, 0.0, nullptr));
          CK(cudaMemcpyAsync(Xc, tmp64, sizeof(double) * nc * n, cudaMemcpyDeviceToDevice, ctx->stream));
        }
      }
    } else if (refine) {
      const double a = th_cur[bf - 1], e = (ub - a) / 2, cc = (ub + a) / 2;
      if (e > 0) {
        const double x0 = std::fabs((th_cur[0] - cc) / e);
        int deg = (int)std::floor(std::acosh(1e6) / std::acosh(std::max(x0, 1.0 + 1e-12)));
        deg = std::max(2, std::min(16, deg));
        bool fused = false;
        TRY(cheb_fused_df(ctx, H64, X64, bf, deg, th_cur[0], a, ub, X64, &fused));
        if (!fused) {
          Workspace wp(ctx);
          double *Y0, *Y1, *Y2, *Yout = nullptr;
          TRY(wp.get(&Y0, (size_t)bf * n));
          TRY(wp.get(&Y1, (size_t)bf * n));
          TRY(wp.get(&Y2, (size_t)bf * n));
          TRY(kron_apply<double>(ctx, H64, X64, bf, HX64, 1.0, 0.0, 0.0, nullptr, Tb64));
          TRY((cheb_filter<double>(ctx, H64, X64, HX64, bf, th_cur[0], a, ub, deg, Y0, Y1, Y2, Tb64, &Yout)));
          CK(cudaMemcpyAsync(X64, Yout, sizeof(double) * bf * n, cudaMemcpyDeviceToDevice, ctx->stream));
          normalize_kernel<double><<<bf, 256, 0, ctx->stream>>>(X64, n, nullptr);
          CKL();
        }
      }
    }
    TRY(cholqr64_refine(ctx, ws, X64, bf, n, tmp64));
    {
      bool done = false;  // the mixed paths form the FP64-accurate product in double-FP32
      if (refine) TRY(cheb_fused_df(ctx, H64, X64, bf, 0, 0.0, 0.0, 0.0, HX64, &done));
      if (!done) TRY(kron_product<double>(ctx, H64, X64, bf, HX64, Tb64));
    }
    TRY(gram<double>(ctx, ws, X64, bf, HX64, bf, n, Gs, true));
    TRY(syev64(ctx, ws, Gs, bf, w, Zs, chunked));
    TRY(combine<double>(ctx, Zs, true, bf, bf, X64, n, C, 1.0, 0.0, nullptr));
    if (!refine || pass + 1 >= kRefinePasses) break;
    // FP64 residuals of the Ritz vectors (H C = Z^T H X)
    double* HC = Tb64;
    TRY(combine<double>(ctx, Zs, true, bf, bf, HX64, n, HC, 1.0, 0.0, nullptr));
    CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    // only the kept vectors need the FP64 accuracy; the extra one beyond them
    // serves the cut rule, whose gap test needs its Ritz value only, and that
    // is accurate to the square of its residual (k_acc)
    residual_kernel<double><<<bf, 256, 0, ctx->stream>>>(C, HC, w, n, k_acc, kRefineTol, rn64, ctx->d_status);
    CKL();
    int fails = 0;
    TRY(read_status(ctx, &fails, 1));
    if (ctx->trace) {
      std::vector<double> r(bf), t(bf);
      TRY(to_host<double>(ctx, rn64, r.data(), bf));
      TRY(to_host<double>(ctx, w, t.data(), bf));
      int wi = 0;
      const double worst = worst_relative(r, t, k_acc, &wi);
      fprintf(stderr, "[rmc refine] n=%ld b=%d k_conv=%d pass=%d fails=%d worst i=%d res=%.3e theta=%.12g thb=%.12g\n",
              n, bf, k_conv, pass, fails, wi, worst, t[wi], t[bf - 1]);
    }
    if (fails == 0) break;
    TRY(to_host<double>(ctx, w, th_cur.data(), bf));
    CK(cudaMemcpyAsync(X64, C, sizeof(double) * bf * n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  std::vector<double> th(bf);
  TRY(to_host<double>(ctx, w, th.data(), bf));
  int keff = std::min(k_ret, bf);
  if (!in.top && k_ret < n) keff = cut_rule(th, keff, ctx->cfg.tau_deg);
  gauge_kernel<<<keff, 256, 0, ctx->stream>>>(C, n);
  CKL();
  const int nc = (int)in.carry.size();
  rmc_block* blk = nullptr;
  TRY(new_block(ctx, keff, nc, (int)n, &blk));
  CK(cudaMemcpyAsync(blk->E, w, sizeof(double) * keff, cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(blk->basis, C, sizeof(double) * keff * n, cudaMemcpyDeviceToDevice, ctx->stream));
  // rotate carried operators: out = C^T (o (x) I) C or C^T (I (x) o) C; the
  // mixed paths form T = (o (x) I) C in double-FP32 like their other
  // FP64-accurate block products (the part's DFMA rate is ~1/4 of that)
  double* Tr = Tb64;
  const bool rot_df = fp64_by_df(ctx);
  ProfScope ps_rot(ctx, 6, 0.0);
  for (int j = 0; j < nc; ++j) {
    const rmc_carry& cr = in.carry[j];
    const rmc_block* src = cr.side == 0 ? A : B;
    const double* o = src->ops + (size_t)cr.op * src->k * src->k;
    if (cr.side == 0) {
      GemmShape s{kA, kB, kA, kA, kB, 0, n, 1};
      EpiAxpby<double> e{Tr, nullptr, kB, 0, n, 0, 1.0, 0.0};
      if (rot_df) gemm_df<false, false>(o, blk->basis, s, keff, e, ctx->stream);
      else gemm_big<double, false, false>(o, blk->basis, s, keff, e, ctx->stream);
    } else {
      GemmShape s{keff * kA, kB, kB, kB, kB, 0, 0, 1};
      EpiAxpby<double> e{Tr, nullptr, kB, 0, 0, 0, 1.0, 0.0};
      if (rot_df) gemm_df<false, true>(blk->basis, o, s, 1, e, ctx->stream);
      else gemm_big<double, false, true>(blk->basis, o, s, 1, e, ctx->stream);
    }
    CKL();
    TRY(gram<double>(ctx, ws, blk->basis, keff, Tr, keff, n, blk->ops + (size_t)j * keff * keff, false));
    blk->tags[j] = src->tags[cr.op];
    blk->opnorm[j] = src->opnorm[cr.op];
  }
  int st[3];
  TRY(read_status(ctx, st, 3));
  CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int) * 3, ctx->stream));
  *out = blk;
  *soft = converged ? RMC_OK : RMC_ERR_NOCONV;
  if (!converged) fail(ctx, RMC_ERR_NOCONV, "subspace iteration did not converge in %d iterations (n=%ld)", iters, n);
  return RMC_OK;
}

rmc_status check_ctx(rmc_ctx* ctx) {
  if (!ctx) return RMC_ERR_INVAL;
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  return RMC_OK;
}

}  // namespace

// Lanes of a context (see rmc_ctx): created on first use, kept until the
// context is destroyed.
constexpr int kMaxLanes = 8;

rmc_status ensure_lanes(rmc_ctx* ctx, int L) {
  while ((int)ctx->lanes.size() < L) {
    std::unique_ptr<rmc_ctx> c(new rmc_ctx);
    rmc_ctx* lc = c.get();
    lc->device = ctx->device;
    lc->cfg = ctx->cfg;
    lc->cfg.stream = nullptr;
    lc->trace = ctx->trace;
    lc->budget = ctx->budget;
    lc->acct = ctx->acct ? ctx->acct : ctx;
    lc->pool = ctx->pool;
    lc->own_pool = false;
    {
      rmc_ctx* ctx = lc;  // the checks below report on the lane
      CK(cudaStreamCreateWithFlags(&lc->stream, cudaStreamNonBlocking));
      lc->own_stream = true;
      CK(cudaMalloc(&lc->d_status, 64 * sizeof(int)));
      CK(cudaMemset(lc->d_status, 0, 64 * sizeof(int)));
      CK(cudaMallocHost(&lc->h_pinned, kPinnedDoubles * sizeof(double)));
    }
    ctx->lanes.push_back(c.release());
  }
  return RMC_OK;
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

rmc_status rmc_create(rmc_ctx** out, const rmc_config* cfg_in) {
  if (!out) return RMC_ERR_INVAL;
  *out = nullptr;
  rmc_config cfg{};
  if (cfg_in) cfg = *cfg_in;
  std::unique_ptr<rmc_ctx> c(new rmc_ctx);
  rmc_ctx* ctx = c.get();
  if (cfg.mem_budget == 0) cfg.mem_budget = (size_t)40 << 30;
  if (cfg.precision < 0 || cfg.precision > 2) return RMC_ERR_INVAL;
  if (cfg.tol <= 0) cfg.tol = cfg.precision == RMC_PREC_FP64 ? 1e-11 : 2e-6;
  if (cfg.max_iter <= 0) cfg.max_iter = 200;
  if (cfg.tau_deg <= 0) cfg.tau_deg = 1e-7;
  ctx->cfg = cfg;
  ctx->device = cfg.device;
  if (const char* t = std::getenv("RMC_TRACE")) ctx->trace = std::atoi(t);
  ctx->budget = cfg.mem_budget;
  CK(cudaSetDevice(ctx->device));
  if (cfg.stream) {
    ctx->stream = (cudaStream_t)cfg.stream;
  } else {
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = ctx->device;
  CK(cudaMemPoolCreate(&ctx->pool, &props));
  uint64_t thr = UINT64_MAX;
  CK(cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr));
  CK(cudaMalloc(&ctx->d_status, 64 * sizeof(int)));
  CK(cudaMemset(ctx->d_status, 0, 64 * sizeof(int)));
  CK(cudaMallocHost(&ctx->h_pinned, kPinnedDoubles * sizeof(double)));
  *out = c.release();
  return RMC_OK;
}

rmc_status rmc_destroy(rmc_ctx* ctx) {
  if (!ctx) return RMC_ERR_INVAL;
  cudaSetDevice(ctx->device);
  for (rmc_ctx* l : ctx->lanes) rmc_destroy(l);
  ctx->lanes.clear();
  std::vector<rmc_block*> bl(ctx->blocks.begin(), ctx->blocks.end());
  for (rmc_block* b : bl) free_block(ctx, b);
  cudaStreamSynchronize(ctx->stream);
  harvest(ctx);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->pool && ctx->own_pool) cudaMemPoolDestroy(ctx->pool);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return RMC_OK;
}

const char* rmc_last_error(const rmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
size_t rmc_mem_in_use(const rmc_ctx* ctx) { return ctx ? ctx->in_use : 0; }  // lanes charge their parent
void* rmc_stream(const rmc_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

rmc_status rmc_stats(const rmc_ctx* ctx, uint64_t* launches, uint64_t* iterations) {
  if (!ctx) return RMC_ERR_INVAL;
  if (launches) *launches = ctx->launches;
  if (iterations) *iterations = ctx->iterations;
  return RMC_OK;
}

rmc_status rmc_profile(rmc_ctx* ctx, int enable) {
  if (!ctx) return RMC_ERR_INVAL;
  if (enable != 0 && enable != 1 && !(enable & RMC_PROFILE_MASK)) return fail(ctx, RMC_ERR_INVAL, "rmc_profile: bad mode");
  ctx->prof = enable == 0 ? 0u : enable == 1 ? (1u << RMC_PROF_KINDS) - 1u
                                             : (unsigned)enable & ((1u << RMC_PROF_KINDS) - 1u);
  return RMC_OK;
}

rmc_status rmc_profile_read(rmc_ctx* ctx, int kind, uint64_t* groups, uint64_t* launches, double* ms,
                            double* flops) {
  if (!ctx || kind < 0 || kind >= RMC_PROF_KINDS) return RMC_ERR_INVAL;
  cudaStreamSynchronize(ctx->stream);
  harvest(ctx);
  if (groups) *groups = ctx->prof_groups[kind];
  if (launches) *launches = ctx->prof_launches[kind];
  if (ms) *ms = ctx->prof_ms[kind];
  if (flops) *flops = ctx->prof_flops[kind];
  ctx->prof_groups[kind] = ctx->prof_launches[kind] = 0;
  ctx->prof_ms[kind] = ctx->prof_flops[kind] = 0;
  return RMC_OK;
}

rmc_status rmc_build_leaf(rmc_ctx* ctx, const double* H, int D, int k, const double* const* ops,
                          const rmc_op_tag* tags, int n_ops, rmc_block** out) {
  TRY(check_ctx(ctx));
  if (!H || !out || D < 1 || D > kMaxSmallDim || k < 1 || n_ops < 0 || n_ops > 4 * kMaxOps || (n_ops && !ops))
    return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf: bad arguments (D=%d k=%d n_ops=%d)", D, k, n_ops);
  double hmax = 0;
  for (int i = 0; i < D * D; ++i) {
    if (!std::isfinite(H[i])) return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf: H has a non-finite entry");
    hmax = std::max(hmax, std::fabs(H[i]));
  }
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < i; ++j)
      if (std::fabs(H[i * D + j] - H[j * D + i]) > 1e-12 * std::max(1.0, hmax))
        return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf: H is not symmetric at (%d,%d)", i, j);
  Workspace ws(ctx);
  double* dH;
  TRY(ws.get(&dH, (size_t)D * D));
  CK(cudaMemcpyAsync(dH, H, sizeof(double) * D * D, cudaMemcpyHostToDevice, ctx->stream));
  std::vector<const double*> dops(n_ops);
  std::vector<rmc_op_tag> tg(n_ops);
  std::vector<double> nrm(n_ops);
  for (int j = 0; j < n_ops; ++j) {
    if (!ops[j]) return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf: operator %d is NULL", j);
    for (int i = 0; i < D * D; ++i)
      if (!std::isfinite(ops[j][i])) return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf: operator %d non-finite", j);
    double* d;
    TRY(ws.get(&d, (size_t)D * D));
    CK(cudaMemcpyAsync(d, ops[j], sizeof(double) * D * D, cudaMemcpyHostToDevice, ctx->stream));
    dops[j] = d;
    tg[j] = tags ? tags[j] : rmc_op_tag{-1, 'O'};
    nrm[j] = host_opnorm2(ops[j], D);
  }
  TRY(leaf_from_device(ctx, ws, dH, D, k, true, dops, tg, nrm, out));
  CK(cudaStreamSynchronize(ctx->stream));
  return RMC_OK;
}

static int pauli_code(char p) {
  switch (p) {
    case 'X': case 'x': return 1;
    case 'Y': case 'y': return 2;
    case 'Z': case 'z': return 3;
    default: return 0;
  }
}

rmc_status rmc_build_leaf_pauli(rmc_ctx* ctx, int L, int k, int n_onsite, const int* onsite_site,
                                const char* onsite_pauli, const double* onsite_coef, int n_bonds, const int* bond_i,
                                const int* bond_j, const char* bond_pauli_i, const char* bond_pauli_j,
                                const double* bond_coef, int n_carry, const rmc_op_tag* carry, rmc_block** out) {
  TRY(check_ctx(ctx));
  if (L < 1 || (1 << L) > kMaxSmallDim || k < 1 || n_onsite < 0 || n_bonds < 0 || n_carry < 0 || !out ||
      n_carry > 4 * kMaxOps)
    return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf_pauli: bad sizes (L=%d k=%d)", L, k);
  std::vector<PauliTerm> terms;
  for (int t = 0; t < n_onsite; ++t) {
    const int c = pauli_code(onsite_pauli[t]);
    if (c == 0 || c == 2 || onsite_site[t] < 0 || onsite_site[t] >= L || !std::isfinite(onsite_coef[t]))
      return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf_pauli: bad on-site term %d (a Y field is imaginary)", t);
    terms.push_back(PauliTerm{onsite_site[t], -1, c, 0, onsite_coef[t]});
  }
  for (int t = 0; t < n_bonds; ++t) {
    const int ci = pauli_code(bond_pauli_i[t]), cj = pauli_code(bond_pauli_j[t]);
    if (!ci || !cj || (ci == 2) != (cj == 2) || bond_i[t] < 0 || bond_j[t] >= L || bond_i[t] >= bond_j[t] ||
        !std::isfinite(bond_coef[t]))
      return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf_pauli: bad bond %d", t);
    // Y Y = -(iY)(iY): the real representation carries iY
    const double cf = (ci == 2) ? -bond_coef[t] : bond_coef[t];
    terms.push_back(PauliTerm{bond_i[t], bond_j[t], ci, cj, cf});
  }
  const int D = 1 << L;
  Workspace ws(ctx);
  PauliTerm* dterms;
  TRY(ws.get(&dterms, std::max<size_t>(1, terms.size())));
  if (!terms.empty())
    CK(cudaMemcpyAsync(dterms, terms.data(), sizeof(PauliTerm) * terms.size(), cudaMemcpyHostToDevice, ctx->stream));
  double* dH;
  TRY(ws.get(&dH, (size_t)D * D));
  pauli_matrix_kernel<<<1, 256, 0, ctx->stream>>>(dterms, (int)terms.size(), L, dH);
  CKL();
  std::vector<const double*> dops(n_carry);
  std::vector<rmc_op_tag> tg(n_carry);
  std::vector<double> nrm(n_carry, 1.0);
  PauliTerm* dct;
  TRY(ws.get(&dct, std::max(1, n_carry)));
  std::vector<PauliTerm> ct(n_carry);
  for (int j = 0; j < n_carry; ++j) {
    const int c = pauli_code(carry[j].pauli);
    if (!c || carry[j].site < 0 || carry[j].site >= L)
      return fail(ctx, RMC_ERR_INVAL, "rmc_build_leaf_pauli: bad carried operator %d", j);
    ct[j] = PauliTerm{carry[j].site, -1, c, 0, 1.0};
    tg[j] = carry[j];
  }
  if (n_carry) CK(cudaMemcpyAsync(dct, ct.data(), sizeof(PauliTerm) * n_carry, cudaMemcpyHostToDevice, ctx->stream));
  for (int j = 0; j < n_carry; ++j) {
    double* d;
    TRY(ws.get(&d, (size_t)D * D));
    pauli_matrix_kernel<<<1, 256, 0, ctx->stream>>>(dct + j, 1, L, d);
    CKL();
    dops[j] = d;
  }
  TRY(leaf_from_device(ctx, ws, dH, D, k, true, dops, tg, nrm, out));
  CK(cudaStreamSynchronize(ctx->stream));
  return RMC_OK;
}

rmc_status rmc_couple(rmc_ctx* ctx, const rmc_block* A, const rmc_block* B, const rmc_term* terms, int n_terms,
                      int k_keep, const rmc_carry* carry, int n_carry, int flags, rmc_block** out) {
  TRY(check_ctx(ctx));
  if (!A || !B || !out || k_keep < 1 || n_terms < 0 || n_terms > kMaxOps || n_carry < 0 || n_carry > 4 * kMaxOps ||
      (n_terms && !terms) || (n_carry && !carry))
    return fail(ctx, RMC_ERR_INVAL, "rmc_couple: bad arguments");
  MergeInput in;
  in.A = A;
  in.B = B;
  in.k_keep = k_keep;
  in.top = (flags & RMC_COUPLE_TOP) != 0;
  for (int t = 0; t < n_terms; ++t) {
    if (terms[t].op_a < 0 || terms[t].op_a >= A->n_ops || terms[t].op_b < 0 || terms[t].op_b >= B->n_ops ||
        !std::isfinite(terms[t].coef))
      return fail(ctx, RMC_ERR_INVAL, "rmc_couple: term %d refers to a missing operator", t);
    in.terms.push_back(terms[t]);
  }
  for (int c = 0; c < n_carry; ++c) {
    const rmc_block* s = carry[c].side == 0 ? A : (carry[c].side == 1 ? B : nullptr);
    if (!s || carry[c].op < 0 || carry[c].op >= s->n_ops)
      return fail(ctx, RMC_ERR_INVAL, "rmc_couple: carry %d refers to a missing operator", c);
    in.carry.push_back(carry[c]);
  }
  rmc_status soft = RMC_OK;
  rmc_status st = (ctx->cfg.precision == RMC_PREC_FP64) ? couple_impl<double>(ctx, in, out, &soft)
                                                        : couple_impl<float>(ctx, in, out, &soft);
  if (st != RMC_OK) return st;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  harvest(ctx);
  if (e != cudaSuccess) return fail(ctx, RMC_ERR_CUDA, "rmc_couple: %s", cudaGetErrorString(e));
  return soft;
}

rmc_status rmc_couple_batch(rmc_ctx* ctx, int n, const rmc_couple_desc* d, rmc_block** out, rmc_status* status) {
  TRY(check_ctx(ctx));
  if (n < 0 || (n > 0 && (!d || !out || !status)))
    return fail(ctx, RMC_ERR_INVAL, "rmc_couple_batch: bad arguments");
  for (int i = 0; i < n; ++i) {
    out[i] = nullptr;
    status[i] = RMC_OK;
  }
  if (n == 0) return RMC_OK;
  const int want = ctx->cfg.lanes > 0 ? ctx->cfg.lanes : kMaxLanes;
  const int L = std::min(n, std::min(want, kMaxLanes));
  if (L <= 1) {  // one at a time on this context
    rmc_status first = RMC_OK;
    std::string msg;
    for (int i = 0; i < n; ++i) {
      status[i] = rmc_couple(ctx, d[i].A, d[i].B, d[i].terms, d[i].n_terms, d[i].k_keep, d[i].carry, d[i].n_carry,
                             d[i].flags, &out[i]);
      if (status[i] != RMC_OK && status[i] != RMC_ERR_NOCONV) out[i] = nullptr;
      const bool hard = status[i] != RMC_OK && status[i] != RMC_ERR_NOCONV;
      if ((hard && (first == RMC_OK || first == RMC_ERR_NOCONV)) || (status[i] == RMC_ERR_NOCONV && first == RMC_OK)) {
        first = status[i];
        msg = ctx->err;
      }
    }
    if (first != RMC_OK) ctx->err = "rmc_couple_batch: " + msg;
    return first;
  }
  TRY(ensure_lanes(ctx, L));
  // the lanes start after everything queued on this context's stream
  cudaEvent_t ready;
  CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  CK(cudaEventRecord(ready, ctx->stream));
  for (int l = 0; l < L; ++l) {
    ctx->lanes[l]->prof = ctx->prof;
    CK(cudaStreamWaitEvent(ctx->lanes[l]->stream, ready, 0));
  }
  std::atomic<int> next{0};
  std::vector<int> lane_of(n, -1);
  std::vector<std::string> msgs(n);
  std::vector<std::thread> th;
  for (int l = 0; l < L; ++l) {
    th.emplace_back([&, l]() {
      rmc_ctx* lc = ctx->lanes[l];
      for (int i = next++; i < n; i = next++) {
        lane_of[i] = l;
        status[i] = rmc_couple(lc, d[i].A, d[i].B, d[i].terms, d[i].n_terms, d[i].k_keep, d[i].carry,
                               d[i].n_carry, d[i].flags, &out[i]);
        if (status[i] != RMC_OK) msgs[i] = lc->err;  // the lane's next call clears it
        if (status[i] != RMC_OK && status[i] != RMC_ERR_NOCONV) out[i] = nullptr;
      }
    });
  }
  for (auto& t : th) t.join();
  cudaEventDestroy(ready);
  // blocks pass to this context; counters and timings join its own
  rmc_status first = RMC_OK;
  std::string msg;
  for (int i = 0; i < n; ++i) {
    rmc_ctx* lc = ctx->lanes[lane_of[i]];
    if (out[i]) {
      lc->blocks.erase(out[i]);
      ctx->blocks.insert(out[i]);
      for (void* p : {(void*)out[i]->E, (void*)out[i]->ops, (void*)out[i]->basis}) {
        auto it = p ? lc->live.find(p) : lc->live.end();
        if (it != lc->live.end()) {
          ctx->live[p] = it->second;
          lc->live.erase(it);
        }
      }
    }
    const bool hard = status[i] != RMC_OK && status[i] != RMC_ERR_NOCONV;
    if ((hard && (first == RMC_OK || first == RMC_ERR_NOCONV)) || (status[i] == RMC_ERR_NOCONV && first == RMC_OK)) {
      first = status[i];
      msg = msgs[i];
    }
  }
  for (int l = 0; l < L; ++l) {
    rmc_ctx* lc = ctx->lanes[l];
    harvest(lc);
    ctx->launches += lc->launches;
    ctx->iterations += lc->iterations;
    lc->launches = lc->iterations = 0;
    for (int k = 0; k < RMC_PROF_KINDS; ++k) {
      ctx->prof_groups[k] += lc->prof_groups[k];
      ctx->prof_launches[k] += lc->prof_launches[k];
      ctx->prof_ms[k] += lc->prof_ms[k];
      ctx->prof_flops[k] += lc->prof_flops[k];
      lc->prof_groups[k] = lc->prof_launches[k] = 0;
      lc->prof_ms[k] = lc->prof_flops[k] = 0;
    }
  }
  if (first != RMC_OK) ctx->err = "rmc_couple_batch: " + msg;
  return first;
}

rmc_status rmc_lowest(rmc_ctx* ctx, const rmc_block* blk, int q, double* E_out, double* C_out, int* k_eff_out) {
  TRY(check_ctx(ctx));
  if (!blk || !E_out || q < 1) return fail(ctx, RMC_ERR_INVAL, "rmc_lowest: bad arguments");
  const int qq = std::min(q, blk->k);
  CK(cudaMemcpyAsync(E_out, blk->E, sizeof(double) * qq, cudaMemcpyDeviceToHost, ctx->stream));
  if (C_out && blk->rows > 0) {
    std::vector<double> tmp((size_t)qq * blk->rows);
    CK(cudaMemcpyAsync(tmp.data(), blk->basis, sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < qq; ++i)
      for (int r = 0; r < blk->rows; ++r) C_out[(size_t)r * qq + i] = tmp[(size_t)i * blk->rows + r];
  }
  CK(cudaStreamSynchronize(ctx->stream));
  if (k_eff_out) *k_eff_out = qq;
  return RMC_OK;
}

rmc_status rmc_block_free(rmc_ctx* ctx, rmc_block* blk) {
  if (!ctx || !blk) return RMC_ERR_INVAL;
  if (!ctx->blocks.count(blk)) return fail(ctx, RMC_ERR_INVAL, "rmc_block_free: unknown block");
  cudaSetDevice(ctx->device);
  free_block(ctx, blk);
  return RMC_OK;
}

rmc_status rmc_block_info(const rmc_block* blk, int* k, int* n_ops, int* rows, rmc_op_tag* tags) {
  if (!blk) return RMC_ERR_INVAL;
  if (k) *k = blk->k;
  if (n_ops) *n_ops = blk->n_ops;
  if (rows) *rows = blk->rows;
  if (tags)
    for (int j = 0; j < blk->n_ops; ++j) tags[j] = blk->tags[j];
  return RMC_OK;
}

rmc_status rmc_block_export(rmc_ctx* ctx, const rmc_block* blk, double* E, double* ops, double* basis) {
  TRY(check_ctx(ctx));
  if (!blk) return fail(ctx, RMC_ERR_INVAL, "rmc_block_export: null block");
  if (E) CK(cudaMemcpyAsync(E, blk->E, sizeof(double) * blk->k, cudaMemcpyDeviceToHost, ctx->stream));
  if (ops && blk->n_ops)
    CK(cudaMemcpyAsync(ops, blk->ops, sizeof(double) * blk->n_ops * blk->k * blk->k, cudaMemcpyDeviceToHost,
                       ctx->stream));
  if (basis && blk->rows)
    CK(cudaMemcpyAsync(basis, blk->basis, sizeof(double) * blk->rows * blk->k, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return RMC_OK;
}

rmc_status rmc_block_import(rmc_ctx* ctx, int k, const double* E, int n_ops, const double* ops,
                            const rmc_op_tag* tags, int rows, const double* basis, rmc_block** out) {
  TRY(check_ctx(ctx));
  if (k < 1 || !E || n_ops < 0 || (n_ops && !ops) || rows < 0 || (rows && !basis) || !out)
    return fail(ctx, RMC_ERR_INVAL, "rmc_block_import: bad arguments");
  for (int i = 0; i < k; ++i)
    if (!std::isfinite(E[i]) || (i && E[i] < E[i - 1]))
      return fail(ctx, RMC_ERR_INVAL, "rmc_block_import: energies must be finite and ascending");
  rmc_block* b = nullptr;
  TRY(new_block(ctx, k, n_ops, rows, &b));
  CK(cudaMemcpyAsync(b->E, E, sizeof(double) * k, cudaMemcpyHostToDevice, ctx->stream));
  if (n_ops) CK(cudaMemcpyAsync(b->ops, ops, sizeof(double) * n_ops * k * k, cudaMemcpyHostToDevice, ctx->stream));
  if (rows) CK(cudaMemcpyAsync(b->basis, basis, sizeof(double) * rows * k, cudaMemcpyHostToDevice, ctx->stream));
  for (int j = 0; j < n_ops; ++j) {
    b->tags[j] = tags ? tags[j] : rmc_op_tag{-1, 'O'};
    b->opnorm[j] = host_opnorm2(ops + (size_t)j * k * k, k);
  }
  CK(cudaStreamSynchronize(ctx->stream));
  *out = b;
  return RMC_OK;
}

rmc_status rmc_kron_matvec(rmc_ctx* ctx, int dtype, int kA, int kB, int n_ops, int nv, const void* EA,
                           const void* EB, const void* A, const void* B, const double* coef, const void* X, void* Y,
                           const void* Z, double alpha, double beta, double gamma) {
  TRY(check_ctx(ctx));
  if (kA < 1 || kB < 1 || n_ops < 0 || n_ops > kMaxOps || nv < 1 || !EA || !EB || !X || !Y ||
      (n_ops && (!A || !B || !coef)) || (gamma != 0.0 && !Z) || dtype < 0 || dtype > 2 || X == Y || Z == Y)
    return fail(ctx, RMC_ERR_INVAL, "rmc_kron_matvec: bad arguments");
  if (dtype == 2 && !tc_fits(kA, kB, n_ops))
    return fail(ctx, RMC_ERR_INVAL, "rmc_kron_matvec: shape outside the tensor-core kernel (n_ops*kB, kA <= 256)");
  Native64Scope native(ctx);
  Workspace ws(ctx);
  Coefs cf{};
  for (int j = 0; j < n_ops; ++j) cf.c[j] = coef[j];
  auto run = [&](auto tag) -> rmc_status {
    using T = decltype(tag);
    KronOp<T> H;
    H.kA = kA;
    H.kB = kB;
    H.n_ops = n_ops;
    H.EA = (const T*)EA;
    H.EB = (const T*)EB;
    H.Bcat = (const T*)B;
    T *Acat, *Tbuf;
    TRY(ws.get(&Acat, (size_t)std::max(1, n_ops) * kA * kA));
    TRY(ws.get(&Tbuf, (size_t)std::max(1, n_ops) * kA * kB * nv));
    if (n_ops) {
      build_acat_kernel<T><<<grid1d((long)kA * kA * n_ops), 256, 0, ctx->stream>>>((const T*)A, cf, kA, n_ops, Acat);
      CKL();
    }
    H.Acat = Acat;
    if constexpr (sizeof(T) == 4) {
      if (dtype == 2)
        return kron_apply_tc(ctx, H, (const float*)X, nv, (float*)Y, (float)alpha, (float)beta, (float)gamma,
                             (const float*)Z, Tbuf);
    }
    return kron_apply<T>(ctx, H, (const T*)X, nv, (T*)Y, (T)alpha, (T)beta, (T)gamma, (const T*)Z, Tbuf);
  };
  return dtype == 0 ? run(double{}) : run(float{});
}

rmc_status rmc_gram(rmc_ctx* ctx, int dtype, int nv1, int nv2, long n, const float* X1, const float* X2, float* G,
                    int symmetrize) {
  TRY(check_ctx(ctx));
  if (nv1 < 1 || nv2 < 1 || n < 1 || !X1 || !X2 || !G || (dtype != 1 && dtype != 2) ||
      (symmetrize && nv1 != nv2))
    return fail(ctx, RMC_ERR_INVAL, "rmc_gram: bad arguments");
  Workspace ws(ctx);
  if (dtype == 2) {
    if (n % 4 != 0 || ((uintptr_t)X1 & 15) || ((uintptr_t)X2 & 15) || !encode_tiled())
      return fail(ctx, RMC_ERR_INVAL, "rmc_gram: the tensor-core form needs n %% 4 == 0 and 16-byte aligned blocks");
    return gram_tc(ctx, ws, X1, nv1, X2, nv2, n, G, symmetrize != 0);
  }
  return gram<float>(ctx, ws, X1, nv1, X2, nv2, n, G, symmetrize != 0, false);
}

rmc_status rmc_cheb_filter(rmc_ctx* ctx, int dtype, int kA, int kB, int n_ops, int nv, const void* EA,
                           const void* EB, const void* A, const void* B, const double* coef, const void* X, int deg,
                           double theta0, double a, double ub, int fused, void* Y) {
  TRY(check_ctx(ctx));
  if (kA < 1 || kB < 1 || n_ops < 0 || n_ops > kMaxOps || nv < 1 || !EA || !EB || !X || !Y ||
      (n_ops && (!A || !B || !coef)) || dtype < 0 || dtype > 3 || dtype == 2 || deg < 0 || deg > 64 ||
      (fused != 0 && fused != 1) || (dtype == 3 && !fused))
    return fail(ctx, RMC_ERR_INVAL, "rmc_cheb_filter: bad arguments");
  if (deg > 0 && !(theta0 < a && a < ub)) return fail(ctx, RMC_ERR_INVAL, "rmc_cheb_filter: need theta0 < a < ub");
  Native64Scope native(ctx);
  Workspace ws(ctx);
  Coefs cf{};
  for (int j = 0; j < n_ops; ++j) cf.c[j] = coef[j];
  auto run = [&](auto tag) -> rmc_status {
    using T = decltype(tag);
    const long n = (long)kA * kB;
    KronOp<T> H;
    H.kA = kA;
    H.kB = kB;
    H.n_ops = n_ops;
    H.EA = (const T*)EA;
    H.EB = (const T*)EB;
    H.Bcat = (const T*)B;
    T* Acat;
    TRY(ws.get(&Acat, (size_t)std::max(1, n_ops) * kA * kA));
    if (n_ops) {
      build_acat_kernel<T><<<grid1d((long)kA * kA * n_ops), 256, 0, ctx->stream>>>((const T*)A, cf, kA, n_ops, Acat);
      CKL();
    }
    H.Acat = Acat;
    if constexpr (sizeof(T) == 8) {
      if (dtype == 3) {
        bool done = false;
        TRY(cheb_fused_df(ctx, H, (const double*)X, nv, deg, theta0, a, ub, (double*)Y, &done));
        if (!done)
          return fail(ctx, RMC_ERR_INVAL, "rmc_cheb_filter: a %d x %d vector does not fit the fused kernel", kA, kB);
        return RMC_OK;
      }
    }
    if (fused) {
      FusedArgs p;
      size_t smem;
      if (!fused_plan<T>(H, nv, &p, &smem))
        return fail(ctx, RMC_ERR_INVAL, "rmc_cheb_filter: a %d x %d vector does not fit the fused kernel", kA, kB);
      if (deg == 0) return launch_fused<T>(ctx, H, (const T*)X, nullptr, (T*)Y, p, smem, 0.0);
      p.deg = deg;
      p.compute_hx = 1;
      p.e = (ub - a) / 2;
      p.c = (ub + a) / 2;
      p.sigma1 = p.e / (theta0 - p.c);
      return launch_fused<T>(ctx, H, (const T*)X, nullptr, (T*)Y, p, smem, 0.0);
    }
    T *Tbuf, *HX, *Y0, *Y1, *Y2;
    TRY(ws.get(&Tbuf, (size_t)std::max(1, n_ops) * n * nv));
    if (deg == 0) return kron_apply<T>(ctx, H, (const T*)X, nv, (T*)Y, T(1), T(0), T(0), nullptr, Tbuf);
    TRY(ws.get(&HX, (size_t)n * nv));
    TRY(ws.get(&Y0, (size_t)n * nv));
    TRY(ws.get(&Y1, (size_t)n * nv));
    TRY(ws.get(&Y2, (size_t)n * nv));
    TRY(kron_apply<T>(ctx, H, (const T*)X, nv, HX, T(1), T(0), T(0), nullptr, Tbuf));
    T* Yout = nullptr;
    if (deg == 1) {
      const double e = (ub - a) / 2, c = (ub + a) / 2, s1 = e / (theta0 - c);
      axpby_kernel<T><<<grid1d((long)nv * n), 256, 0, ctx->stream>>>(HX, (const T*)X, (long)nv * n, T(s1 / e),
                                                                      T(-c * s1 / e), Y1);
      CKL();
      Yout = Y1;
    } else {
      TRY((cheb_filter<T>(ctx, H, (const T*)X, HX, nv, theta0, a, ub, deg, Y0, Y1, Y2, Tbuf, &Yout)));
    }
    CK(cudaMemcpyAsync(Y, Yout, sizeof(T) * n * nv, cudaMemcpyDeviceToDevice, ctx->stream));
    normalize_kernel<T><<<nv, 256, 0, ctx->stream>>>((T*)Y, n, nullptr);
    CKL();
    return RMC_OK;
  };
  return (dtype == 0 || dtype == 3) ? run(double{}) : run(float{});
}

rmc_status rmc_syev(rmc_ctx* ctx, int m, const double* S, double* w, double* V) {
  TRY(check_ctx(ctx));
  if (m < 1 || m > kMaxSmallDim || !S || !w || !V) return fail(ctx, RMC_ERR_INVAL, "rmc_syev: bad arguments");
  Workspace ws(ctx);
  TRY(syev64(ctx, ws, S, m, w, V));
  CK(cudaStreamSynchronize(ctx->stream));
  return RMC_OK;
}

rmc_status rmc_rotate_op(rmc_ctx* ctx, int side, int kA, int kB, int kr, const double* C, const double* o,
                         double* out) {
  TRY(check_ctx(ctx));
  if ((side != 0 && side != 1) || kA < 1 || kB < 1 || kr < 1 || !C || !o || !out)
    return fail(ctx, RMC_ERR_INVAL, "rmc_rotate_op: bad arguments");
  Native64Scope native(ctx);
  Workspace ws(ctx);
  const long n = (long)kA * kB;
  double* Tr;
  TRY(ws.get(&Tr, (size_t)kr * n));
  if (side == 0) {
    GemmShape s{kA, kB, kA, kA, kB, 0, n, 1};
    EpiAxpby<double> e{Tr, nullptr, kB, 0, n, 0, 1.0, 0.0};
    gemm_big<double, false, false>(o, C, s, kr, e, ctx->stream);
  } else {
    GemmShape s{kr * kA, kB, kB, kB, kB, 0, 0, 1};
    EpiAxpby<double> e{Tr, nullptr, kB, 0, 0, 0, 1.0, 0.0};
    gemm_big<double, false, true>(C, o, s, 1, e, ctx->stream);
  }
  CKL();
  TRY(gram<double>(ctx, ws, C, kr, Tr, kr, n, out, false));
  CK(cudaStreamSynchronize(ctx->stream));
  return RMC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Recursion loop of Algorithm 1 over a chain (host scheduler).
// ---------------------------------------------------------------------------
namespace {

struct CTerm {  // on-site (j < 0) or two-site term with chain-global sites
  int i, j;
  char pi, pj;
  double coef;
};

struct ChainNode {
  int lo, hi;
  int left = -1, right = -1;
  bool sub = false;  // piece of a leaf wider than the dense leaf solver: keeps all its states
  std::string sig;
  std::vector<std::pair<int, char>> carry;  // relative (site, pauli), sorted
};

// Widest leaf the dense leaf solver takes (D = 2^7 = 128 <= the small
// eigensolver's 160).  A wider leaf (up to twice this) is built exactly as
// two dense sub-leaves that keep all their states and one merge that keeps
// min(k, D): the merge's product space is the leaf's whole Hilbert space, so
// its lowest states are the leaf's (Algorithm 1, first step, for L0 up to 14).
constexpr int kDenseLeafSites = 7;

// Largest chain whose lowest states rmc_solve_chain_states lifts to the full
// 2^N computational basis (2^24 doubles = 128 MiB per state).
constexpr int kMaxLiftSites = 24;

// Largest merged block whose exact ground energy and discarded-sector gap
// rmc_solve_chain_bounds evaluates on the full 2^L basis (Krylov vectors of
// 2^22 doubles, 32 MiB each, 96 of them and their products: 6 GiB).
constexpr int kMaxFullSpaceSites = 22;

int build_tree(std::vector<ChainNode>& nodes, int lo, int hi, int L0) {
  nodes.push_back(ChainNode{lo, hi});
  const int id = (int)nodes.size() - 1;
  if (hi - lo > L0) {
    const int mid = lo + (hi - lo) / 2;
    const int l = build_tree(nodes, lo, mid, L0);
    const int r = build_tree(nodes, mid, hi, L0);
    nodes[id].left = l;
    nodes[id].right = r;
  }
  return id;
}

// Signature of a block: its length and every term lying inside it, with
// sites relative to its first site.  Blocks with equal signatures have equal
// spectra and operator matrices (the paper's homogeneous reuse).
std::string signature(const std::vector<CTerm>& terms, int lo, int hi) {
  std::vector<std::string> parts;
  char buf[128];
  for (const CTerm& t : terms) {
    const bool in = t.j < 0 ? (t.i >= lo && t.i < hi) : (t.i >= lo && t.j < hi);
    if (!in) continue;
    snprintf(buf, sizeof buf, "%d,%d,%c,%c,%.17g", t.i - lo, t.j < 0 ? -1 : t.j - lo, t.pi, t.j < 0 ? '-' : t.pj, t.coef);
    parts.push_back(buf);
  }
  std::sort(parts.begin(), parts.end());
  std::string s = std::to_string(hi - lo) + "|";
  for (auto& p : parts) s += p + ";";
  return s;
}

int find_tag(const rmc_block* b, int site, char p) {
  for (int j = 0; j < b->n_ops; ++j)
    if (b->tags[j].site == site && b->tags[j].pauli == p) return j;
  return -1;
}

}  // namespace

namespace {

// Lifted states of a block (Eq. (11) applied recursively, psi = (U_A (x) U_B) C):
// out (k x 2^L, vector-major) for a block of L sites.  Leaf: its basis.
// Merge: for each kept vector c_j (a k_A x k_B matrix), psi_j = U_A^T c_j U_B
// with U_A, U_B the children's lifted states, in two batched GEMMs.
rmc_status lift_block(rmc_ctx* ctx, Workspace& ws, const std::vector<ChainNode>& nodes,
                      const std::vector<rmc_block*>& blk_of, int id, int kuse, double** out) {
  const ChainNode& nd = nodes[id];
  const rmc_block* b = blk_of[id];
  const long len = 1L << (nd.hi - nd.lo);
  if (nd.left < 0) {
    *out = b->basis;
    return RMC_OK;
  }
  double *UA, *UB;
  TRY(lift_block(ctx, ws, nodes, blk_of, nd.left, blk_of[nd.left]->k, &UA));
  TRY(lift_block(ctx, ws, nodes, blk_of, nd.right, blk_of[nd.right]->k, &UB));
  const int kA = blk_of[nd.left]->k, kB = blk_of[nd.right]->k;
  const long LA = 1L << (nodes[nd.left].hi - nodes[nd.left].lo), LB = len / LA;
  double *T, *Psi;
  TRY(ws.get(&T, (size_t)kuse * kA * LB));
  TRY(ws.get(&Psi, (size_t)kuse * len));
  // T[(j, a)][y] = sum_b C[j][a][b] U_B[b][y]
  GemmShape s1{kuse * kA, (int)LB, kB, kB, LB, 0, 0, 1};
  gemm_big<double, false, false>(b->basis, UB, s1, 1, EpiAxpby<double>{T, nullptr, LB, 0, 0, 0, 1.0, 0.0},
                                 ctx->stream);
  CKL();
  // Psi_j[x][y] = sum_a U_A[a][x] T_j[a][y]
  GemmShape s2{(int)LA, (int)LB, kA, LA, LB, 0, (long)kA * LB, 1};
  gemm_big<double, true, false>(UA, T, s2, kuse, EpiAxpby<double>{Psi, nullptr, LB, 0, len, 0, 1.0, 0.0},
                                ctx->stream);
  CKL();
  *out = Psi;
  return RMC_OK;
}

// ---------------------------------------------------------------------------
// Per-merge truncation diagnostics (Sec. IV and Appendix B).  For the merge
// of blocks A and B let P project the merged block's Hilbert space onto the
// retained product sector span{|a>|b>} (the kept states of A and B) and
// Q = I - P.  Then a = lambda_min(PHP) is the merge's lowest eigenvalue of
// Eq. (7), b = ||PHQ||_2 = ||PVQ||_2 (the uncoupled part does not mix the
// sectors), gamma = lambda_min(QHQ on range Q) - a, and the merge's error
// obeys 0 <= a - E0 <= r(b, gamma) = (sqrt(gamma^2 + 4 b^2) - gamma) / 2.
// ---------------------------------------------------------------------------

// Product of two real single-site Paulis (Y carried as iY): p1 p2 = sign * out,
// out = 'I' for the identity.  Returns false for a non-Pauli tag.
bool pauli_product(char p1, char p2, char* out, double* sign) {
  auto idx = [](char p) { return p == 'X' ? 0 : p == 'Y' ? 1 : p == 'Z' ? 2 : -1; };
  const int i = idx(p1), j = idx(p2);
  if (i < 0 || j < 0) return false;
  // rows: p1 = X, iY, Z; columns: p2 = X, iY, Z (matrix products of the real forms)
  static const char prod[3][3] = {{'I', 'Z', 'Y'}, {'Z', 'I', 'X'}, {'Y', 'X', 'I'}};
  static const double sgn[3][3] = {{1, -1, -1}, {1, -1, -1}, {1, 1, 1}};
  *out = prod[i][j];
  *sign = sgn[i][j];
  return true;
}

// b = ||P V Q||_2 of the merge of A and B with coupling V = sum_t c_t O_A^t (x) O_B^t,
// from b^2 = lambda_max(P V^2 P - (P V P)^2) restricted to range(P) (Appendix B).
// In the product basis of the kept states
//   P V P   = sum_t c_t o_A^t (x) o_B^t                  (the coupling of Eq. (7)),
//   P V^2 P = sum_{s,t} c_s c_t [O_A^s O_A^t] (x) [O_B^s O_B^t],
// with [O] = U^T O U the projection of a physical operator onto a block's kept
// states.  Two Paulis on one site multiply to +-(a Pauli or I), so [O^s O^t] is
// a carried operator up to sign, or the identity; a product of operators on
// different sites is not carried, and then b is unavailable (*available =
// false, *b_out = NaN).  M = P V^2 P - (P V P)^2 is itself a Kronecker sum, so
// lambda_max(M) = -lambda_min(-M) comes from the merge's own FP64 subspace
// iteration on -M.
rmc_status coupling_norm(rmc_ctx* ctx, const rmc_block* A, const rmc_block* B, const rmc_term* terms, int nt,
                         double* b_out, bool* available, std::string* why) {
  *available = false;
  *b_out = NAN;
  const int kA = A->k, kB = B->k;
  const long n = (long)kA * kB;
  if (nt == 0) {
    *available = true;
    *b_out = 0.0;
    return RMC_OK;
  }
  struct KTerm { int ia, ib; int qs, qt; double coef; };  // ia/ib: carried op, -1 identity; q: -1 or (s, t)
  std::vector<KTerm> kt;
  for (int s = 0; s < nt; ++s)
    for (int t = 0; t < nt; ++t) {
      const rmc_op_tag as = A->tags[terms[s].op_a], at = A->tags[terms[t].op_a];
      const rmc_op_tag bs = B->tags[terms[s].op_b], bt = B->tags[terms[t].op_b];
      char pa, pb;
      double sa, sb;
      if (as.site != at.site || bs.site != bt.site || !pauli_product(as.pauli, at.pauli, &pa, &sa) ||
          !pauli_product(bs.pauli, bt.pauli, &pb, &sb)) {
        *why = "the coupling's operator products are not single-site Paulis";
        return RMC_OK;
      }
      const int ia = pa == 'I' ? -1 : find_tag(A, as.site, pa);
      const int ib = pb == 'I' ? -1 : find_tag(B, bs.site, pb);
      if ((pa != 'I' && ia < 0) || (pb != 'I' && ib < 0)) {
        *why = "an operator product is not carried by the blocks";
        return RMC_OK;
      }
      // -M = -P V^2 P + (P V P)^2: the product term enters negated
      const double c = -terms[s].coef * terms[t].coef * sa * sb;
      bool merged = false;
      for (KTerm& k : kt)
        if (k.qs < 0 && k.ia == ia && k.ib == ib) { k.coef += c; merged = true; break; }
      if (!merged) kt.push_back(KTerm{ia, ib, -1, -1, c});
    }
  for (int s = 0; s < nt; ++s)
    for (int t = 0; t < nt; ++t) kt.push_back(KTerm{-1, -1, s, t, terms[s].coef * terms[t].coef});
  const int no = (int)kt.size();
  if (no > kMaxOps) {
    *why = "too many coupling terms for the product operator";
    return RMC_OK;
  }
  Workspace ws(ctx);
  double *Am, *Bm, *Acat, *EA, *EB, *D, *dmm;
  int* idx;
  TRY(ws.get(&Am, (size_t)no * kA * kA));
  TRY(ws.get(&Bm, (size_t)no * kB * kB));
  TRY(ws.get(&Acat, (size_t)no * kA * kA));
  TRY(ws.get(&EA, kA));
  TRY(ws.get(&EB, kB));
  TRY(ws.get(&D, n));
  TRY(ws.get(&dmm, 2));
  CK(cudaMemsetAsync(EA, 0, sizeof(double) * kA, ctx->stream));
  CK(cudaMemsetAsync(EB, 0, sizeof(double) * kB, ctx->stream));
  Coefs cf{};
  double norm_bound = 0.0;
  auto put = [&](const rmc_block* X, int k, int i, double* dst) -> rmc_status {
    if (i < 0) {
      identity_fill_kernel<<<grid1d((long)k * k), 256, 0, ctx->stream>>>(dst, k);
      CKL();
    } else {
      CK(cudaMemcpyAsync(dst, X->ops + (size_t)i * k * k, sizeof(double) * k * k, cudaMemcpyDeviceToDevice,
                         ctx->stream));
    }
    return RMC_OK;
  };
  for (int j = 0; j < no; ++j) {
    const KTerm& t = kt[j];
    double* aj = Am + (size_t)j * kA * kA;
    double* bj = Bm + (size_t)j * kB * kB;
    cf.c[j] = t.coef;
    if (t.qs < 0) {
      TRY(put(A, kA, t.ia, aj));
      TRY(put(B, kB, t.ib, bj));
      norm_bound += std::fabs(t.coef) * (t.ia < 0 ? 1.0 : A->opnorm[t.ia]) * (t.ib < 0 ? 1.0 : B->opnorm[t.ib]);
    } else {
      // o^s o^t of the projected operators (the square of the coupling of Eq. (7))
      const int as = terms[t.qs].op_a, at = terms[t.qt].op_a, bs = terms[t.qs].op_b, bt = terms[t.qt].op_b;
      TRY((small_mm<double, false, false>(ctx, A->ops + (size_t)as * kA * kA, A->ops + (size_t)at * kA * kA, kA, aj,
                                          1.0, 0.0, nullptr)));
      TRY((small_mm<double, false, false>(ctx, B->ops + (size_t)bs * kB * kB, B->ops + (size_t)bt * kB * kB, kB, bj,
                                          1.0, 0.0, nullptr)));
      norm_bound += std::fabs(t.coef) * A->opnorm[as] * A->opnorm[at] * B->opnorm[bs] * B->opnorm[bt];
    }
  }
  build_acat_kernel<double><<<grid1d((long)kA * kA * no), 256, 0, ctx->stream>>>(Am, cf, kA, no, Acat);
  CKL();
  KronOp<double> K;
  K.kA = kA;
  K.kB = kB;
  K.n_ops = no;
  K.EA = EA;
  K.EB = EB;
  K.Acat = Acat;
  K.Bcat = Bm;
  // start block: the smallest diagonal entries of -M; the whole space when it is small
  const int bsz = (int)std::min<long>(n, n <= 48 ? n : 32);
  TRY(ws.get(&idx, bsz));
  diag_kernel<<<grid1d(n), 256, 0, ctx->stream>>>(EA, EB, Am, Bm, cf, no, kA, kB, D);
  CKL();
  select_smallest_kernel<<<1, 1024, 0, ctx->stream>>>(D, n, bsz, idx, dmm);
  CKL();
  double hdmm[2];
  TRY(to_host<double>(ctx, dmm, hdmm, 2));
  const double ub = hdmm[1] + norm_bound + 1e-12 * std::max(1.0, hdmm[1] + norm_bound);
  double *X, *HX, *th;
  TRY(ws.get(&X, (size_t)bsz * n));
  TRY(ws.get(&HX, (size_t)bsz * n));
  TRY(ws.get(&th, bsz));
  int iters = 0;
  bool conv = false;
  TRY((chfsi<double>(ctx, ws, K, bsz, 1, idx, ub, 1e-11, ctx->cfg.max_iter, X, HX, th, &iters, &conv, true)));
  double th0 = 0.0;
  TRY(to_host<double>(ctx, th, &th0, 1));
  if (!conv) return fail(ctx, RMC_ERR_NOCONV, "coupling norm: the eigensolve did not converge in %d iterations", iters);
  *b_out = std::sqrt(std::max(0.0, -th0));
  *available = true;
  return RMC_OK;
}

// The merged block's Hamiltonian on its own 2^L computational basis and the
// projector onto the retained product sector, P = W W^T with W = U_A (x) U_B
// (U_A: kA lifted kept states of A, vector-major kA x 2^LA; U_B likewise).
struct FullSpace {
  int L = 0;
  long dim = 0;
  const FullTerm* terms = nullptr;  // device
  int nt = 0;
  const double* UA = nullptr;
  const double* UB = nullptr;
  int kA = 0, kB = 0, LA = 0, LB = 0;
};

// out = x - P x: c = U_A X U_B^T (X the 2^LA x 2^LB reshaping of x, A's sites
// the more significant bits), then P x = U_A^T c U_B.
rmc_status project_q(rmc_ctx* ctx, const FullSpace& fs, const double* x, double* out) {
  Workspace ws(ctx);
  const long nA = 1L << fs.LA, nB = 1L << fs.LB;
  double *G1, *Cm, *T2;
  TRY(ws.get(&G1, (size_t)nA * fs.kB));
  TRY(ws.get(&Cm, (size_t)fs.kA * fs.kB));
  TRY(ws.get(&T2, (size_t)fs.kA * nB));
  TRY(gram<double>(ctx, ws, x, (int)nA, fs.UB, fs.kB, nB, G1, false));
  TRY(combine<double>(ctx, fs.UA, false, fs.kA, (int)nA, G1, fs.kB, Cm, 1.0, 0.0, nullptr));
  TRY(combine<double>(ctx, Cm, false, fs.kA, fs.kB, fs.UB, nB, T2, 1.0, 0.0, nullptr));
  TRY(combine<double>(ctx, fs.UA, true, (int)nA, fs.kA, T2, nB, out, -1.0, 1.0, x));
  return RMC_OK;
}

// Lowest eigenvalue of a symmetric operator S on R^n by a Krylov-Rayleigh-Ritz
// method in FP64: Lanczos vectors with two classical Gram-Schmidt passes
// against all earlier ones (full reorthogonalisation), the Rayleigh-Ritz
// matrix V^T S V formed from the stored products, explicit restarts from the
// lowest Ritz vector.  apply(x, y) sets y = S x; keep(x, tmp) maps x into the
// invariant subspace the solve is restricted to (in place, tmp a scratch
// vector; a no-op for the whole space).  Converged when the Ritz vector's
// residual is below tol * max(1, |theta|), when the Krylov space is exhausted
// (its Ritz values are then exact), or when theta has not moved by 1e-13
// relative over 16 steps (the value alone is wanted, and a near-degenerate
// partner can keep the vector's residual up long after the value settled).
template <class Apply, class Keep>
rmc_status krylov_lowest(rmc_ctx* ctx, long n, long dim_eff, double tol, Apply&& apply, Keep&& keep, double* lam) {
  const int m = (int)std::min<long>(96, dim_eff);
  constexpr int kRestarts = 30;
  Workspace ws(ctx);
  double *V, *SV, *tmp, *h, *G, *w, *Z, *z0, *x0, *sx0, *rn, *nrm;
  TRY(ws.get(&V, (size_t)m * n));
  TRY(ws.get(&SV, (size_t)m * n));
  TRY(ws.get(&tmp, (size_t)n));
  TRY(ws.get(&x0, (size_t)n));
  TRY(ws.get(&sx0, (size_t)n));
  TRY(ws.get(&h, (size_t)m));
  TRY(ws.get(&G, (size_t)m * m));
  TRY(ws.get(&w, (size_t)m));
  TRY(ws.get(&Z, (size_t)m * m));
  TRY(ws.get(&z0, (size_t)m * m));
  TRY(ws.get(&rn, 1));
  TRY(ws.get(&nrm, 1));
  seeded_vector_kernel<<<grid1d(n), 256, 0, ctx->stream>>>(V, n, 2609ull);
  CKL();
  TRY(keep(V, tmp));
  normalize_kernel<double><<<1, 1024, 0, ctx->stream>>>(V, n, nullptr);
  CKL();
  double th_prev = NAN;
  for (int rs = 0; rs < kRestarts; ++rs) {
    for (int j = 0; j < m; ++j) {
      double* vj = V + (size_t)j * n;
      TRY(apply(vj, SV + (size_t)j * n));
      bool breakdown = false;
      if (j + 1 < m) {
        double* vn = V + (size_t)(j + 1) * n;
        CK(cudaMemcpyAsync(vn, SV + (size_t)j * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        for (int pass = 0; pass < 2; ++pass) {
          Workspace wl(ctx);
          TRY(gram<double>(ctx, wl, V, j + 1, vn, 1, n, h, false));  // h = V vn (j+1 x 1)
          TRY(combine<double>(ctx, h, true, 1, j + 1, V, n, tmp, -1.0, 1.0, vn));
          CK(cudaMemcpyAsync(vn, tmp, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        TRY(keep(vn, tmp));
        normalize_kernel<double><<<1, 1024, 0, ctx->stream>>>(vn, n, nrm);
        CKL();
        double hn = 0.0;
        TRY(to_host<double>(ctx, nrm, &hn, 1));
        breakdown = !(hn > 1e-10);  // the Krylov space is invariant: its Ritz values are exact
      }
      const int mj = j + 1;
      if (!(mj % 16 == 0 || mj == m || breakdown)) continue;
      Workspace wl(ctx);
      TRY(gram<double>(ctx, wl, V, mj, SV, mj, n, G, true));
      TRY(syev64(ctx, wl, G, mj, w, Z));
      columns_to_vectors_kernel<double><<<grid1d((long)mj), 256, 0, ctx->stream>>>(Z, mj, 1, z0);
      CKL();
      TRY(combine<double>(ctx, z0, false, 1, mj, V, n, x0, 1.0, 0.0, nullptr));
      TRY(combine<double>(ctx, z0, false, 1, mj, SV, n, sx0, 1.0, 0.0, nullptr));
      CK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
      residual_kernel<double><<<1, 1024, 0, ctx->stream>>>(x0, sx0, w, n, 1, tol, rn, ctx->d_status);
      CKL();
      int fails = 0;
      TRY(read_status(ctx, &fails, 1));
      double th0 = 0.0;
      TRY(to_host<double>(ctx, w, &th0, 1));
      const bool steady = std::fabs(th0 - th_prev) <= 1e-13 * std::max(1.0, std::fabs(th0));
      th_prev = th0;
      if (fails == 0 || breakdown || steady) {
        *lam = th0;
        return RMC_OK;
      }
      if (mj == m) break;
    }
    // restart from the lowest Ritz vector
    CK(cudaMemcpyAsync(V, x0, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    TRY(keep(V, tmp));
    normalize_kernel<double><<<1, 1024, 0, ctx->stream>>>(V, n, nullptr);
    CKL();
  }
  return fail(ctx, RMC_ERR_NOCONV, "Krylov eigensolve did not converge (dimension %ld)", n);
}

// out (2^L) = W x = U_A^T X U_B for x the kA x kB coefficient matrix X of a
// product-basis vector of the merge (its state lifted to the block's basis).
rmc_status lift_product(rmc_ctx* ctx, const FullSpace& fs, const double* x, double* out) {
  Workspace ws(ctx);
  const long nB = 1L << fs.LB;
  double* T1;
  TRY(ws.get(&T1, (size_t)fs.kA * nB));
  TRY(combine<double>(ctx, x, false, fs.kA, fs.kB, fs.UB, nB, T1, 1.0, 0.0, nullptr));
  TRY(combine<double>(ctx, fs.UA, true, (int)(1L << fs.LA), fs.kA, T1, nB, out, 1.0, 0.0, nullptr));
  return RMC_OK;
}

// out (kA x kB) = alpha W^T y = alpha U_A Y U_B^T: a block-basis vector's
// coefficients in the retained product basis.
rmc_status restrict_product(rmc_ctx* ctx, const FullSpace& fs, const double* y, double* out, double alpha) {
  Workspace ws(ctx);
  const long nA = 1L << fs.LA, nB = 1L << fs.LB;
  double* G1;
  TRY(ws.get(&G1, (size_t)nA * fs.kB));
  TRY(gram<double>(ctx, ws, y, (int)nA, fs.UB, fs.kB, nB, G1, false));
  TRY(combine<double>(ctx, fs.UA, false, fs.kA, (int)nA, G1, fs.kB, out, alpha, 0.0, nullptr));
  return RMC_OK;
}

// Pauli-string terms of the block [lo, hi) of a chain, on its own sites.
std::vector<FullTerm> block_full_terms(const std::vector<CTerm>& terms, int lo, int hi) {
  const int L = hi - lo;
  std::vector<FullTerm> out;
  auto bit = [&](int site) { return 1ull << (L - 1 - (site - lo)); };
  auto add = [&](FullTerm& f, int site, char p) {
    if (p == 'X' || p == 'Y') f.flip |= bit(site);
    if (p == 'Z' || p == 'Y') f.sign |= bit(site);
  };
  for (const CTerm& t : terms) {
    const bool in = t.j < 0 ? (t.i >= lo && t.i < hi) : (t.i >= lo && t.j < hi);
    if (!in) continue;
    FullTerm f{0, 0, t.coef};
    add(f, t.i, t.pi);
    if (t.j >= 0) {
      add(f, t.j, t.pj);
      if (t.pi == 'Y' && t.pj == 'Y') f.coef = -t.coef;  // YY = -(iY)(iY)
    } else if (t.pi == 'Y') {
      f.coef = NAN;  // a lone Y is imaginary: not a real Hamiltonian term
    }
    out.push_back(f);
  }
  return out;
}

// The recursion loop of Algorithm 1 over a chain, optionally carrying extra
// single-site operators (observables) to the top and lifting the top states.
rmc_status solve_chain_core(rmc_ctx* ctx, int n_sites, int L0, int k, int q, int n_onsite, const int* onsite_site,
                            const char* onsite_pauli, const double* onsite_coef, int n_bonds, const int* bond_i,
                            const int* bond_j, const char* bond_pauli_i, const char* bond_pauli_j,
                            const double* bond_coef, int n_obs, const rmc_op_tag* obs, double* E_out,
                            double* obs_out, double* psi_out, int diag_sites = 0, int max_diag = 0,
                            rmc_merge_diag* diag = nullptr, int* n_diag = nullptr) {
  TRY(check_ctx(ctx));
  if (n_sites < 1 || L0 < 1 || k < 1 || q < 1 || n_onsite < 0 || n_bonds < 0 || !E_out || n_obs < 0 ||
      (n_obs > 0 && (!obs || !obs_out)))
    return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain: bad arguments");
  if (psi_out && n_sites > kMaxLiftSites)
    return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain_states: lifting needs n_sites <= %d", kMaxLiftSites);
  std::vector<CTerm> terms;
  for (int t = 0; t < n_onsite; ++t) {
    if (onsite_site[t] < 0 || onsite_site[t] >= n_sites)
      return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain: on-site term %d out of range", t);
    terms.push_back(CTerm{onsite_site[t], -1, (char)toupper(onsite_pauli[t]), 0, onsite_coef[t]});
  }
  for (int t = 0; t < n_bonds; ++t) {
    if (bond_i[t] < 0 || bond_j[t] >= n_sites || bond_i[t] >= bond_j[t])
      return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain: bond %d out of range", t);
    terms.push_back(CTerm{bond_i[t], bond_j[t], (char)toupper(bond_pauli_i[t]), (char)toupper(bond_pauli_j[t]),
                          bond_coef[t]});
  }
  std::vector<std::pair<int, char>> observables;
  for (int o = 0; o < n_obs; ++o) {
    const char p = (char)toupper(obs[o].pauli);
    if (obs[o].site < 0 || obs[o].site >= n_sites || (p != 'X' && p != 'Y' && p != 'Z'))
      return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain_states: observable %d is not a site Pauli", o);
    observables.push_back({obs[o].site, p});
  }
  if (L0 > 2 * kDenseLeafSites)
    return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain: leaves of more than %d sites are not supported",
                2 * kDenseLeafSites);
  std::vector<ChainNode> nodes;
  build_tree(nodes, 0, n_sites, L0);
  const size_t n_tree = nodes.size();
  for (size_t id = 0; id < n_tree; ++id) {
    if (nodes[id].left >= 0 || nodes[id].hi - nodes[id].lo <= kDenseLeafSites) continue;
    const int lo = nodes[id].lo, hi = nodes[id].hi, mid = lo + (hi - lo) / 2;
    if (id != 0 && k >= (1 << (hi - lo)))
      return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain: k = %d keeps a whole %d-site leaf; use k < %d", k, hi - lo,
                  1 << (hi - lo));
    ChainNode l{lo, mid}, r{mid, hi};
    l.sub = r.sub = true;
    nodes.push_back(l);
    nodes.push_back(r);
    nodes[id].left = (int)nodes.size() - 2;
    nodes[id].right = (int)nodes.size() - 1;
  }
  // carried operators per node: inside ends of terms crossing its boundary,
  // plus every observable on its sites (rotated up to the top); nodes with
  // one signature carry the union so one block serves them all.
  std::map<std::string, std::set<std::pair<int, char>>> need;
  for (ChainNode& nd : nodes) {
    nd.sig = (nd.sub ? std::string("all|") : std::string()) + signature(terms, nd.lo, nd.hi);
    auto& st = need[nd.sig];
    for (const CTerm& t : terms) {
      if (t.j < 0) continue;
      const bool iin = t.i >= nd.lo && t.i < nd.hi, jin = t.j >= nd.lo && t.j < nd.hi;
      if (iin && !jin) st.insert({t.i - nd.lo, t.pi});
      if (jin && !iin) st.insert({t.j - nd.lo, t.pj});
    }
  }
  // observables: a site's operator rides on every block containing it; the
  // signature gains the observed sites so that such blocks are not shared
  // with unobserved twins elsewhere in the chain
  if (!observables.empty()) {
    for (ChainNode& nd : nodes) {
      std::string extra;
      for (auto& o : observables)
        if (o.first >= nd.lo && o.first < nd.hi) extra += std::to_string(o.first - nd.lo) + o.second + ",";
      if (extra.empty()) continue;
      auto base = need[nd.sig];
      nd.sig = "obs:" + extra + "|" + nd.sig;
      auto& st = need[nd.sig];
      st.insert(base.begin(), base.end());
      for (auto& o : observables)
        if (o.first >= nd.lo && o.first < nd.hi) st.insert({o.first - nd.lo, o.second});
    }
  }
  for (ChainNode& nd : nodes) nd.carry.assign(need[nd.sig].begin(), need[nd.sig].end());

  // Build level by level: the leaves, then every merge of one height as one
  // batch (independent merges of Algorithm 1's recursion run at once on the
  // context's lanes).  Blocks with equal signatures are built once.
  std::vector<int> height(nodes.size(), 0);
  std::function<int(int)> measure = [&](int id) -> int {
    if (nodes[id].left < 0) return height[id] = 0;
    return height[id] = 1 + std::max(measure(nodes[id].left), measure(nodes[id].right));
  };
  measure(0);
  std::map<std::string, rmc_block*> cache;
  std::vector<rmc_block*> owned;
  std::vector<rmc_block*> blk_of(nodes.size(), nullptr);
  rmc_status soft = RMC_OK;
  auto cleanup = [&]() {
    for (rmc_block* b : owned) free_block(ctx, b);
  };
  auto bail = [&](rmc_status st) {
    std::string e = ctx->err;
    cleanup();
    ctx->err = e;
    return st;
  };
  for (size_t id = 0; id < nodes.size(); ++id) {
    const ChainNode& nd = nodes[id];
    if (nd.left >= 0) continue;
    const bool top = id == 0;
    if (!top) {
      auto it = cache.find(nd.sig);
      if (it != cache.end()) { blk_of[id] = it->second; continue; }
    }
    const int L = nd.hi - nd.lo;
    std::vector<int> os, bi, bj;
    std::vector<char> op, pi, pj;
    std::vector<double> oc, bc;
    for (const CTerm& t : terms) {
      if (t.j < 0 && t.i >= nd.lo && t.i < nd.hi) { os.push_back(t.i - nd.lo); op.push_back(t.pi); oc.push_back(t.coef); }
      if (t.j >= 0 && t.i >= nd.lo && t.j < nd.hi) {
        bi.push_back(t.i - nd.lo); bj.push_back(t.j - nd.lo); pi.push_back(t.pi); pj.push_back(t.pj); bc.push_back(t.coef);
      }
    }
    std::vector<rmc_op_tag> cr;
    for (auto& c : nd.carry) cr.push_back(rmc_op_tag{c.first, c.second});
    rmc_block* blk = nullptr;
    rmc_status st = rmc_build_leaf_pauli(ctx, L, (top || nd.sub) ? (1 << L) : k, (int)os.size(), os.data(), op.data(),
                                         oc.data(), (int)bi.size(), bi.data(), bj.data(), pi.data(), pj.data(),
                                         bc.data(), (int)cr.size(), cr.data(), &blk);
    if (st != RMC_OK) return bail(st);
    owned.push_back(blk);
    if (!top) cache[nd.sig] = blk;
    blk_of[id] = blk;
  }
  // coupling terms of the merge at an inner node, in its children's carried operators
  auto merge_terms_of = [&](int id, std::vector<rmc_term>* mt) -> bool {
    const ChainNode& nd = nodes[id];
    const rmc_block* A = blk_of[nd.left];
    const rmc_block* B = blk_of[nd.right];
    const int Alo = nodes[nd.left].lo, Blo = nodes[nd.right].lo, Bhi = nodes[nd.right].hi;
    mt->clear();
    for (const CTerm& t : terms) {
      if (t.j < 0 || !(t.i >= Alo && t.i < Blo && t.j >= Blo && t.j < Bhi)) continue;
      const int oa = find_tag(A, t.i - Alo, t.pi), ob = find_tag(B, t.j - Blo, t.pj);
      if (oa < 0 || ob < 0) return false;
      // Y Y = -(iY)(iY): carried Y operators are iY
      mt->push_back(rmc_term{(t.pi == 'Y' && t.pj == 'Y') ? -t.coef : t.coef, oa, ob});
    }
    return true;
  };
  for (int h = 1; h <= height[0]; ++h) {
    std::vector<int> ids, dup;
    std::set<std::string> queued;
    std::vector<std::vector<rmc_term>> mts;
    std::vector<std::vector<rmc_carry>> cys;
    std::vector<int> keeps, flags;
    for (size_t id = 0; id < nodes.size(); ++id) {
      const ChainNode& nd = nodes[id];
      if (nd.left < 0 || height[id] != h) continue;
      const bool top = id == 0;
      if (!top) {
        auto it = cache.find(nd.sig);
        if (it != cache.end()) { blk_of[id] = it->second; continue; }
        if (queued.count(nd.sig)) { dup.push_back((int)id); continue; }
        queued.insert(nd.sig);
      }
      const rmc_block* A = blk_of[nd.left];
      const rmc_block* B = blk_of[nd.right];
      const int Alo = nodes[nd.left].lo, Blo = nodes[nd.right].lo;
      std::vector<rmc_term> mt;
      if (!merge_terms_of((int)id, &mt))
        return bail(fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain: missing carried operator"));
      std::vector<rmc_carry> cy;
      for (auto& c : nd.carry) {  // the top carries only observables
        const int gsite = nd.lo + c.first;
        if (gsite < Blo) cy.push_back(rmc_carry{0, find_tag(A, gsite - Alo, c.second)});
        else cy.push_back(rmc_carry{1, find_tag(B, gsite - Blo, c.second)});
        if (cy.back().op < 0)
          return bail(fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain: missing operator to carry"));
      }
      ids.push_back((int)id);
      mts.push_back(std::move(mt));
      cys.push_back(std::move(cy));
      keeps.push_back(top ? q : k);
      flags.push_back(top ? RMC_COUPLE_TOP : 0);
    }
    const int nb = (int)ids.size();
    std::vector<rmc_couple_desc> descs(nb);
    for (int b = 0; b < nb; ++b) {
      const ChainNode& nd = nodes[ids[b]];
      descs[b] = rmc_couple_desc{blk_of[nd.left], blk_of[nd.right], mts[b].data(), (int)mts[b].size(), keeps[b],
                                 cys[b].data(), (int)cys[b].size(), flags[b]};
    }
    std::vector<rmc_block*> outs(nb, nullptr);
    std::vector<rmc_status> sts(nb, RMC_OK);
    const rmc_status st = rmc_couple_batch(ctx, nb, descs.data(), outs.data(), sts.data());
    for (int b = 0; b < nb; ++b)
      if (outs[b]) owned.push_back(outs[b]);
    if (st != RMC_OK && st != RMC_ERR_NOCONV) return bail(st);
    if (st == RMC_ERR_NOCONV) soft = st;
    for (int b = 0; b < nb; ++b) {
      const ChainNode& nd = nodes[ids[b]];
      rmc_block* blk = outs[b];
      // re-base inherited tags to this block's first site
      for (size_t j = 0; j < cys[b].size(); ++j) {
        const ChainNode& src = nodes[cys[b][j].side == 0 ? nd.left : nd.right];
        blk->tags[j].site += src.lo - nd.lo;
      }
      if (ids[b] != 0) cache[nd.sig] = blk;
      blk_of[ids[b]] = blk;
    }
    for (int id : dup) blk_of[id] = cache[nodes[id].sig];
  }
  rmc_block* topb = blk_of[0];
  rmc_status st = RMC_OK;
  const int qe = std::min(q, topb->k);
  std::vector<double> E(qe);
  st = rmc_lowest(ctx, topb, q, E.data(), nullptr, nullptr);
  for (int i = 0; i < q; ++i) E_out[i] = i < qe ? E[i] : NAN;
  if (st == RMC_OK && n_obs > 0) {
    // <psi_mu| O |psi_nu> = the carried operator in the top basis, q x q
    std::vector<double> m((size_t)topb->k * topb->k);
    for (int o = 0; o < n_obs && st == RMC_OK; ++o) {
      const int j = find_tag(topb, observables[o].first, observables[o].second);
      double* dst = obs_out + (size_t)o * q * q;
      if (j < 0) { st = fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain_states: observable not carried"); break; }
      if (cudaMemcpy(m.data(), topb->ops + (size_t)j * topb->k * topb->k, sizeof(double) * m.size(),
                     cudaMemcpyDeviceToHost) != cudaSuccess) {
        st = fail(ctx, RMC_ERR_CUDA, "rmc_solve_chain_states: copy of an observable failed");
        break;
      }
      for (int a = 0; a < q; ++a)
        for (int b = 0; b < q; ++b) dst[(size_t)a * q + b] = (a < qe && b < qe) ? m[(size_t)a * topb->k + b] : NAN;
    }
  }
  if (st == RMC_OK && psi_out) {
    Workspace ws(ctx);
    double* psi = nullptr;
    st = lift_block(ctx, ws, nodes, blk_of, 0, qe, &psi);
    if (st == RMC_OK) {
      const size_t len = (size_t)1 << n_sites;
      if (cudaMemcpyAsync(psi_out, psi, sizeof(double) * qe * len, cudaMemcpyDeviceToHost, ctx->stream) !=
              cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess)
        st = fail(ctx, RMC_ERR_CUDA, "rmc_solve_chain_states: copy of the states failed");
      for (size_t i = (size_t)qe * len; i < (size_t)q * len; ++i) psi_out[i] = NAN;
    }
  }
  if (st == RMC_OK && diag) {
    // one record per merge, children before parents; merges of equal
    // signature (homogeneous reuse) share their numbers
    std::vector<int> order;
    std::function<void(int)> post = [&](int id) {
      if (nodes[id].left < 0) return;
      post(nodes[id].left);
      post(nodes[id].right);
      order.push_back(id);
    };
    post(0);
    *n_diag = (int)order.size();
    std::map<std::string, rmc_merge_diag> seen;
    for (int i = 0; i < (int)order.size() && i < max_diag && st == RMC_OK; ++i) {
      const int id = order[i];
      const ChainNode& nd = nodes[id];
      const rmc_block* A = blk_of[nd.left];
      const rmc_block* B = blk_of[nd.right];
      rmc_merge_diag dg{};
      auto hit = id != 0 ? seen.find(nd.sig) : seen.end();
      if (hit != seen.end()) {
        dg = hit->second;
      } else {
        dg.kA = A->k;
        dg.kB = B->k;
        dg.k = blk_of[id]->k;
        dg.b = dg.bH = dg.gamma = dg.r = dg.E0 = NAN;
        st = to_host<double>(ctx, blk_of[id]->E, &dg.a, 1);
        std::vector<rmc_term> mt;
        if (st == RMC_OK && !merge_terms_of(id, &mt))
          st = fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain_bounds: missing carried operator");
        bool avail = false;
        std::string why;
        const int L = nd.hi - nd.lo;
        const int LA = nodes[nd.left].hi - nodes[nd.left].lo, LB = nodes[nd.right].hi - nodes[nd.right].lo;
        const bool all_kept = LA < 31 && LB < 31 && A->k == (1L << LA) && B->k == (1L << LB);
        if (all_kept) {  // P = I: b vanishes exactly (its Kronecker form would leave rounding)
          dg.b = 0.0;
          avail = true;
        } else if (st == RMC_OK) {
          st = coupling_norm(ctx, A, B, mt.data(), (int)mt.size(), &dg.b, &avail, &why);
        }
        std::vector<FullTerm> ft = block_full_terms(terms, nd.lo, nd.hi);
        bool real_terms = true;
        for (const FullTerm& f : ft) real_terms = real_terms && std::isfinite(f.coef);
        if (st == RMC_OK && L <= diag_sites && real_terms) {
          Workspace wd(ctx);
          FullSpace fs;
          fs.L = L;
          fs.dim = 1L << L;
          fs.nt = (int)ft.size();
          fs.kA = A->k;
          fs.kB = B->k;
          fs.LA = LA;
          fs.LB = LB;
          FullTerm* dterms = nullptr;
          double *UA = nullptr, *UB = nullptr;
          st = wd.get(&dterms, std::max<size_t>(1, ft.size()));
          if (st == RMC_OK && !ft.empty() &&
              (cudaMemcpyAsync(dterms, ft.data(), sizeof(FullTerm) * ft.size(), cudaMemcpyHostToDevice,
                               ctx->stream) != cudaSuccess ||
               cudaStreamSynchronize(ctx->stream) != cudaSuccess))
            st = fail(ctx, RMC_ERR_CUDA, "rmc_solve_chain_bounds: copy of the block terms failed");
          if (st == RMC_OK) st = lift_block(ctx, wd, nodes, blk_of, nd.left, A->k, &UA);
          if (st == RMC_OK) st = lift_block(ctx, wd, nodes, blk_of, nd.right, B->k, &UB);
          fs.terms = dterms;
          fs.UA = UA;
          fs.UB = UB;
          double *f1 = nullptr, *f2 = nullptr;
          if (st == RMC_OK) st = wd.get(&f1, (size_t)fs.dim);
          if (st == RMC_OK) st = wd.get(&f2, (size_t)fs.dim);
          auto whole = [&](double*, double*) -> rmc_status { return RMC_OK; };
          auto in_q = [&](double* x, double* tmp) -> rmc_status {  // x <- Q x
            TRY(project_q(ctx, fs, x, tmp));
            CK(cudaMemcpyAsync(x, tmp, sizeof(double) * fs.dim, cudaMemcpyDeviceToDevice, ctx->stream));
            return RMC_OK;
          };
          // E0 = lambda_min(H) on the block's whole space
          auto h_apply = [&](const double* x, double* y) -> rmc_status {
            full_apply_kernel<<<grid1d(fs.dim), 256, 0, ctx->stream>>>(fs.terms, fs.nt, fs.dim, x, y);
            CKL();
            return RMC_OK;
          };
          if (st == RMC_OK) st = krylov_lowest(ctx, fs.dim, fs.dim, 1e-9, h_apply, whole, &dg.E0);
          // lambda_min(Q H Q) on range(Q)
          auto qhq_apply = [&](const double* x, double* y) -> rmc_status {
            TRY(project_q(ctx, fs, x, f1));
            TRY(h_apply(f1, f2));
            TRY(project_q(ctx, fs, f2, y));
            return RMC_OK;
          };
          const long nr = (long)A->k * B->k, dq = fs.dim - nr;
          double lq = INFINITY;
          if (st == RMC_OK && dq > 0) st = krylov_lowest(ctx, fs.dim, dq, 1e-9, qhq_apply, in_q, &lq);
          // ||P H Q||_2^2 = lambda_max(W^T H Q H W) on the retained product
          // sector (W = U_A (x) U_B): the lowest eigenvalue of its negative
          auto phq_apply = [&](const double* x, double* y) -> rmc_status {
            TRY(lift_product(ctx, fs, x, f1));
            TRY(h_apply(f1, f2));
            TRY(project_q(ctx, fs, f2, f1));
            TRY(h_apply(f1, f2));
            TRY(restrict_product(ctx, fs, f2, y, -1.0));
            return RMC_OK;
          };
          double mb = 0.0;
          if (st == RMC_OK && dq > 0) st = krylov_lowest(ctx, nr, nr, 1e-9, phq_apply, whole, &mb);
          if (st == RMC_OK) {
            dg.bH = dq > 0 ? std::sqrt(std::max(0.0, -mb)) : 0.0;
            dg.gamma = lq - dg.a;
            if (dg.bH == 0.0 || std::isinf(dg.gamma)) dg.r = 0.0;
            else dg.r = 0.5 * (std::sqrt(dg.gamma * dg.gamma + 4.0 * dg.bH * dg.bH) - dg.gamma);
          }
        }
        if (id != 0) seen[nd.sig] = dg;
      }
      dg.lo = nd.lo;
      dg.mid = nodes[nd.left].hi;
      dg.hi = nd.hi;
      diag[i] = dg;
    }
  }
  cleanup();
  if (st != RMC_OK) return st;
  if (soft != RMC_OK) return fail(ctx, soft, "rmc_solve_chain: a merge did not converge");
  return RMC_OK;
}

}  // namespace

extern "C" rmc_status rmc_solve_chain(rmc_ctx* ctx, int n_sites, int L0, int k, int q, int n_onsite,
                                      const int* onsite_site, const char* onsite_pauli, const double* onsite_coef,
                                      int n_bonds, const int* bond_i, const int* bond_j, const char* bond_pauli_i,
                                      const char* bond_pauli_j, const double* bond_coef, double* E_out) {
  return solve_chain_core(ctx, n_sites, L0, k, q, n_onsite, onsite_site, onsite_pauli, onsite_coef, n_bonds, bond_i,
                          bond_j, bond_pauli_i, bond_pauli_j, bond_coef, 0, nullptr, E_out, nullptr, nullptr);
}

extern "C" rmc_status rmc_solve_chain_states(rmc_ctx* ctx, const rmc_chain* c, int n_obs, const rmc_op_tag* obs,
                                             double* E_out, double* obs_out, double* psi_out) {
  if (!ctx) return RMC_ERR_INVAL;
  if (!c) return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain_states: no chain");
  return solve_chain_core(ctx, c->n_sites, c->L0, c->k, c->q, c->n_onsite, c->onsite_site, c->onsite_pauli,
                          c->onsite_coef, c->n_bonds, c->bond_i, c->bond_j, c->bond_pauli_i, c->bond_pauli_j,
                          c->bond_coef, n_obs, obs, E_out, obs_out, psi_out);
}

extern "C" rmc_status rmc_solve_chain_bounds(rmc_ctx* ctx, const rmc_chain* c, int full_space_sites,
                                             int max_merges, rmc_merge_diag* diag, int* n_merges, double* E_out) {
  if (!ctx) return RMC_ERR_INVAL;
  if (!c || !n_merges || max_merges < 0 || (max_merges > 0 && !diag))
    return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain_bounds: bad arguments");
  if (full_space_sites > kMaxFullSpaceSites)
    return fail(ctx, RMC_ERR_INVAL, "rmc_solve_chain_bounds: full-space evaluation needs <= %d sites",
                kMaxFullSpaceSites);
  std::vector<double> E(std::max(1, c->q));
  rmc_status st = solve_chain_core(ctx, c->n_sites, c->L0, c->k, c->q, c->n_onsite, c->onsite_site, c->onsite_pauli,
                                   c->onsite_coef, c->n_bonds, c->bond_i, c->bond_j, c->bond_pauli_i,
                                   c->bond_pauli_j, c->bond_coef, 0, nullptr, E_out ? E_out : E.data(), nullptr,
                                   nullptr, std::max(0, full_space_sites), max_merges, diag ? diag : nullptr,
                                   n_merges);
  return st;
}

extern "C" rmc_status rmc_merge_bound(rmc_ctx* ctx, const rmc_block* A, const rmc_block* B, const rmc_term* terms,
                                      int n_terms, double* b_out) {
  TRY(check_ctx(ctx));
  if (!A || !B || !b_out || n_terms < 0 || (n_terms > 0 && !terms))
    return fail(ctx, RMC_ERR_INVAL, "rmc_merge_bound: bad arguments");
  for (int t = 0; t < n_terms; ++t)
    if (terms[t].op_a < 0 || terms[t].op_a >= A->n_ops || terms[t].op_b < 0 || terms[t].op_b >= B->n_ops ||
        !std::isfinite(terms[t].coef))
      return fail(ctx, RMC_ERR_INVAL, "rmc_merge_bound: term %d names no carried operator", t);
  bool avail = false;
  std::string why;
  TRY(coupling_norm(ctx, A, B, terms, n_terms, b_out, &avail, &why));
  if (!avail) return fail(ctx, RMC_ERR_INVAL, "rmc_merge_bound: %s", why.c_str());
  return RMC_OK;
}

extern "C" rmc_status rmc_autotune(rmc_ctx* ctx, const rmc_chain* c, double* E_out) {
  if (!ctx) return RMC_ERR_INVAL;
  if (!c) return fail(ctx, RMC_ERR_INVAL, "rmc_autotune: no chain");
  TuneTable& tt = tune_table();
  tt.tuning.fetch_add(1);
  // merges one at a time, so each candidate is timed on an otherwise idle stream
  const int lanes = ctx->cfg.lanes;
  ctx->cfg.lanes = 1;
  std::vector<double> E(std::max(1, c->q));
  const rmc_status st = solve_chain_core(ctx, c->n_sites, c->L0, c->k, c->q, c->n_onsite, c->onsite_site,
                                         c->onsite_pauli, c->onsite_coef, c->n_bonds, c->bond_i, c->bond_j,
                                         c->bond_pauli_i, c->bond_pauli_j, c->bond_coef, 0, nullptr,
                                         E_out ? E_out : E.data(), nullptr, nullptr);
  ctx->cfg.lanes = lanes;
  tt.tuning.fetch_sub(1);
  return st;
}

extern "C" size_t rmc_tune_dump(char* buf, size_t len) {
  TuneTable& tt = tune_table();
  std::string text;
  {
    std::lock_guard<std::mutex> lk(tt.mu);
    for (const auto& kv : tt.choice) text += kv.first + "=" + std::to_string(kv.second) + "\n";
  }
  if (buf && len > 0) {
    const size_t n = std::min(len - 1, text.size());
    std::memcpy(buf, text.data(), n);
    buf[n] = '\0';
  }
  return text.size() + 1;
}

extern "C" int rmc_tune_load(const char* text) {
  if (!text) return -1;
  TuneTable& tt = tune_table();
  std::lock_guard<std::mutex> lk(tt.mu);
  int count = 0;
  const char* p = text;
  while (*p) {
    const char* e = std::strchr(p, '\n');
    const std::string line = e ? std::string(p, e - p) : std::string(p);
    p = e ? e + 1 : p + line.size();
    if (line.empty()) continue;
    const size_t eq = line.rfind('=');
    if (eq == std::string::npos || eq == 0 || eq + 1 >= line.size()) return -1;
    char* end = nullptr;
    const long v = std::strtol(line.c_str() + eq + 1, &end, 10);
    if (!end || *end != '\0' || v < 0 || v > 64) return -1;
    tt.choice[line.substr(0, eq)] = (int)v;
    ++count;
  }
  return count;
}

extern "C" void rmc_tune_clear(void) {
  TuneTable& tt = tune_table();
  std::lock_guard<std::mutex> lk(tt.mu);
  tt.choice.clear();
}

// ---------------------------------------------------------------------------
// Allocation-free Kronecker-form product (a library service; the paper has
// no counterpart).  Its scratch is this fixed device array, not pool memory.
// In host code `g_noalloc_scratch` is only a handle: the device address comes
// from cudaGetSymbolAddress, once per device, cached below.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[RMC_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoallocMaxDevices] = {};

cudaError_t noalloc_scratch_address(int device, void** addr) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // the calling thread's current device
    if (e != cudaSuccess) return e;
    g_noalloc_addr[device] = p;
  }
  *addr = g_noalloc_addr[device];
  return cudaSuccess;
}

template <typename T>
rmc_status noalloc_kron(cudaStream_t st, int kA, int kB, int n_ops, int nv, const T* EA, const T* EB, const T* A,
                        const T* B, const double* coef, const T* X, T* Y, const T* Z, double alpha, double beta,
                        double gamma, unsigned char* scratch) {
  const size_t acat_bytes = ((sizeof(T) * (size_t)std::max(1, n_ops) * kA * kA + 255) / 256) * 256;
  T* Acat = (T*)scratch;
  T* Tbuf = (T*)(scratch + acat_bytes);
  Coefs cf{};
  for (int j = 0; j < n_ops; ++j) cf.c[j] = coef[j];
  // the caller's pending error state was checked on entry, so an error read
  // here comes from the launch just made
  if (n_ops > 0) {
    build_acat_kernel<T><<<grid1d((long)kA * kA * n_ops), 256, 0, st>>>(A, cf, kA, n_ops, Acat);
    if (cudaGetLastError() != cudaSuccess) return RMC_ERR_CUDA;
    GemmShape s1{nv * kA, n_ops * kB, kB, kB, kB, 0, 0, 1};
    EpiKron1<T> e1{Tbuf, kA, kB, nv};
    gemm_big<T, false, true>(X, B, s1, 1, e1, st);
    if (cudaGetLastError() != cudaSuccess) return RMC_ERR_CUDA;
    GemmShape s2{kA, nv * kB, n_ops * kA, (long)n_ops * kA, (long)nv * kB, 0, 0, 1};
    EpiKron2<T> e2{X, Z, EA, EB, Y, kA, kB, (T)alpha, (T)beta, (T)gamma};
    gemm_big<T, false, false>(Acat, Tbuf, s2, 1, e2, st);
  } else {
    // no coupling terms: a K = 0 product whose epilogue forms D o X (the A
    // operand is never read)
    GemmShape s0{kA, nv * kB, 0, 1, (long)nv * kB, 0, 0, 1};
    EpiKron2<T> e2{X, Z, EA, EB, Y, kA, kB, (T)alpha, (T)beta, (T)gamma};
    gemm_big<T, false, false>(EA, X, s0, 1, e2, st);
  }
  return cudaGetLastError() == cudaSuccess ? RMC_OK : RMC_ERR_CUDA;
}
}  // namespace

extern "C" rmc_status rmc_kron_matvec_noalloc(void* stream, int dtype, int kA, int kB, int n_ops, int nv,
                                              const void* EA, const void* EB, const void* A, const void* B,
                                              const double* coef, const void* X, void* Y, const void* Z,
                                              double alpha, double beta, double gamma) {
  if (kA < 1 || kB < 1 || n_ops < 0 || n_ops > kMaxOps || nv < 1 || !EA || !EB || !X || !Y ||
      (n_ops && (!A || !B || !coef)) || (gamma != 0.0 && !Z) || (dtype != 0 && dtype != 1) || X == Y || Z == Y)
    return RMC_ERR_INVAL;
  const size_t elt = dtype == 0 ? sizeof(double) : sizeof(float);
  const size_t need = ((elt * (size_t)std::max(1, n_ops) * kA * kA + 255) / 256) * 256 +
                      elt * (size_t)std::max(1, n_ops) * kA * kB * nv;
  if (need > (size_t)RMC_NOALLOC_SCRATCH_BYTES) return RMC_ERR_NOMEM;
  // an error the caller left pending is reported, not cleared, and nothing
  // is launched on top of it
  if (cudaPeekAtLastError() != cudaSuccess) return RMC_ERR_CUDA;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kNoallocMaxDevices) return RMC_ERR_CUDA;
  void* scratch = nullptr;
  if (noalloc_scratch_address(device, &scratch) != cudaSuccess) return RMC_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == 0)
    return noalloc_kron<double>(st, kA, kB, n_ops, nv, (const double*)EA, (const double*)EB, (const double*)A,
                                (const double*)B, coef, (const double*)X, (double*)Y, (const double*)Z, alpha, beta,
                                gamma, (unsigned char*)scratch);
  return noalloc_kron<float>(st, kA, kB, n_ops, nv, (const float*)EA, (const float*)EB, (const float*)A,
                             (const float*)B, coef, (const float*)X, (float*)Y, (const float*)Z, alpha, beta, gamma,
                             (unsigned char*)scratch);
}
