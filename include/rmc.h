/*
 * rmc.h -- C ABI of the recursive module-coupling eigensolver (B300, sm_103a).
 *
 * The library computes Algorithm 1 of "A Recursive Module-Coupling Algorithm
 * for Computing Low-Energy Eigenstates" (arXiv 2609.02394) on one GPU:
 * diagonalise small leaf modules (Sec. II, Eq. (4)); repeatedly couple two
 * neighbouring blocks A and B, solving for the lowest eigenpairs of the
 * effective Hamiltonian in the product basis of their retained states,
 *     H_eff = diag(E_A[a] + E_B[b]) + sum_j coef_j o_A^j (x) o_B^j      (Eq. (7))
 * (the minus sign of Eq. (3) is folded into coef_j), keeping the lowest states
 * (Eq. (10)) and rotating the boundary operators the next merge needs into the
 * new basis (Algorithm 1, inner loop); return the lowest q eigenpairs of the
 * final block.  The effective Hamiltonian is never formed: every product with
 * it is a Kronecker-form product Y = D o X + sum_j coef_j O_A^j X (O_B^j)^T on
 * the k_A x k_B coefficient matrix X of a product-basis vector.
 *
 * Conventions
 *   - Product-basis index: row = a * k_B + b (a from module A is the slow
 *     index, Eq. (5)); a vector is a row-major k_A x k_B matrix.
 *   - All host arrays are row-major, FP64, owned by the caller and copied at
 *     call time.  All blocks are opaque device-resident handles owned by the
 *     caller and released with rmc_block_free.  No call consumes its inputs.
 *   - Calls are ordered on the context's CUDA stream.  rmc_couple and
 *     rmc_solve_chain synchronise with the host between solver iterations
 *     (convergence is checked on the host); rmc_lowest and the export calls
 *     synchronise before returning.  One context per host thread.
 *   - Every call returns an rmc_status; on failure rmc_last_error(ctx) returns
 *     a one-line description.  A failed call leaves its outputs unset and
 *     frees whatever it allocated.
 *
 * Kernel-level entry points (rmc_kron_matvec, ...) take DEVICE pointers and
 * run one kernel of the hot path on the given stream; they exist so that each
 * step can be checked on its own against the CPU oracle.
 */
#ifndef RMC_H_
#define RMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rmc_status {
  RMC_OK = 0,
  RMC_ERR_INVAL = 1,    /* bad argument: sizes, NaN, asymmetric H, unknown op */
  RMC_ERR_NOMEM = 2,    /* request exceeds the context's device-memory budget */
  RMC_ERR_NOCONV = 3,   /* eigensolver hit max_iter; best Ritz values kept   */
  RMC_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up                 */
  RMC_ERR_CUDA = 5      /* a CUDA runtime call failed                         */
} rmc_status;

typedef enum rmc_precision {
  /* Every floating-point step in FP64 (DFMA): the plain per-solve form. */
  RMC_PREC_FP64 = 0,
  /* Filter, orthogonalisation and Rayleigh-Ritz of the subspace iteration in
   * FP32 (FP32 accumulation); every merge then refines the converged block
   * to an FP64 residual of 1e-8 (Chebyshev filter passes; for blocks wider
   * than the small eigensolver in defect form, FP32 products on the small
   * correction) and ends with the FP64 finalisation (FP64 Cholesky-QR, FP64
   * Rayleigh-Ritz with refined eigenvectors, FP64 rotation), so energies and
   * retained bases are FP64-consistent projections.  The Kronecker products
   * of wide merges (k_A k_B >= 16384, row pitches of 16 bytes) run on the
   * tcgen05 tensor cores in 3xTF32 (FP32 accuracy), the rest on the FP32
   * pipe. */
  RMC_PREC_MIXED = 1,
  /* As RMC_PREC_MIXED with every Kronecker product of the working precision
   * that fits a tensor-core kernel on the tcgen05 tensor cores (3xTF32). */
  RMC_PREC_MIXED_TF32 = 2
} rmc_precision;

typedef struct rmc_config {
  int device;              /* CUDA device ordinal                               */
  void* stream;            /* cudaStream_t to run on; NULL: the library makes one */
  size_t mem_budget;       /* bytes of device memory the context may hold; 0: 40 GiB */
  int precision;           /* rmc_precision                                    */
  double tol;              /* residual tolerance (relative to max(1,|theta|)) of
                              the working-precision solve; <= 0: 1e-11 (FP64),
                              2e-6 (mixed)                                      */
  int max_iter;            /* outer subspace iterations per merge; <= 0: 200   */
  int guard;               /* extra vectors beyond the retained count; <= 0:
                              max(16, k_ret / 2), capped by the dimension       */
  double tau_deg;          /* degenerate-cut threshold; <= 0: 1e-7              */
  int lanes;               /* merges of one level that rmc_solve_chain and
                              rmc_couple_batch run at once, each on its own
                              stream and host thread; <= 0: up to 8; 1: one
                              at a time (the solve server's slots use 1)        */
} rmc_config;

typedef struct rmc_ctx rmc_ctx;
typedef struct rmc_block rmc_block;

/* Tags of the operators a block carries, so that callers can look them up:
 * site index (chain-global) and a Pauli letter ('X', 'Y', 'Z'; 'Y' is carried
 * as the real matrix iY = [[0,1],[-1,0]]) or 'O' for an arbitrary operator. */
typedef struct rmc_op_tag {
  int site;
  char pauli;
} rmc_op_tag;

/* One coupling term of a merge: coef * o_A[op_a] (x) o_B[op_b]  (Eq. (3)/(8)). */
typedef struct rmc_term {
  double coef;
  int op_a;
  int op_b;
} rmc_term;

/* An operator to carry into the merged block: side 0 = from A (rotated as
 * C^T (o (x) I) C), side 1 = from B (rotated as C^T (I (x) o) C). */
typedef struct rmc_carry {
  int side;
  int op;
} rmc_carry;

/* Flags of rmc_couple. */
#define RMC_COUPLE_TOP 1   /* top level: keep exactly k_keep, skip the degenerate cut */

/* ---- context ------------------------------------------------------------ */

/* Create a context on cfg->device (cfg may be NULL for all defaults). */
rmc_status rmc_create(rmc_ctx** ctx, const rmc_config* cfg);
/* Destroy a context; blocks still alive are freed with it. */
rmc_status rmc_destroy(rmc_ctx* ctx);
/* Text of the last error on this context ("" if none).  Owned by ctx. */
const char* rmc_last_error(const rmc_ctx* ctx);
/* Bytes of device memory currently held (blocks + cached workspace). */
size_t rmc_mem_in_use(const rmc_ctx* ctx);
/* Counters since creation: kernel launches issued, outer iterations run. */
rmc_status rmc_stats(const rmc_ctx* ctx, uint64_t* launches, uint64_t* iterations);
/* The stream the context runs on (a cudaStream_t). */
void* rmc_stream(const rmc_ctx* ctx);

/* Opt-in timing of the hot-path kernels on the context stream (CUDA events
 * around every launch group, harvested at the next host synchronisation).
 * Kinds: 0 two-stage Kronecker-form product in the working precision of the
 * subspace iteration (FP32 for the mixed paths), 1 Kronecker-form product in
 * FP64 (either form), 2 small eigensolver (Jacobi + refinement), 3
 * Cholesky-QR, 4 Gram products, 5 basis combinations, 6 operator rotation,
 * 7 single-launch (fused) Chebyshev filter or product in the working
 * precision.  rmc_profile_read returns the totals since the last read (launch
 * groups, milliseconds, algorithmic FLOPs) and resets them. */
#define RMC_PROF_KINDS 8
/* enable: 0 off, 1 every kind, or RMC_PROFILE_MASK | (bit k for each kind k to
 * time): each timed launch group costs two event records, so timing only the
 * kinds of interest keeps the host's launch path as it is without timing. */
#define RMC_PROFILE_MASK 0x100
rmc_status rmc_profile(rmc_ctx* ctx, int enable);
rmc_status rmc_profile_read(rmc_ctx* ctx, int kind, uint64_t* groups, uint64_t* launches, double* ms,
                            double* flops);

/* ---- Algorithm 1 --------------------------------------------------------- */

/* Leaf module (Algorithm 1, first step; Eqs. (4), (9)).
 *   H    : D x D row-major module Hamiltonian; must be symmetric within 1e-12
 *          (relative to max|H|) and finite, else RMC_ERR_INVAL.
 *   k    : number of lowest states to keep; the kept count is min(k, D),
 *          reduced by the degenerate-cut rule so no multiplet is split.
 *   ops  : n_ops pointers to D x D operators to carry (projected o = U^T O U).
 *   tags : n_ops tags (may be NULL).
 * On success *out is a new block with energies (ascending), carried
 * operators and the D x k eigenvector matrix U. 1 <= D <= 256. */
rmc_status rmc_build_leaf(rmc_ctx* ctx, const double* H, int D, int k,
                          const double* const* ops, const rmc_op_tag* tags,
                          int n_ops, rmc_block** out);

/* Pauli-term leaf: the module Hamiltonian of L sites (D = 2^L <= 256) is built
 * on the device from on-site terms coef*P_site and bond terms coef*P_i P_j
 * (site indices local, 0 = most significant factor; Y Y is written as
 * -(iY)(iY)); carried operators are the single-site Paulis in `carry`.
 * onsite: n_onsite triples (site, pauli, coef) packed as
 *         int sites[n], char paulis[n], double coefs[n]; bonds likewise. */
rmc_status rmc_build_leaf_pauli(rmc_ctx* ctx, int L, int k,
                                int n_onsite, const int* onsite_site,
                                const char* onsite_pauli, const double* onsite_coef,
                                int n_bonds, const int* bond_i, const int* bond_j,
                                const char* bond_pauli_i, const char* bond_pauli_j,
                                const double* bond_coef,
                                int n_carry, const rmc_op_tag* carry, rmc_block** out);

/* One merge of Algorithm 1 (inner loop; Eqs. (5)-(10)).
 *   terms  : the coupling V = sum coef o_A[op_a] (x) o_B[op_b]; A and B may be
 *            the same block (homogeneous reuse: identical modules).
 *   k_keep : states to keep: min(k_keep, k_A k_B), then the degenerate-cut rule
 *            (largest k' with theta[k'] - theta[k'-1] > tau max(1,|theta[k']|))
 *            unless flags has RMC_COUPLE_TOP.
 *   carry  : which of A's and B's operators to rotate into the new block
 *            (Algorithm 1: the carried boundary operators are rotated into
 *            the merged basis for the next merge); tags are inherited.
 * The lowest eigenpairs are found by Chebyshev-filtered subspace iteration on
 * the Kronecker-form product, then finalised in FP64.  RMC_ERR_NOCONV when
 * max_iter is reached (*out is still produced from the best iterate). */
rmc_status rmc_couple(rmc_ctx* ctx, const rmc_block* A, const rmc_block* B,
                      const rmc_term* terms, int n_terms, int k_keep,
                      const rmc_carry* carry, int n_carry, int flags,
                      rmc_block** out);

/* One merge of a batch: the arguments of rmc_couple. */
typedef struct rmc_couple_desc {
  const rmc_block* A;
  const rmc_block* B;
  const rmc_term* terms;
  int n_terms;
  int k_keep;
  const rmc_carry* carry;
  int n_carry;
  int flags;
} rmc_couple_desc;

/* n independent merges (for instance every merge of one level of the
 * recursion, Algorithm 1, for one chain or many) run at once: up to
 * cfg.lanes of them concurrently, each on its own CUDA stream and host thread
 * inside the context, sharing its memory pool and budget.  out[i] and
 * status[i] receive each merge's block and status as rmc_couple would return
 * them (out[i] is NULL unless status[i] is RMC_OK or RMC_ERR_NOCONV); the
 * blocks belong to ctx.  The inputs must not be freed while the call runs; the
 * call synchronises before returning, and returns the first failing status
 * (hard errors before RMC_ERR_NOCONV) with that merge's message in
 * rmc_last_error. */
rmc_status rmc_couple_batch(rmc_ctx* ctx, int n, const rmc_couple_desc* descs,
                            rmc_block** out, rmc_status* status);

/* Lowest q energies of a block (Algorithm 1, last step), ascending, into the
 * host array E_out[q]; q is clipped to the block's kept count, which is
 * written to *k_eff_out (may be NULL).  C_out (may be NULL) receives the
 * block's coefficient matrix, row-major (k_A k_B) x q (or D x q for a leaf). */
rmc_status rmc_lowest(rmc_ctx* ctx, const rmc_block* blk, int q, double* E_out,
                      double* C_out, int* k_eff_out);

/* Whole chain (the recursion loop of Algorithm 1): sites 0..n_sites-1 with
 * on-site terms and two-site terms (i < j) as in rmc_build_leaf_pauli but with
 * chain-global site indices; the chain is split into floor/ceil halves until a
 * part has <= L0 sites; every level keeps k states, the top returns q.
 * E_out[q] receives the lowest energies (host). */
rmc_status rmc_solve_chain(rmc_ctx* ctx, int n_sites, int L0, int k, int q,
                           int n_onsite, const int* onsite_site,
                           const char* onsite_pauli, const double* onsite_coef,
                           int n_bonds, const int* bond_i, const int* bond_j,
                           const char* bond_pauli_i, const char* bond_pauli_j,
                           const double* bond_coef, double* E_out);

/* ---- many solves at once: batched and served (continuous batching) -------- */

/* A chain Hamiltonian for the solve calls below (same fields as
 * rmc_solve_chain's arguments; arrays are read at submission and copied). */
typedef struct rmc_chain {
  int n_sites, L0, k, q;
  int n_onsite;
  const int* onsite_site;
  const char* onsite_pauli;
  const double* onsite_coef;
  int n_bonds;
  const int* bond_i;
  const int* bond_j;
  const char* bond_pauli_i;
  const char* bond_pauli_j;
  const double* bond_coef;
} rmc_chain;

/* The chain solve of rmc_solve_chain (for `chain`, described as for the
 * server below) with two optional products for its q lowest states |psi_mu>:
 *   obs_out[o][mu][nu] = <psi_mu| O_o |psi_nu>   (n_obs x q x q, host)
 * for the single-site Pauli observables obs[o] ('X', 'Z', or 'Y' given as the
 * real antisymmetric iY, so the result is -i<psi_mu|Y|psi_nu>): each is
 * carried through every basis rotation on its way to the top block (Sec. II,
 * the projected operators of Algorithm 1), so it costs one k x k operator per
 * block and works at any chain length; and
 *   psi_out[mu][x] = the state lifted to the 2^n_sites computational basis
 * (x = sum_s bit_s 2^(n_sites-1-s), site 0 most significant; the recursive
 * product of Eq. (11) psi = (U_A (x) U_B) C), for n_sites <= 24 (else
 * RMC_ERR_INVAL), q x 2^n_sites host doubles.  Either may be NULL (obs_out
 * only when n_obs = 0).  States beyond the top block's kept count are NaN.
 * Observed sites make their blocks distinct from unobserved twins, so
 * homogeneous reuse covers fewer blocks.  The paper has these as the
 * fidelities of Sec. III A and the state-lifting of Eq. (11).  Synchronises. */
rmc_status rmc_solve_chain_states(rmc_ctx* ctx, const struct rmc_chain* chain, int n_obs,
                                  const rmc_op_tag* obs, double* E_out, double* obs_out,
                                  double* psi_out);

/* ---- per-merge truncation diagnostics (Sec. IV and Appendix B) ----------- */

/* For a merge of modules A and B, P projects the merged block's Hilbert space
 * onto the retained product sector span{|a>|b>} of A's and B's kept states and
 * Q = I - P.  With H the merged block's Hamiltonian and V its inter-module
 * coupling, the paper bounds the merge's ground-energy error by
 *     0 <= a - E0 <= r(b, gamma) = (sqrt(gamma^2 + 4 b^2) - gamma) / 2 <= b^2 / gamma
 * (Sec. IV, Appendix B), where a = lambda_min(PHP), b = ||PHQ||_2 = ||PVQ||_2,
 * gamma = lambda_min(QHQ on range Q) - a, E0 = lambda_min(H). */
typedef struct rmc_merge_diag {
  int lo, mid, hi;   /* module A = sites [lo, mid), module B = [mid, hi) (chain-global)  */
  int kA, kB, k;     /* kept states of A, of B, and of the merged block                   */
  double a;          /* lowest eigenvalue of the merge's H_eff (Eq. (7)): the block's E[0] */
  double b;          /* ||P V Q||_2 in Kronecker form (Appendix B's expression); NaN when V's
                        operator products are not carried (b needs [O^s O^t] for every pair
                        of coupling operators on one side: single-site Paulis multiply to
                        carried Paulis, operators on two different sites of one module do
                        not).  Equals ||P H Q||_2 when both modules' kept states are exact
                        eigenstates of their own Hamiltonians (leaves); for merged modules
                        H_A (x) I also leaks out of the sector and bH below is the bound's b */
  double bH;         /* ||P H Q||_2 on the block's full space; NaN when not evaluated      */
  double gamma;      /* lambda_min(QHQ) - a; +inf when Q = 0 (every state kept); NaN when
                        the block is not evaluated on its full space                       */
  double r;          /* r(bH, gamma) above; 0 when bH = 0 or Q = 0; NaN when not evaluated */
  double E0;         /* exact ground energy of the merged block's own Hamiltonian; NaN when
                        not evaluated                                                      */
} rmc_merge_diag;

/* b = ||P V Q||_2 for the merge of A and B with coupling V = sum_t coef_t
 * o_A[op_a] (x) o_B[op_b] (the terms of rmc_couple), computed in Kronecker form
 * on the device from b^2 = lambda_max(P V^2 P - (P V P)^2) on range(P)
 * (Appendix B): P V P is the coupling of Eq. (7), and P V^2 P is assembled from
 * the blocks' carried operators, since two Paulis on one site multiply to +-(a
 * Pauli or the identity).  Blocks must be tagged with single-site Paulis and
 * must carry every such product (the chain solver's blocks do for
 * nearest-neighbour couplings); otherwise RMC_ERR_INVAL.  FP64 subspace
 * iteration on the Kronecker sum -M, residual 1e-12.  *b_out on the host.
 * Synchronises. */
rmc_status rmc_merge_bound(rmc_ctx* ctx, const rmc_block* A, const rmc_block* B, const rmc_term* terms,
                           int n_terms, double* b_out);

/* The chain solve of rmc_solve_chain_states (E_out[q] as there) plus one
 * rmc_merge_diag per merge of the recursion tree, children before parents
 * (post-order; merges of equal signature share their numbers).  *n_merges
 * receives the number of merges; the first min(*n_merges, max_merges) records
 * are written to diag.  a and b are evaluated for every merge; E0, bH, gamma
 * and r for merged blocks of at most full_space_sites sites (<= 22, else
 * RMC_ERR_INVAL; 0: none), on the block's 2^L computational basis by an FP64
 * Krylov-Rayleigh-Ritz method with full reorthogonalisation (residual 1e-9
 * relative, or the value settled to 1e-13): the lowest eigenvalue of the
 * block's Hamiltonian, that of Q H Q on range(Q) with Q formed from the
 * children's lifted kept states, and the largest of W^T H Q H W on the
 * retained sector (W = U_A (x) U_B).  The paper evaluates these for its 10- and
 * 20-site validation (Appendix B figure).
 * Synchronises. */
rmc_status rmc_solve_chain_bounds(rmc_ctx* ctx, const struct rmc_chain* chain, int full_space_sites,
                                  int max_merges, rmc_merge_diag* diag, int* n_merges, double* E_out);

/* ---- autotuned tile shapes --------------------------------------------- */

/* The solver's block products (Gram matrices X1 X2^T over the product-basis
 * vectors and basis combinations op(W) X, in FP32, FP64 or double-FP32) each
 * have a short list of launch configurations (SIMT tiles of 64 x 64, 48 x 48
 * or 32 x 32; for Gram matrices also the split-K factor).  A process-wide
 * table maps a product's shape bin to its configuration; bins without an entry
 * use the first (untuned) one.  rmc_autotune solves `chain` once with tuning
 * on: every product whose bin is new times each candidate on its own operands
 * (CUDA events on the context's stream; merges run one at a time) and records
 * the fastest.  Candidates differ only in summation order, so results change
 * at rounding level, well inside the solver's tolerances.  Call it while no
 * other solve runs in the process (tuning is process-wide while it runs).
 * E_out[q] receives the solve's energies (may be NULL).  Synchronises. */
rmc_status rmc_autotune(rmc_ctx* ctx, const struct rmc_chain* chain, double* E_out);

/* The table as text, one "key=choice" line per shape bin, into buf (at most
 * len bytes including the terminating NUL; buf may be NULL).  Returns the
 * bytes the whole text needs, NUL included.  Needs no GPU. */
size_t rmc_tune_dump(char* buf, size_t len);

/* Merge "key=choice" lines (as written by rmc_tune_dump) into the table.
 * Returns the number of entries read, or -1 on a malformed line (entries
 * before it are kept).  Needs no GPU. */
int rmc_tune_load(const char* text);

/* Empty the table (every product then uses its untuned configuration). */
void rmc_tune_clear(void);

typedef struct rmc_server rmc_server;

/* A solve server: `slots` solves run at once, each on its own host worker
 * thread, CUDA stream and memory pool, so their kernels overlap on the device.
 * Independent solves are whole units of Algorithm 1 (its merges within a
 * level and separate parameter points never exchange data).  Requests are
 * admitted in arrival order as soon as a slot is free AND their estimated
 * device memory fits in cfg->mem_budget (shared by all slots; 0 = 40 GiB);
 * requests that arrive while others run join as those finish (continuous
 * batching).  cfg->stream is ignored.  Results stay on the device between the
 * levels of a solve; only energies come back.
 * Slots only overlap on the device if the driver gives their streams separate
 * hardware queues: CUDA_DEVICE_MAX_CONNECTIONS (read when the CUDA context is
 * created; 8 unless set) should be at least the number of slots.  Loading the
 * library sets it to 32 when it is unset; a context created earlier keeps 8
 * (measured on one B300 with 16 slots: 40 solves/s with 8 queues, 73 with 32). */
rmc_status rmc_server_create(const rmc_config* cfg, int slots, rmc_server** out);
/* Stop accepting work, finish what was admitted or queued, join the workers. */
rmc_status rmc_server_destroy(rmc_server* srv);
/* Queue one solve; *id receives its ticket.  RMC_ERR_NOMEM at once if the
 * request alone can never fit the budget; RMC_ERR_INVAL for a malformed chain. */
rmc_status rmc_submit(rmc_server* srv, const rmc_chain* chain, uint64_t* id);
/* Result of a ticket.  wait != 0 blocks until it is done.  *done = 1 when the
 * result is ready: then E_out[q] (may be NULL) gets the energies,
 * *solve_status the solve's rmc_status, *latency_ms the time from submission
 * to completion and *queue_ms the time from submission to admission (each
 * pointer may be NULL), and the ticket is released.  *done = 0: still queued
 * or running.  RMC_ERR_INVAL for an unknown ticket. */
rmc_status rmc_poll(rmc_server* srv, uint64_t id, int wait, int* done, double* E_out, int* solve_status,
                    double* latency_ms, double* queue_ms);
/* Text of the most recent failed solve on this server ("" if none). */
const char* rmc_server_last_error(rmc_server* srv);
/* Counters: submitted, completed, running, queued, bytes reserved by admitted
 * solves, kernel launches issued by all slots. */
rmc_status rmc_server_stats(rmc_server* srv, uint64_t* submitted, uint64_t* completed, int* running,
                            int* queued, size_t* reserved_bytes, uint64_t* launches);
/* rmc_profile / rmc_profile_read over every slot of a server (summed).  The
 * times are per-stream event intervals, so under concurrency they include the
 * time a launch waited for SMs that other slots held. */
rmc_status rmc_server_profile(rmc_server* srv, int enable);
rmc_status rmc_server_profile_read(rmc_server* srv, int kind, uint64_t* groups, uint64_t* launches, double* ms,
                                   double* flops);
/* Estimated peak device memory of one solve (what admission reserves). */
size_t rmc_estimate_bytes(const rmc_chain* chain, int precision);
/* Solve n chains with `slots` concurrent slots and wait: E_out is n x q_max
 * row-major (entries past a chain's q are NaN), status_out[n] the per-solve
 * status.  Returns the first non-OK solve status, else RMC_OK. */
rmc_status rmc_solve_chains(const rmc_config* cfg, int slots, int n, const rmc_chain* chains, int q_max,
                            double* E_out, int* status_out);

/* ---- blocks -------------------------------------------------------------- */

rmc_status rmc_block_free(rmc_ctx* ctx, rmc_block* blk);
/* Kept count k, number of carried operators, basis rows (D for a leaf,
 * k_A k_B for a merged block), and the tag of each operator (tags may be NULL,
 * else n_ops entries). */
rmc_status rmc_block_info(const rmc_block* blk, int* k, int* n_ops, int* basis_rows,
                          rmc_op_tag* tags);
/* Copy a block to host arrays: E[k], ops (n_ops x k x k), basis (rows x k,
 * row-major).  Any pointer may be NULL to skip that part. Synchronises. */
rmc_status rmc_block_export(rmc_ctx* ctx, const rmc_block* blk, double* E,
                            double* ops, double* basis);
/* A block from host data (energies ascending, operators k x k each); the
 * basis is optional (rows = 0 to omit).  Used for checkpoints and for
 * per-merge checks against the oracle. */
rmc_status rmc_block_import(rmc_ctx* ctx, int k, const double* E, int n_ops,
                            const double* ops, const rmc_op_tag* tags, int rows,
                            const double* basis, rmc_block** out);

/* ---- kernel-level entry points (device pointers, one step each) ----------- */

/* The Kronecker-form product with the effective Hamiltonian of Eq. (7) for a
 * block of nv vectors:
 *   Y[v] = alpha * (D o X[v] + sum_j coef_j A_j X[v] B_j^T) + beta * X[v] + gamma * Z[v]
 * with D[a][b] = EA[a] + EB[b].  X, Y, Z: nv x kA x kB (Z may be NULL when
 * gamma == 0; Y must not alias X or Z); A: n_ops x kA x kA; B: n_ops x kB x kB;
 * EA[kA], EB[kB], coef[n_ops]: all device pointers of `dtype` (0 = FP64,
 * 1 = FP32 on the FP32 pipe, 2 = FP32 data on the tcgen05 tensor cores in the
 * 3xTF32 form, which needs n_ops >= 1 and, for each of the two stages, either
 * 16-byte row pitches (kB % 4 == 0 for the first, n_ops * kA % 4 == 0 for the
 * second: the TMA-fed kernel, any size) or at most 256 output columns
 * (n_ops * kB, resp. kA: the plain-load kernel), else RMC_ERR_INVAL; coef,
 * alpha, beta, gamma are always double on the host side and coef is a host
 * array).  The intermediate products are held in scratch
 * memory the library allocates from the context (RMC_ERR_NOMEM if the budget
 * is exceeded).  Runs on the context stream; does not synchronise. */
rmc_status rmc_kron_matvec(rmc_ctx* ctx, int dtype, int kA, int kB, int n_ops, int nv,
                           const void* EA, const void* EB, const void* A, const void* B,
                           const double* coef, const void* X, void* Y, const void* Z,
                           double alpha, double beta, double gamma);

/* Gram product of two vector blocks (the orthogonalisation and Rayleigh-Ritz
 * contractions of the subspace iteration):
 *   G[i][j] = <X1[i], X2[j]>  (G: nv1 x nv2, row-major; X1: nv1 x n, X2: nv2 x n,
 *                              vector-major, all device FP32),
 * symmetrised ((G + G^T) / 2) when symmetrize != 0 and nv1 == nv2.  dtype 1:
 * the FP32 pipe (split-K SIMT GEMM); dtype 2: the tcgen05 tensor cores in the
 * 3xTF32 form, split-K over the TMA-fed kernel (needs n % 4 == 0 and 16-byte
 * aligned blocks, else RMC_ERR_INVAL).  Partial products of the splits go to
 * library scratch (RMC_ERR_NOMEM beyond the budget) and are summed in a fixed
 * order.  Runs on the context stream; does not synchronise. */
rmc_status rmc_gram(rmc_ctx* ctx, int dtype, int nv1, int nv2, long n, const float* X1, const float* X2,
                    float* G, int symmetrize);

/* The Chebyshev filter of one subspace iteration (Zhou and Saad's scaled
 * three-term recurrence on the H_eff of Eq. (7), the operator arguments as in
 * rmc_kron_matvec with dtype 0 = FP64, 1 = FP32, or 3 = FP64 data with the
 * products in double-FP32 arithmetic on the FP32 pipe (single-launch form
 * only; ~1e-13 relative, the form the mixed paths refine with)):
 *   Y[v] = p(H) X[v] / ||p(H) X[v]||,   p = T_deg((H - c) / e) / T_deg((theta0 - c) / e),
 * e = (ub - a) / 2, c = (ub + a) / 2: the polynomial damps [a, ub] (bounded by
 * 1 / |T_deg((theta0 - c) / e)| there) and grows below a; theta0 < a < ub
 * (else RMC_ERR_INVAL), 1 <= deg <= 64.  With deg = 0 it is the plain product
 * Y = H X (not normalised; theta0, a, ub unused).  fused = 1 runs the
 * single-launch form that holds the vectors in shared memory for the whole
 * polynomial (RMC_ERR_INVAL when one k_A x k_B vector with its intermediates
 * does not fit); fused = 0 runs the multi-launch form (two GEMM launches per
 * degree).  Y may alias X.  Device pointers; runs on the context stream; does
 * not synchronise. */
rmc_status rmc_cheb_filter(rmc_ctx* ctx, int dtype, int kA, int kB, int n_ops, int nv,
                           const void* EA, const void* EB, const void* A, const void* B,
                           const double* coef, const void* X, int deg, double theta0, double a,
                           double ub, int fused, void* Y);

/* Allocation-free variant of rmc_kron_matvec, for callers that cannot call
 * cudaMalloc: a plug-in running inside a host application that reserved the
 * device memory for its own allocator, or a latency-critical loop that must
 * not allocate because cudaMalloc and cudaFree can synchronise the device and
 * stall every stream.  The paper has no counterpart; this is a service of the
 * library, not a step of the method.
 *
 * Same arguments and result as rmc_kron_matvec, but no context: it runs on the
 * CURRENT device, on `stream` (a cudaStream_t of that device; NULL = the legacy
 * default stream), and never allocates.  Its scratch (the scaled operator
 * concatenation and the stage-one products) lives in one fixed device array of
 * RMC_NOALLOC_SCRATCH_BYTES (16 MiB) inside the library, which every GPU that
 * loads the library holds until the process exits.  The bytes needed are
 *   sizeof(T) * n_ops * kA * kA, rounded up to 256, plus sizeof(T) * n_ops * kA * kB * nv
 * (T = double for dtype 0, float for dtype 1); a larger request returns
 * RMC_ERR_NOMEM and launches nothing.  Bad arguments return RMC_ERR_INVAL, a
 * failed CUDA call RMC_ERR_CUDA (there is no context to hold error text).
 *
 * The first call on a device looks up that device's address of the array
 * (cudaGetSymbolAddress, with the device current) and caches it; make that
 * first call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents; every scratch element a call reads is first
 * written by that same call, so nothing has to be cleared.  Calls whose work
 * overlaps on the GPU (different streams, or different host threads) race on
 * the array: order them on one stream or synchronise between them.  Does not
 * synchronise. */
#define RMC_NOALLOC_SCRATCH_BYTES (16u << 20)
rmc_status rmc_kron_matvec_noalloc(void* stream, int dtype, int kA, int kB, int n_ops, int nv,
                                   const void* EA, const void* EB, const void* A, const void* B,
                                   const double* coef, const void* X, void* Y, const void* Z,
                                   double alpha, double beta, double gamma);

/* Lowest eigenpairs of a symmetric m x m FP64 matrix (device pointers): all m
 * eigenvalues ascending into w[m], eigenvectors as columns of the row-major
 * m x m matrix V.  FP32 parallel Jacobi followed by FP64 refinement of the
 * eigenvector matrix (Ogita-Aishima).  1 <= m <= 160. */
rmc_status rmc_syev(rmc_ctx* ctx, int m, const double* S, double* w, double* V);

/* Rotation of one carried operator into the merged basis (Algorithm 1, the
 * operator transform after each merge): out = C^T (o (x) I_kB) C
 * (side 0) or C^T (I_kA (x) o) C (side 1).  C: kr vectors of kA x kB (device,
 * FP64, vector-major), o: k x k (k = kA or kB), out: kr x kr. */
rmc_status rmc_rotate_op(rmc_ctx* ctx, int side, int kA, int kB, int kr,
                         const double* C, const double* o, double* out);

#ifdef __cplusplus
}
#endif

#endif /* RMC_H_ */
