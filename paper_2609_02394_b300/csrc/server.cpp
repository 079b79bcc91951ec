// Solve server: continuous batching of independent chain solves over worker
// slots (host threads), each with its own context, CUDA stream and memory
// pool, so that the device runs the kernels of several solves at once.  Built
// only on the public C ABI of rmc.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/rmc.h"

namespace {

using Clock = std::chrono::steady_clock;

struct ChainCopy {
  int n_sites = 0, L0 = 0, k = 0, q = 0;
  std::vector<int> os, bi, bj;
  std::vector<char> op, pi, pj;
  std::vector<double> oc, bc;
  ChainCopy() = default;
  explicit ChainCopy(const rmc_chain& c)
      : n_sites(c.n_sites), L0(c.L0), k(c.k), q(c.q),
        os(c.onsite_site, c.onsite_site + c.n_onsite), bi(c.bond_i, c.bond_i + c.n_bonds),
        bj(c.bond_j, c.bond_j + c.n_bonds), op(c.onsite_pauli, c.onsite_pauli + c.n_onsite),
        pi(c.bond_pauli_i, c.bond_pauli_i + c.n_bonds), pj(c.bond_pauli_j, c.bond_pauli_j + c.n_bonds),
        oc(c.onsite_coef, c.onsite_coef + c.n_onsite), bc(c.bond_coef, c.bond_coef + c.n_bonds) {}
};

struct Request {
  uint64_t id = 0;
  ChainCopy chain;
  size_t bytes = 0;
  Clock::time_point t_submit, t_admit, t_done;
  bool done = false;
  rmc_status status = RMC_OK;
  std::vector<double> E;
};

bool chain_ok(const rmc_chain* c) {
  if (!c || c->n_sites < 1 || c->L0 < 1 || c->k < 1 || c->q < 1 || c->n_onsite < 0 || c->n_bonds < 0) return false;
  if (c->n_onsite && (!c->onsite_site || !c->onsite_pauli || !c->onsite_coef)) return false;
  if (c->n_bonds && (!c->bond_i || !c->bond_j || !c->bond_pauli_i || !c->bond_pauli_j || !c->bond_coef)) return false;
  return true;
}

// Upper bound of a solve's peak device memory: every block of the recursion
// kept to the end (the chain solver caches them) plus the largest merge's
// workspace, with a margin for pool granularity and per-iteration temporaries.
size_t estimate(const ChainCopy& c, int precision) {
  struct Rec {
    static void walk(int lo, int hi, int L0, int k, int q, bool top, int n_ops, int* kout, double* blocks,
                     double* peak, int precision) {
      const int n = hi - lo;
      if (n <= L0) {
        const int D = 1 << n;
        const int kk = top ? D : std::min(k, D);
        *blocks += 8.0 * (kk + (double)n_ops * kk * kk + (double)D * kk);
        *kout = kk;
        return;
      }
      const int mid = lo + n / 2;
      int ka, kb;
      walk(lo, mid, L0, k, q, false, n_ops, &ka, blocks, peak, precision);
      walk(mid, hi, L0, k, q, false, n_ops, &kb, blocks, peak, precision);
      const double dim = (double)ka * kb;
      const int kr = (int)std::min<double>(top ? q : k, dim);
      const int g = std::max(16, kr / 2);
      double b = std::min<double>(dim, kr + g);
      const bool chunked = b > 160.0 && kr + 1 + 16 > 160 && dim > 160.0;
      if (chunked) b = std::min<double>(dim, kr + 32);
      else b = std::min(b, 160.0);
      const double bw = std::min(b, 160.0);  // working block of the subspace iteration
      const double no = std::max(1, n_ops);
      double ws = 8.0 * b * dim * (4.0 + no) + 8.0 * 3.0 * std::min(b, 128.0) * dim + 8.0 * dim +
                  64.0 * 8.0 * b * b * 6.0;
      if (precision != RMC_PREC_FP64) ws += 4.0 * (2.0 * b + bw * (4.0 + no)) * dim;
      else ws += 8.0 * bw * (4.0 + no) * dim;
      *peak = std::max(*peak, ws);
      *blocks += 8.0 * (kr + (double)n_ops * kr * kr + dim * kr);
      *kout = kr;
    }
  };
  // carried operators per block: at most (Pauli letters used by two-site
  // terms) x (range of the longest term) on each side of the block
  bool used[3] = {false, false, false};
  int range = 0;
  for (size_t t = 0; t < c.bi.size(); ++t) {
    for (char p : {c.pi[t], c.pj[t]}) {
      if (p == 'X' || p == 'x') used[0] = true;
      if (p == 'Y' || p == 'y') used[1] = true;
      if (p == 'Z' || p == 'z') used[2] = true;
    }
    range = std::max(range, c.bj[t] - c.bi[t]);
  }
  const int n_ops = 2 * (used[0] + used[1] + used[2]) * std::max(1, range);
  int kout = 0;
  double blocks = 0, peak = 0;
  Rec::walk(0, c.n_sites, c.L0, c.k, c.q, true, n_ops, &kout, &blocks, &peak, precision);
  return (size_t)(1.25 * (blocks + peak)) + ((size_t)8 << 20);
}

}  // namespace

struct rmc_server {
  rmc_config cfg{};
  size_t budget = 0;
  size_t reserved = 0;
  uint64_t next_id = 1, submitted = 0, completed = 0;
  int running = 0;
  bool stopping = false;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> table;
  std::vector<std::thread> workers;
  std::vector<rmc_ctx*> ctxs;
  rmc_status init_status = RMC_OK;
  std::string last_error;
};

namespace {

void worker_main(rmc_server* s, int slot) {
  rmc_ctx* ctx = s->ctxs[slot];
  for (;;) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] {
        if (s->queue.empty()) return s->stopping;
        return s->reserved + s->queue.front()->bytes <= s->budget || s->running == 0;
      });
      if (s->queue.empty()) return;  // stopping and drained
      r = s->queue.front();
      s->queue.pop_front();
      s->reserved += r->bytes;
      s->running += 1;
      r->t_admit = Clock::now();
    }
    const ChainCopy& c = r->chain;
    std::vector<double> E(c.q, NAN);
    rmc_status st = rmc_solve_chain(ctx, c.n_sites, c.L0, c.k, c.q, (int)c.os.size(), c.os.data(), c.op.data(),
                                    c.oc.data(), (int)c.bi.size(), c.bi.data(), c.bj.data(), c.pi.data(), c.pj.data(),
                                    c.bc.data(), E.data());
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->E = std::move(E);
      r->status = st;
      if (st != RMC_OK)
        s->last_error = "request " + std::to_string(r->id) + ": " + rmc_last_error(ctx);
      r->t_done = Clock::now();
      r->done = true;
      s->reserved -= r->bytes;
      s->running -= 1;
      s->completed += 1;
    }
    s->cv.notify_all();
  }
}

}  // namespace

extern "C" {

size_t rmc_estimate_bytes(const rmc_chain* chain, int precision) {
  if (!chain_ok(chain)) return 0;
  return estimate(ChainCopy(*chain), precision);
}

rmc_status rmc_server_create(const rmc_config* cfg_in, int slots, rmc_server** out) {
  if (!out || slots < 1 || slots > 256) return RMC_ERR_INVAL;
  *out = nullptr;
  std::unique_ptr<rmc_server> s(new rmc_server);
  if (cfg_in) s->cfg = *cfg_in;
  s->cfg.stream = nullptr;
  s->cfg.lanes = 1;  // the slots already run whole solves concurrently
  s->budget = s->cfg.mem_budget ? s->cfg.mem_budget : ((size_t)40 << 30);
  for (int i = 0; i < slots; ++i) {
    rmc_ctx* c = nullptr;
    rmc_status st = rmc_create(&c, &s->cfg);
    if (st != RMC_OK) {
      for (rmc_ctx* x : s->ctxs) rmc_destroy(x);
      return st;
    }
    s->ctxs.push_back(c);
  }
  for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_main, s.get(), i);
  *out = s.release();
  return RMC_OK;
}

rmc_status rmc_server_destroy(rmc_server* s) {
  if (!s) return RMC_ERR_INVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto& t : s->workers) t.join();
  for (rmc_ctx* c : s->ctxs) rmc_destroy(c);
  delete s;
  return RMC_OK;
}

rmc_status rmc_submit(rmc_server* s, const rmc_chain* chain, uint64_t* id) {
  if (!s || !id || !chain_ok(chain)) return RMC_ERR_INVAL;
  auto r = std::make_shared<Request>();
  r->chain = ChainCopy(*chain);
  r->bytes = estimate(r->chain, s->cfg.precision);
  if (r->bytes > s->budget) return RMC_ERR_NOMEM;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return RMC_ERR_INVAL;
    r->id = s->next_id++;
    s->queue.push_back(r);
    s->table[r->id] = r;
    s->submitted += 1;
    *id = r->id;
  }
  s->cv.notify_all();
  return RMC_OK;
}

rmc_status rmc_poll(rmc_server* s, uint64_t id, int wait, int* done, double* E_out, int* solve_status,
                    double* latency_ms, double* queue_ms) {
  if (!s || !done) return RMC_ERR_INVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(id);
  if (it == s->table.end()) return RMC_ERR_INVAL;
  std::shared_ptr<Request> r = it->second;
  if (wait) s->cv.wait(lk, [&] { return r->done; });
  *done = r->done ? 1 : 0;
  if (!r->done) return RMC_OK;
  if (E_out) std::copy(r->E.begin(), r->E.end(), E_out);
  if (solve_status) *solve_status = r->status;
  using ms = std::chrono::duration<double, std::milli>;
  if (latency_ms) *latency_ms = ms(r->t_done - r->t_submit).count();
  if (queue_ms) *queue_ms = ms(r->t_admit - r->t_submit).count();
  s->table.erase(it);
  return RMC_OK;
}

const char* rmc_server_last_error(rmc_server* s) {
  if (!s) return "null server";
  std::lock_guard<std::mutex> lk(s->mu);
  return s->last_error.c_str();
}

rmc_status rmc_server_stats(rmc_server* s, uint64_t* submitted, uint64_t* completed, int* running, int* queued,
                            size_t* reserved_bytes, uint64_t* launches) {
  if (!s) return RMC_ERR_INVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (submitted) *submitted = s->submitted;
  if (completed) *completed = s->completed;
  if (running) *running = s->running;
  if (queued) *queued = (int)s->queue.size();
  if (reserved_bytes) *reserved_bytes = s->reserved;
  if (launches) {
    uint64_t tot = 0;
    for (rmc_ctx* c : s->ctxs) {
      uint64_t l = 0;
      rmc_stats(c, &l, nullptr);
      tot += l;
    }
    *launches = tot;
  }
  return RMC_OK;
}

rmc_status rmc_server_profile(rmc_server* s, int enable) {
  if (!s) return RMC_ERR_INVAL;
  for (rmc_ctx* c : s->ctxs) rmc_profile(c, enable);
  return RMC_OK;
}

rmc_status rmc_server_profile_read(rmc_server* s, int kind, uint64_t* groups, uint64_t* launches, double* ms,
                                   double* flops) {
  if (!s || kind < 0 || kind >= RMC_PROF_KINDS) return RMC_ERR_INVAL;
  uint64_t g = 0, l = 0;
  double t = 0, f = 0;
  for (rmc_ctx* c : s->ctxs) {
    uint64_t g1 = 0, l1 = 0;
    double t1 = 0, f1 = 0;
    rmc_profile_read(c, kind, &g1, &l1, &t1, &f1);
    g += g1; l += l1; t += t1; f += f1;
  }
  if (groups) *groups = g;
  if (launches) *launches = l;
  if (ms) *ms = t;
  if (flops) *flops = f;
  return RMC_OK;
}

rmc_status rmc_solve_chains(const rmc_config* cfg, int slots, int n, const rmc_chain* chains, int q_max,
                            double* E_out, int* status_out) {
  if (n < 0 || q_max < 1 || (n && (!chains || !E_out))) return RMC_ERR_INVAL;
  for (int i = 0; i < n; ++i)
    if (!chain_ok(&chains[i]) || chains[i].q > q_max) return RMC_ERR_INVAL;
  rmc_server* s = nullptr;
  rmc_status st = rmc_server_create(cfg, std::max(1, std::min(slots, std::max(1, n))), &s);
  if (st != RMC_OK) return st;
  std::vector<uint64_t> ids(n, 0);
  rmc_status first = RMC_OK;
  for (int i = 0; i < n; ++i) {
    rmc_status r = rmc_submit(s, &chains[i], &ids[i]);
    if (r != RMC_OK) {
      if (status_out) status_out[i] = r;
      if (first == RMC_OK) first = r;
      ids[i] = 0;
    }
  }
  for (int i = 0; i < n; ++i) {
    double* row = E_out + (size_t)i * q_max;
    for (int j = 0; j < q_max; ++j) row[j] = NAN;
    if (!ids[i]) continue;
    int done = 0, sst = RMC_OK;
    rmc_poll(s, ids[i], 1, &done, row, &sst, nullptr, nullptr);
    if (status_out) status_out[i] = sst;
    if (sst != RMC_OK && first == RMC_OK) first = (rmc_status)sst;
  }
  rmc_server_destroy(s);
  return first;
}

}  // extern "C"
