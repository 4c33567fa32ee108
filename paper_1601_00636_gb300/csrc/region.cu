// Region search of section 5: the rows p of the region of Theorem 1.2 (Eq. 1.2),
// min(cbrt(p/9), p/59) <= q <= 59 p -- for p >= 152 the segment of Eq. 5.2 -- walked
// upward in batches of 100 rows through the batched sieve (one range per row), with the
// paper's toolkit: start at (p, q), read the current p and the deepest prime needed per
// hundred rows, stop with a report that a later start resumes from.  The scan runs on a
// host thread; the device work is the sieve and root test of the batched path.  Past the
// paper's p_max (59 p beyond 32 bits) a synchronous scan continues through the 64-bit
// ranges, rows of p with q cut into pieces below and above 2^32.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "cuboid_internal.cuh"

struct cuboid_result;
namespace cuboid {
int result_create(const cuboid_tables* t, uint32_t max_ranges, uint64_t surv_cap, uint64_t root_cap,
                  cuboid_result** out);
int sieve_into(cuboid_result* r, const cuboid_range* ranges, uint32_t n, uint32_t mode, cudaStream_t s,
               bool device_ranges, bool download);
int result_wait(cuboid_result* r);
int sieve_wide_into(cuboid_result* r, const cuboid_range_wide* ranges, uint32_t n, cudaStream_t s);
}  // namespace cuboid

using namespace cuboid;

namespace {

constexpr uint32_t kPMax = 72796055u;   // 59 p stays below 2^32 (section 5)
constexpr uint32_t kBatchRows = 100;     // the granularity of the paper's progress probe
constexpr uint32_t kScanRows = 2000;     // rows per batch of the synchronous scan
constexpr uint32_t kFirstSearchP = 152;  // Eq. 5.2 holds from here on (section 5)

// Smallest q >= 1 with q >= min(cbrt(p/9), p/59), in integers: 9 q^3 >= p or 59 q >= p.
uint32_t qmin(uint32_t p) {
  uint64_t q1 = 1;
  while (9 * q1 * q1 * q1 < p) ++q1;
  const uint64_t q2 = ((uint64_t)p + 58) / 59;  // p + 58 may pass 2^32
  uint64_t q = std::min(q1, q2);
  return (uint32_t)std::max<uint64_t>(q, 1);
}

// Totals of a scan, in the caller's prime order.
struct Totals {
  std::vector<uint64_t> counts;
  uint64_t pairs = 0, n_surv = 0, n_roots = 0;
  std::vector<uint64_t> surv;
  std::vector<cuboid_root> roots;
};

// Deepest prime needed: the last effective position with a nonzero count, or all of them
// when a pair survived.
void deepest(const cuboid_tables* t, const std::vector<uint64_t>& counts, uint64_t n_surv, uint32_t* depth,
             uint32_t* r_max) {
  uint32_t d = 0;
  if (n_surv) {
    d = t->n;
  } else {
    for (uint32_t e = 0; e < t->n; ++e)
      if (counts[t->order[e]]) d = e + 1;
  }
  *depth = d;
  *r_max = d ? t->info[d - 1].r : 0;
}

// Enqueue rows [p, p_end] (row p from q0 on) as one batched launch on res (results copied
// back in stream order); *n_ranges receives the number of row ranges.
int scan_submit(cuboid_result* res, uint32_t p, uint32_t q0, uint32_t p_end, cudaStream_t s,
                uint32_t* n_ranges) {
  std::vector<cuboid_range> rg;
  rg.reserve(p_end - p + 1);
  for (uint64_t x = p; x <= p_end; ++x) {
    const uint32_t lo = x == p ? std::max(q0, qmin((uint32_t)x)) : qmin((uint32_t)x);
    const uint32_t hi = (uint32_t)(59ull * x);
    if (lo > hi) continue;
    rg.push_back(cuboid_range{(uint32_t)x, (uint32_t)x, lo, hi, 0u, 0u});
  }
  *n_ranges = (uint32_t)rg.size();
  if (rg.empty()) return CUBOID_OK;
  return sieve_into(res, rg.data(), (uint32_t)rg.size(), CUBOID_MODE_BATCHED, s, false, true);
}

// Wait for a submitted batch and add it into `tot` and `batch_counts` / `batch_surv` (this
// batch alone).  Returns OK, EOVERFLOW (records capped; counts exact) or an error.
int scan_collect(cuboid_result* res, const cuboid_tables* t, uint32_t n_ranges, Totals& tot,
                 std::vector<uint64_t>& batch_counts, uint64_t& batch_surv) {
  batch_counts.assign(t->n, 0);
  batch_surv = 0;
  if (n_ranges == 0) return CUBOID_OK;
  const int st = result_wait(res);
  if (st != CUBOID_OK && st != CUBOID_EOVERFLOW) return st;
  std::vector<uint64_t> c(t->n);
  for (uint32_t k = 0; k < n_ranges; ++k) {
    uint64_t np = 0, ns = 0, nr = 0;
    const uint64_t* sv = nullptr;
    const cuboid_root* rv = nullptr;
    cuboid_result_get(res, k, &np, c.data(), &ns, &sv, &nr, &rv);
    for (uint32_t i = 0; i < t->n; ++i) batch_counts[i] += c[i];
    tot.pairs += np;
    tot.n_surv += ns;
    tot.n_roots += nr;
    batch_surv += ns;
    tot.surv.insert(tot.surv.end(), sv, sv + ns);
    tot.roots.insert(tot.roots.end(), rv, rv + nr);
  }
  for (uint32_t i = 0; i < t->n; ++i) tot.counts[i] += batch_counts[i];
  return st;
}

// Sieve rows [p, p_end] (row p from q0 on) as one batched launch and add the results.
int scan_batch(cuboid_result* res, const cuboid_tables* t, uint32_t p, uint32_t q0, uint32_t p_end,
               cudaStream_t s, Totals& tot, std::vector<uint64_t>& batch_counts, uint64_t& batch_surv) {
  uint32_t nr = 0;
  const int st = scan_submit(res, p, q0, p_end, s, &nr);
  if (st != CUBOID_OK) return st;
  return scan_collect(res, t, nr, tot, batch_counts, batch_surv);
}

int check_start(const cuboid_tables* t, uint32_t p, uint32_t q, bool search) {
  if (!t) return CUBOID_ENOTABLES;
  if (p == 0 || (search && p < kFirstSearchP)) return CUBOID_ERANGE;
  if (search && q == 0) return CUBOID_EQLOW;
  if (p > kPMax) return CUBOID_EPMAX;
  if (q != 0 && q < qmin(p)) return CUBOID_EQLOW;
  if (q > 59ull * p) return CUBOID_EQHIGH;
  return CUBOID_OK;
}

}  // namespace

// Last row of a batch of `rows` rows starting in the hundred that holds p (batches are
// aligned to hundreds of p).
static uint32_t batch_end(uint32_t p, uint32_t p_to, uint32_t rows = kBatchRows) {
  const uint64_t e = (uint64_t)p / kBatchRows * kBatchRows + rows - 1;
  return (uint32_t)std::min<uint64_t>(e, p_to);
}

static void fill_report(const cuboid_tables* t, const Totals& tot, uint32_t next_p, uint32_t next_q,
                        cuboid_search_report* rep) {
  if (!rep) return;
  cuboid_search_report r{};
  r.p = next_p;
  r.q = next_q;
  deepest(t, tot.counts, tot.n_surv, &r.depth, &r.r_max);
  r.pairs = tot.pairs;
  r.n_surv = tot.n_surv;
  r.n_roots = tot.n_roots;
  *rep = r;
}

extern "C" uint32_t cuboid_region_qmin(uint32_t p) { return p ? qmin(p) : 1u; }

extern "C" int cuboid_region_scan(cuboid_tables* t, uint32_t p_from, uint32_t q_from, uint32_t p_to, void* stream,
                                  uint64_t* counts, uint64_t* surv, uint64_t surv_cap, cuboid_root* roots,
                                  uint64_t root_cap, cuboid_search_report* rep) {
  int st = check_start(t, p_from, q_from, false);
  if (st != CUBOID_OK) return st;
  if (p_to < p_from) return CUBOID_ERANGE;
  if (p_to > kPMax) return CUBOID_EPMAX;
  cudaStream_t s = (cudaStream_t)stream;
  // Two result objects: the next batch is sieved while the host adds up the last one.
  cuboid_result* res[2] = {nullptr, nullptr};
  st = result_create(t, kScanRows, 1ull << 16, 1ull << 12, &res[0]);
  if (st == CUBOID_OK) st = result_create(t, kScanRows, 1ull << 16, 1ull << 12, &res[1]);
  if (st != CUBOID_OK) {
    if (res[0]) cuboid_result_free(res[0]);
    return st;
  }
  Totals tot;
  tot.counts.assign(t->n, 0);
  std::vector<uint64_t> bc;
  uint64_t bs = 0;
  bool overflow = false;
  uint32_t n_in[2] = {0, 0};
  uint32_t e = batch_end(p_from, p_to, kScanRows);
  st = scan_submit(res[0], p_from, q_from, e, s, &n_in[0]);
  int cur = 0;
  while (st == CUBOID_OK) {
    const bool more = e < p_to;
    uint32_t e2 = e;
    if (more) {
      e2 = batch_end(e + 1, p_to, kScanRows);
      st = scan_submit(res[cur ^ 1], e + 1, 0, e2, s, &n_in[cur ^ 1]);
    }
    const int sc = scan_collect(res[cur], t, n_in[cur], tot, bc, bs);
    if (sc == CUBOID_EOVERFLOW) {
      overflow = true;
    } else if (sc != CUBOID_OK && st == CUBOID_OK) {
      st = sc;
    }
    if (!more || st != CUBOID_OK) break;
    cur ^= 1;
    e = e2;
  }
  // a batch still in flight after an error is waited for before its buffers go
  for (int k = 0; k < 2; ++k) {
    result_wait(res[k]);
    cuboid_result_free(res[k]);
  }
  if (st != CUBOID_OK) return st;
  if (counts) std::memcpy(counts, tot.counts.data(), t->n * sizeof(uint64_t));
  if (surv) std::memcpy(surv, tot.surv.data(), std::min<uint64_t>(surv_cap, tot.surv.size()) * sizeof(uint64_t));
  if (roots)
    std::memcpy(roots, tot.roots.data(), std::min<uint64_t>(root_cap, tot.roots.size()) * sizeof(cuboid_root));
  const uint32_t np = p_to + 1;
  fill_report(t, tot, np, np <= kPMax ? qmin(np) : 0u, rep);
  if (overflow || tot.surv.size() > surv_cap || tot.roots.size() > root_cap) return CUBOID_EOVERFLOW;
  return CUBOID_OK;
}

// ------------------------------------------------------------------ past p_max (64-bit q)

extern "C" int cuboid_region_scan_wide(cuboid_tables* t, uint64_t p_from, uint64_t q_from, uint64_t p_to,
                                       void* stream, uint64_t* counts, uint64_t* surv, uint64_t surv_cap,
                                       cuboid_root_wide* roots, uint64_t root_cap, cuboid_region_report_wide* rep) {
  constexpr uint64_t k2p32 = 1ull << 32;
  if (!t) return CUBOID_ENOTABLES;
  if (p_from == 0 || p_to < p_from || p_to >= k2p32) return CUBOID_ERANGE;
  if (q_from != 0 && q_from < qmin((uint32_t)p_from)) return CUBOID_EQLOW;
  if (q_from > 59ull * p_from) return CUBOID_EQHIGH;
  cudaStream_t s = (cudaStream_t)stream;
  // pieces of one row: the q below 2^32, then at most 2^32 - 64 q a piece
  const uint64_t top = 59ull * p_to;
  const uint64_t per_row = 1 + (top >= k2p32 ? (top - k2p32) / (k2p32 - 64) + 1 : 0);
  cuboid_result* res = nullptr;
  int st = result_create(t, (uint32_t)(kBatchRows * per_row), 1ull << 16, 1ull << 12, &res);
  if (st != CUBOID_OK) return st;
  Totals tot;
  tot.counts.assign(t->n, 0);
  std::vector<uint64_t> c(t->n), sv;
  std::vector<cuboid_root_wide> rv;
  std::vector<cuboid_range_wide> rg;
  bool overflow = false;
  for (uint64_t p = p_from; p <= p_to && st == CUBOID_OK;) {
    const uint64_t e = std::min<uint64_t>(p_to, p / kBatchRows * kBatchRows + kBatchRows - 1);
    rg.clear();
    for (uint64_t x = p; x <= e; ++x) {
      const uint64_t lo = x == p_from ? std::max<uint64_t>(q_from, qmin((uint32_t)x)) : qmin((uint32_t)x);
      if (lo <= 59ull * x) rg.push_back(cuboid_range_wide{x, x, lo, 59ull * x, CUBOID_ROWS_P, 0u});
    }
    p = e + 1;
    if (rg.empty()) continue;
    st = sieve_wide_into(res, rg.data(), (uint32_t)rg.size(), s);
    if (st != CUBOID_OK) break;
    st = result_wait(res);
    if (st == CUBOID_EOVERFLOW) {
      overflow = true;
      st = CUBOID_OK;
    }
    for (uint32_t k = 0; k < rg.size() && st == CUBOID_OK; ++k) {
      uint64_t np = 0, ns = 0, nr = 0;
      const uint64_t* sp = nullptr;
      const cuboid_root_wide* rp = nullptr;
      st = cuboid_result_get_wide(res, k, &np, c.data(), &ns, &sp, &nr, &rp);
      for (uint32_t i = 0; i < t->n; ++i) tot.counts[i] += c[i];
      tot.pairs += np;
      tot.n_surv += ns;
      tot.n_roots += nr;
      sv.insert(sv.end(), sp, sp + 2 * ns);
      rv.insert(rv.end(), rp, rp + nr);
    }
  }
  result_wait(res);
  cuboid_result_free(res);
  if (st != CUBOID_OK) return st;
  if (counts) std::memcpy(counts, tot.counts.data(), t->n * sizeof(uint64_t));
  if (surv) std::memcpy(surv, sv.data(), std::min<uint64_t>(2 * surv_cap, sv.size()) * sizeof(uint64_t));
  if (roots) std::memcpy(roots, rv.data(), std::min<uint64_t>(root_cap, rv.size()) * sizeof(cuboid_root_wide));
  if (rep) {
    cuboid_region_report_wide r{};
    r.p = p_to + 1;
    r.q = p_to + 1 < k2p32 ? qmin((uint32_t)(p_to + 1)) : 0;
    deepest(t, tot.counts, tot.n_surv, &r.depth, &r.r_max);
    r.pairs = tot.pairs;
    r.n_surv = tot.n_surv;
    r.n_roots = tot.n_roots;
    *rep = r;
  }
  if (overflow || sv.size() > 2 * surv_cap || rv.size() > root_cap) return CUBOID_EOVERFLOW;
  return CUBOID_OK;
}

// ------------------------------------------------------------------ asynchronous search

struct cuboid_search {
  cuboid_tables* t = nullptr;
  std::thread worker;
  std::atomic<bool> stop{false};
  std::atomic<uint32_t> cur_p{0};
  std::atomic<uint32_t> cur_rmax{0};
  std::mutex mu;
  Totals tot;
  uint32_t next_p = 0, next_q = 0;
  int status = CUBOID_OK;
};

namespace {
std::mutex g_search_mu;  // one search per tables object (the paper's single search thread)
}

static void search_loop(cuboid_search* S, uint32_t p, uint32_t q) {
  cudaSetDevice(S->t->device);
  cudaStream_t s = nullptr;
  cuboid_result* res = nullptr;
  int st = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess ? CUBOID_OK : CUBOID_ECUDA;
  if (st == CUBOID_OK) st = result_create(S->t, kBatchRows, 1ull << 16, 1ull << 12, &res);
  std::vector<uint64_t> bc;
  uint64_t bs = 0;
  uint32_t q0 = q;
  while (st == CUBOID_OK && !S->stop.load() && p <= kPMax) {
    const uint32_t e = batch_end(p, kPMax);
    S->cur_p.store(p / kBatchRows * kBatchRows);
    Totals part;
    part.counts.assign(S->t->n, 0);
    st = scan_batch(res, S->t, p, q0, e, s, part, bc, bs);
    if (st == CUBOID_EOVERFLOW) st = CUBOID_OK;  // counts stay exact; records were capped
    if (st != CUBOID_OK) break;
    uint32_t d = 0, rm = 0;
    deepest(S->t, bc, bs, &d, &rm);  // per hundred rows, as the paper's r_max
    S->cur_rmax.store(rm);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (uint32_t i = 0; i < S->t->n; ++i) S->tot.counts[i] += part.counts[i];
      S->tot.pairs += part.pairs;
      S->tot.n_surv += part.n_surv;
      S->tot.n_roots += part.n_roots;
      S->next_p = e + 1;
      S->next_q = e + 1 <= kPMax ? qmin(e + 1) : 0u;
    }
    p = e + 1;
    q0 = 0;
  }
  if (res) cuboid_result_free(res);
  if (s) cudaStreamDestroy(s);
  std::lock_guard<std::mutex> lk(S->mu);
  S->status = st;
}

extern "C" int cuboid_search_start(cuboid_tables* t, uint32_t p, uint32_t q, cuboid_search** out) {
  const int st = check_start(t, p, q, true);
  if (st != CUBOID_OK) return st;
  if (!out) return CUBOID_EINVAL;
  std::lock_guard<std::mutex> lk(g_search_mu);
  if (t->searching) return CUBOID_EBUSY;
  cuboid_search* S = new (std::nothrow) cuboid_search();
  if (!S) return CUBOID_ENOMEM;
  S->t = t;
  S->tot.counts.assign(t->n, 0);
  S->next_p = p;
  S->next_q = q;
  S->cur_p.store(p / kBatchRows * kBatchRows);
  t->searching = true;
  t->users++;
  S->worker = std::thread(search_loop, S, p, q);
  *out = S;
  return CUBOID_OK;
}

extern "C" int cuboid_search_current(const cuboid_search* s, uint32_t* p, uint32_t* r_max) {
  if (!s) return CUBOID_EINVAL;
  if (p) *p = s->cur_p.load();
  if (r_max) *r_max = s->cur_rmax.load();
  return CUBOID_OK;
}

extern "C" int cuboid_search_stop(cuboid_search* s, cuboid_search_report* rep, uint64_t* counts) {
  if (!s) return CUBOID_EINVAL;
  s->stop.store(true);
  s->worker.join();
  int st;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    fill_report(s->t, s->tot, s->next_p, s->next_q, rep);
    if (counts) std::memcpy(counts, s->tot.counts.data(), s->t->n * sizeof(uint64_t));
    st = s->status;
  }
  {
    std::lock_guard<std::mutex> lk(g_search_mu);
    s->t->searching = false;
    s->t->users--;
  }
  delete s;
  return st;
}

extern "C" int cuboid_search_report_write(const cuboid_search_report* rep, const char* path) {
  if (!rep || !path) return CUBOID_EINVAL;
  FILE* f = std::fopen(path, "a");
  if (!f) return CUBOID_EINVAL;
  const std::time_t now = std::time(nullptr);
  std::tm tmv{};
  localtime_r(&now, &tmv);
  std::fprintf(f, "%d-%d-%d %02d:%02d\nStop with p=%u, q=%u, r_max=%u\n", tmv.tm_year + 1900, tmv.tm_mon + 1,
               tmv.tm_mday, tmv.tm_hour, tmv.tm_min, rep->p, rep->q, rep->r_max);
  const int bad = std::fclose(f);
  return bad ? CUBOID_EINVAL : CUBOID_OK;
}
