// K7: request loop with continuous batching.
//
// Range queries are admitted by cuboid_server_submit while a slot and memory are free
// (admission control), queued on the host, and a dispatcher thread packs whatever is
// pending into a batch as soon as one of several streams is free.  Each batch is one
// persistent sieve launch (the batched path: device work queue, CUDA graph) on its own
// stream, so batches admitted while others run overlap on the device.  Tables and the
// per-stream result buffers stay resident; finished batches are split back into one
// result per query, polled by ticket.  A query whose survivor or root records did not all
// fit in its batch's buffers (its counts are exact, so the number of its survivors is
// known) is run again alone instead of failing; the other queries of the batch keep their
// results.  Every wait in the loop is bounded.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cuboid_internal.cuh"

struct cuboid_result;
namespace cuboid {
int result_create(const cuboid_tables* t, uint32_t max_ranges, uint64_t surv_cap, uint64_t root_cap,
                  cuboid_result** out);
int sieve_into(cuboid_result* r, const cuboid_range* ranges, uint32_t n, uint32_t mode, cudaStream_t s,
               bool device_ranges, bool download);
int result_wait(cuboid_result* r);
int result_snapshot(cuboid_result* r, std::vector<unsigned long long>& counts,
                    std::vector<unsigned long long>& npairs, unsigned long long& n_surv,
                    unsigned long long& n_roots);
cuboid_result* result_host_only(const cuboid_tables* t, uint64_t npairs, const uint64_t* counts,
                                const uint64_t* surv, uint64_t n_surv, const cuboid_root* roots,
                                uint64_t n_roots, int status);
bool result_event_done(cuboid_result* r);
}  // namespace cuboid

using namespace cuboid;

namespace {

constexpr uint32_t kStreams = 4;
constexpr uint64_t kSlotSurvCap = 1ull << 16;
constexpr uint64_t kSlotRootCap = 1ull << 12;
constexpr uint64_t kFreeMemMargin = 64ull << 20;

using Clock = std::chrono::steady_clock;

struct Query {
  uint64_t ticket;
  cuboid_range range;
  Clock::time_point t_submit;
  bool alone = false;  // run in a batch of its own (a retry after a record overflow)
};

struct Finished {
  uint64_t npairs = 0;
  std::vector<uint64_t> counts;
  std::vector<uint64_t> surv;
  std::vector<cuboid_root> roots;
  int status = CUBOID_OK;
  Clock::time_point t_submit, t_done;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cuboid_result* res = nullptr;
  std::vector<Query> queries;
  bool busy = false;
};

}  // namespace

struct cuboid_server {
  cuboid_tables* t = nullptr;
  int device = 0;
  uint64_t budget = 0;
  uint32_t max_slots = 0;
  uint32_t batch_cap = 0;
  uint64_t per_query_bytes = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Query> pending;
  std::unordered_map<uint64_t, Finished> finished;
  std::vector<Slot> slots;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  uint64_t in_flight = 0, admitted = 0, refused = 0, n_finished = 0, batches = 0, retried = 0;
  uint64_t free_mem = ~0ull;
};

static void collect(cuboid_server* s, Slot& sl) {
  const int st = result_wait(sl.res);
  const uint32_t np = s->t->n;
  const size_t nq = sl.queries.size();
  std::vector<Finished> out(nq);
  std::vector<char> again(nq, 0);
  uint64_t roots_kept = 0;
  for (size_t k = 0; k < nq; ++k) {
    Finished& f = out[k];
    f.counts.resize(np);
    uint64_t ns = 0, nr = 0;
    const uint64_t* sv = nullptr;
    const cuboid_root* rv = nullptr;
    cuboid_result_get(sl.res, (uint32_t)k, &f.npairs, f.counts.data(), &ns, &sv, &nr, &rv);
    f.surv.assign(sv, sv + ns);
    f.roots.assign(rv, rv + nr);
    f.status = st;
    f.t_submit = sl.queries[k].t_submit;
    roots_kept += nr;
  }
  if (st == CUBOID_EOVERFLOW) {
    // Counts are exact, so a query's survivors number its pairs minus its counts: a query
    // that got all of them (and, if root records were dropped, has no survivor) is
    // complete; any other runs again alone (or, alone already, keeps EOVERFLOW).
    std::vector<unsigned long long> c, npr;
    unsigned long long ns_all = 0, nr_all = 0;
    result_snapshot(sl.res, c, npr, ns_all, nr_all);
    const bool roots_dropped = nr_all > roots_kept;
    for (size_t k = 0; k < nq; ++k) {
      Finished& f = out[k];
      uint64_t rejected = 0;
      for (uint64_t x : f.counts) rejected += x;
      const uint64_t want = f.npairs - rejected;
      const bool complete = f.surv.size() == want && !(roots_dropped && want > 0);
      if (complete) f.status = CUBOID_OK;
      else if (nq > 1) again[k] = 1;
    }
  }
  const auto now = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  size_t n_again = 0;
  for (size_t k = nq; k-- > 0;) {  // retries go to the front, in their order
    if (!again[k]) continue;
    Query q = sl.queries[k];
    q.alone = true;
    s->pending.push_front(q);
    ++n_again;
  }
  for (size_t k = 0; k < nq; ++k) {
    if (again[k]) continue;
    out[k].t_done = now;
    s->finished[sl.queries[k].ticket] = std::move(out[k]);
  }
  s->retried += n_again;
  s->in_flight -= nq - n_again;
  s->n_finished += nq - n_again;
  sl.queries.clear();
  sl.busy = false;
}

static void dispatcher(cuboid_server* s) {
  cudaSetDevice(s->device);
  std::vector<cuboid_range> batch;
  auto last_mem = std::chrono::steady_clock::now();
  for (;;) {
    bool progressed = false;
    for (Slot& sl : s->slots) {
      if (sl.busy && result_event_done(sl.res)) {
        collect(s, sl);
        progressed = true;
      }
    }
    const auto now = std::chrono::steady_clock::now();
    if (now - last_mem > std::chrono::milliseconds(50)) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->free_mem = fr;
      }
      last_mem = now;
    }
    for (Slot& sl : s->slots) {
      if (sl.busy) continue;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->pending.empty()) break;
        while (!s->pending.empty() && sl.queries.size() < s->batch_cap) {
          // a retried query runs in a batch of its own
          if (s->pending.front().alone && !sl.queries.empty()) break;
          sl.queries.push_back(s->pending.front());
          s->pending.pop_front();
          if (sl.queries.back().alone) break;
        }
      }
      batch.clear();
      for (const Query& q : sl.queries) batch.push_back(q.range);
      // a lone query takes the single-range path (no plan kernel, no graph)
      const uint32_t mode = batch.size() == 1 ? CUBOID_MODE_PLAIN : CUBOID_MODE_BATCHED;
      const int st = sieve_into(sl.res, batch.data(), (uint32_t)batch.size(), mode, sl.stream,
                                false, true);
      if (st != CUBOID_OK) {  // report the failure on every query of the batch
        std::lock_guard<std::mutex> lk(s->mu);
        for (const Query& q : sl.queries) {
          Finished f;
          f.counts.assign(s->t->n, 0);
          f.status = st;
          f.t_submit = q.t_submit;
          f.t_done = Clock::now();
          s->finished[q.ticket] = std::move(f);
        }
        s->in_flight -= sl.queries.size();
        s->n_finished += sl.queries.size();
        sl.queries.clear();
        continue;
      }
      sl.busy = true;
      progressed = true;
      std::lock_guard<std::mutex> lk(s->mu);
      s->batches++;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    bool any_busy = false;
    for (Slot& sl : s->slots) any_busy |= sl.busy;
    if (s->stop && !any_busy && s->pending.empty()) break;
    if (!progressed) {
      if (any_busy)
        s->cv.wait_for(lk, std::chrono::microseconds(20));
      else
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

extern "C" int cuboid_server_create(cuboid_tables* t, uint64_t mem_budget, uint32_t max_slots,
                                    cuboid_server** out) {
  if (!t) return CUBOID_ENOTABLES;
  if (!out) return CUBOID_EINVAL;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != t->device) return CUBOID_EINVAL;
  cuboid_server* s = new (std::nothrow) cuboid_server();
  if (!s) return CUBOID_ENOMEM;
  s->t = t;
  s->device = dev;
  s->budget = mem_budget ? mem_budget : (1ull << 30);
  s->max_slots = max_slots ? max_slots : 4096;
  s->batch_cap = std::max<uint32_t>(1, (s->max_slots + kStreams - 1) / kStreams);
  // bytes one slot of a batch holds on the device (ranges, plan, counts, pair total)
  const uint64_t per_range = sizeof(cuboid_range) + sizeof(TilePlan) + 8ull * t->n + 8;
  const uint64_t per_batch_fixed = sizeof(DevHeader) + kSlotSurvCap * 12 + kSlotRootCap * 28;
  const uint64_t total = kStreams * (per_batch_fixed + per_range * s->batch_cap);
  size_t fr = 0, tot = 0;
  cudaMemGetInfo(&fr, &tot);
  if (total > s->budget || total + kFreeMemMargin > fr) {
    delete s;
    return CUBOID_ENOMEM;
  }
  s->per_query_bytes = per_range + per_batch_fixed / s->batch_cap;
  s->free_mem = fr;
  s->slots.resize(kStreams);
  for (Slot& sl : s->slots) {
    int st = CUBOID_OK;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) st = CUBOID_ECUDA;
    if (st == CUBOID_OK) st = result_create(t, s->batch_cap, kSlotSurvCap, kSlotRootCap, &sl.res);
    if (st != CUBOID_OK) {
      for (Slot& x : s->slots) {
        if (x.res) cuboid_result_free(x.res);
        if (x.stream) cudaStreamDestroy(x.stream);
      }
      delete s;
      return st;
    }
  }
  t->users++;
  s->worker = std::thread(dispatcher, s);
  *out = s;
  return CUBOID_OK;
}

extern "C" int cuboid_server_submit(cuboid_server* s, const cuboid_range* range, uint64_t* ticket) {
  if (!s || !range || !ticket) return CUBOID_EINVAL;
  const cuboid_range& R = *range;
  if (R.p_lo == 0 || R.q_lo == 0 || R.p_lo > R.p_hi || R.q_lo > R.q_hi) return CUBOID_ERANGE;
  if (R.reserved || (R.flags & ~0xFu) || ((R.flags & CUBOID_ROWS_P) && (R.flags & CUBOID_ROWS_Q)))
    return CUBOID_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return CUBOID_EINVAL;
  // admission: a free slot, the server's memory budget, and free device memory
  if (s->in_flight >= s->max_slots || (s->in_flight + 1) * s->per_query_bytes > s->budget ||
      s->free_mem < kFreeMemMargin) {
    s->refused++;
    return CUBOID_EBUSY;
  }
  const uint64_t tk = s->next_ticket++;
  s->pending.push_back(Query{tk, R, Clock::now(), false});
  s->in_flight++;
  s->admitted++;
  *ticket = tk;
  s->cv.notify_one();
  return CUBOID_OK;
}

extern "C" int cuboid_server_poll(cuboid_server* s, uint64_t ticket, cuboid_result** out) {
  if (!s || !out) return CUBOID_EINVAL;
  Finished f;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->finished.find(ticket);
    if (it == s->finished.end()) {
      if (ticket == 0 || ticket >= s->next_ticket) return CUBOID_EINVAL;
      bool queued = false;
      for (const Query& q : s->pending) queued |= q.ticket == ticket;
      for (const Slot& sl : s->slots)
        for (const Query& q : sl.queries) queued |= q.ticket == ticket;
      return queued ? CUBOID_EAGAIN : CUBOID_EINVAL;
    }
    f = std::move(it->second);
    s->finished.erase(it);
  }
  cuboid_result* r = result_host_only(s->t, f.npairs, f.counts.data(), f.surv.data(), f.surv.size(),
                                      f.roots.data(), f.roots.size(), f.status);
  if (!r) return CUBOID_ENOMEM;
  *out = r;
  return CUBOID_OK;
}

extern "C" int cuboid_server_stats(const cuboid_server* s, uint64_t* in_flight, uint64_t* admitted,
                                   uint64_t* refused, uint64_t* finished, uint64_t* batches,
                                   uint64_t* retried) {
  if (!s) return CUBOID_EINVAL;
  cuboid_server* m = const_cast<cuboid_server*>(s);
  std::lock_guard<std::mutex> lk(m->mu);
  if (in_flight) *in_flight = s->in_flight;
  if (admitted) *admitted = s->admitted;
  if (refused) *refused = s->refused;
  if (finished) *finished = s->n_finished;
  if (batches) *batches = s->batches;
  if (retried) *retried = s->retried;
  return CUBOID_OK;
}

extern "C" int cuboid_server_replay(cuboid_server* s, const cuboid_range* queries, const double* arrival_s,
                                    uint32_t n, uint32_t timeout_ms, uint64_t* tickets, double* latency_s,
                                    uint64_t* npairs, int32_t* status, double* wall_s, uint64_t* refused) {
  if (!s || (n && (!queries || !arrival_s || !tickets || !latency_s || !npairs || !status)) || !wall_s ||
      !refused)
    return CUBOID_EINVAL;
  for (uint32_t i = 1; i < n; ++i)
    if (!(arrival_s[i] >= arrival_s[i - 1])) return CUBOID_EINVAL;
  const auto t0 = Clock::now();
  const auto limit = t0 + std::chrono::milliseconds(timeout_ms);
  auto since = [&](Clock::time_point t) { return std::chrono::duration<double>(t - t0).count(); };
  uint64_t busy = 0;
  uint32_t i = 0;
  while (i < n) {
    const double now = since(Clock::now());
    bool refused_now = false;
    while (i < n && arrival_s[i] <= now) {
      const int st = cuboid_server_submit(s, &queries[i], &tickets[i]);
      if (st == CUBOID_EBUSY) {  // admission refused: the query waits, the clock runs on
        ++busy;
        refused_now = true;
        break;
      }
      if (st != CUBOID_OK) return st;
      ++i;
    }
    if (Clock::now() > limit) return CUBOID_ETIMEOUT;
    if (i >= n) break;
    const double gap = refused_now ? 20e-6 : arrival_s[i] - since(Clock::now());
    if (gap > 200e-6)
      std::this_thread::sleep_for(std::chrono::duration<double>(gap - 100e-6));
    else if (gap > 0)
      std::this_thread::yield();
  }
  // every query finished (its result stays for cuboid_server_poll)
  for (;;) {
    uint32_t done = 0;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (uint32_t k = 0; k < n; ++k) done += s->finished.count(tickets[k]) ? 1u : 0u;
      if (done == n) {
        double last = 0.0;
        for (uint32_t k = 0; k < n; ++k) {
          const Finished& f = s->finished[tickets[k]];
          latency_s[k] = std::chrono::duration<double>(f.t_done - f.t_submit).count();
          npairs[k] = f.npairs;
          status[k] = f.status;
          last = std::max(last, since(f.t_done));
        }
        *wall_s = last;
        *refused = busy;
        return CUBOID_OK;
      }
    }
    if (Clock::now() > limit) return CUBOID_ETIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" int cuboid_server_destroy(cuboid_server* s, uint32_t timeout_ms) {
  if (!s) return CUBOID_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->in_flight == 0) break;
    }
    if (std::chrono::steady_clock::now() - t0 > std::chrono::milliseconds(timeout_ms)) return CUBOID_ETIMEOUT;
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  s->worker.join();
  for (Slot& sl : s->slots) {
    if (sl.res) cuboid_result_free(sl.res);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  s->t->users--;
  delete s;
  return CUBOID_OK;
}
