// Host runtime of libcuboid: result objects, the plain (one range per launch) and batched
// (one persistent launch, CUDA graph) execution paths, the exact-root-test entry point,
// and the integer-issue probe.  The serving loop lives in server.cu.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "cuboid_internal.cuh"

namespace cuboid {

constexpr uint64_t kDefaultSurvCap = 1ull << 20;
constexpr uint64_t kDefaultRootCap = 1ull << 16;
// default shape: the one the autotuner picks most often on this part (two 256-thread CTAs
// per SM with the 128-register build, six hot primes)
constexpr uint32_t kDefaultThreads = 256;
constexpr uint32_t kDefaultCtasPerSm = 2;
constexpr uint32_t kDefaultTilesPerWarp = 3;
constexpr uint32_t kDefaultHot = 6;
constexpr size_t kDefaultTableSmem = 48 * 1024;

}  // namespace cuboid

using namespace cuboid;

struct cuboid_result {
  const cuboid_tables* t = nullptr;
  int device = 0;
  uint32_t max_ranges = 0;
  uint64_t surv_cap = 0, root_cap = 0;
  // device: header, pair totals and counts share one block (one copy brings them back).
  // Two blocks: a plain single-range run on a one-range result works in the block the
  // last run did not use, which that run's root-test kernel cleared, so it needs no plan
  // kernel; other runs reset the current block with the plan kernel.
  unsigned char* d_blocks[2] = {nullptr, nullptr};
  unsigned char* d_block = nullptr;  // the current one
  size_t block_bytes = 0;
  int cur = 0;
  unsigned char* h_block = nullptr;  // its pinned host mirror
  DevHeader* d_hdr = nullptr;
  cuboid_range* d_ranges = nullptr;
  TilePlan* d_plan = nullptr;
  unsigned long long* d_counts = nullptr;
  unsigned long long* d_npairs = nullptr;
  unsigned long long* d_surv = nullptr;
  uint32_t* d_surv_range = nullptr;
  cuboid_root* d_roots = nullptr;
  uint32_t* d_root_range = nullptr;
  // pinned host
  DevHeader* h_hdr = nullptr;
  cuboid_range* h_ranges = nullptr;
  unsigned long long* h_counts = nullptr;
  unsigned long long* h_npairs = nullptr;
  cudaEvent_t done = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph[8] = {};     // [count_steps + 2 * time_sieve + 4 * current block]
  cuboid_tuning graph_tuning[8] = {};  // tuning each graph was captured with
  // last run
  uint32_t n_ranges = 0;
  bool downloaded = false;
  bool fetched = false;
  int wait_status = CUBOID_OK;
  // host results (after wait)
  std::vector<uint64_t> counts;  // [range][caller index]
  std::vector<uint64_t> npairs;
  std::vector<std::vector<uint64_t>> surv;
  std::vector<std::vector<cuboid_root>> roots;
  cuboid_stats stats{};
  std::vector<cudaEvent_t> tev;  // sieve timing events, two per launch
  uint32_t timed_launches = 0;
  float sieve_ms = 0.f;
  bool host_only = false;        // results delivered by the server (no device buffers)
  // 64-bit ranges: the run's ranges are the pieces; piece k belongs to range piece_of[k]
  // and its records are relative to h_base[2 k] (p) and h_base[2 k + 1] (q)
  bool wide = false;
  uint32_t n_wide = 0;
  std::vector<uint32_t> piece_of;
  std::vector<unsigned long long> h_base;
  unsigned long long* d_base = nullptr;
  size_t d_base_cap = 0;
  std::vector<uint64_t> wcounts, wnpairs;
  std::vector<std::vector<uint64_t>> wsurv;  // per range: p0, q0, p1, q1, ...
  std::vector<std::vector<cuboid_root_wide>> wroots;
};

namespace cuboid {

constexpr size_t kHdrBytes = (sizeof(DevHeader) + 63) / 64 * 64;  // header padded to 128 B

// Point the header, pair-total and count pointers at block b.
static void use_block(cuboid_result* r, int b) {
  r->cur = b;
  r->d_block = r->d_blocks[b];
  r->d_hdr = reinterpret_cast<DevHeader*>(r->d_block);
  r->d_npairs = reinterpret_cast<unsigned long long*>(r->d_block + kHdrBytes);
  r->d_counts = r->d_npairs + r->max_ranges;
}

// Result block: the device header (padded to 64 bytes), then max_ranges pair totals, then
// the counts of as many ranges as a run fills.
static size_t result_block_bytes(uint32_t max_ranges, size_t n_counts) {
  return kHdrBytes + (size_t)max_ranges * sizeof(unsigned long long) + n_counts * sizeof(unsigned long long);
}

LaunchShape launch_shape(const cuboid_tables* t, bool count_steps, bool wide) {
  const cuboid_tuning& T = t->tuning;
  LaunchShape L;
  L.threads = T.block_threads ? T.block_threads : kDefaultThreads;
  L.row_lanes = (count_steps || wide || !T.row_lanes) ? 32u : T.row_lanes;
  const uint32_t ctas = T.ctas_per_sm ? T.ctas_per_sm : kDefaultCtasPerSm;
  const int smem_sm = t->smem_per_sm, smem_blk = t->smem_per_block;
  const size_t fixed = sieve_smem_bytes(0, t->n, L.threads, L.row_lanes, wide);
  // (128 bytes left for the kernel's static shared memory: the staging barrier)
  size_t per_cta = std::min<size_t>((size_t)smem_blk - 128, (size_t)smem_sm / ctas - 1024);
  size_t table_budget = per_cta > fixed ? per_cta - fixed : 0;
  if (!T.smem_primes) table_budget = std::min(table_budget, kDefaultTableSmem);
  const uint32_t want = T.smem_primes ? std::min(T.smem_primes, t->n) : t->n;
  uint32_t k = 0;
  uint64_t words = 0;
  while (k < want) {
    const PrimeInfo& pi = t->info[k];
    const uint64_t end = (uint64_t)pi.off + (uint64_t)pi.r * pi.W;
    if (((end * 4 + 15) & ~15ull) > table_budget) break;  // staged in whole 16-byte units
    words = end;
    ++k;
  }
  L.n_smem = k;
  L.smem_words = (uint32_t)words;
  // hot primes: an instantiated count (0, 2, 4, 5, 6, 8), all inside the shared-memory prefix
  uint32_t hot = T.hot_primes ? T.hot_primes : kDefaultHot;
  if (hot > k) hot = k;
  if (hot > kMaxHot) hot = kMaxHot;
  static const uint32_t kInst[] = {6, 5, 4, 2, 0};
  for (uint32_t c : kInst)
    if (c <= hot) {
      L.n_hot = c;
      break;
    }
  L.smem = sieve_smem_bytes(L.smem_words, t->n, L.threads, L.row_lanes, wide);
  L.blocks = (uint32_t)t->sms * ctas;
  const uint32_t tpw = T.tiles_per_warp ? T.tiles_per_warp : kDefaultTilesPerWarp;
  L.target_tiles = L.blocks * (L.threads / 32) * tpw;
  return L;
}

void fill_hot(SieveArgs& a, const cuboid_tables* t, const LaunchShape& L) {
  a.n_hot = L.n_hot;
  a.n_sms = (uint32_t)t->sms;
  a.total_words = t->total_words;
  a.row_lanes = L.row_lanes;
  a.stage_spins = kStageSpins;
  for (uint32_t h = 0; h < kMaxHot; ++h) {
    const PrimeInfo pi = h < L.n_hot ? t->info[h] : PrimeInfo{1u, 0u, 0u, 0u};
    a.hot_r[h] = pi.r;
    a.hot_magic[h] = pi.magic;
    a.hot_off[h] = pi.off;
    a.hot_W[h] = pi.W;
    a.hot_step[h] = (128u * L.row_lanes) % pi.r;  // a lane's stride between pairs of words
    a.hot_step_m[h] = a.hot_step[h] - pi.r;
  }
}

static SieveArgs sieve_args(cuboid_result* r, const LaunchShape& L, uint32_t first, uint32_t count) {
  const cuboid_tables* t = r->t;
  SieveArgs a;
  a.info = t->d_info;
  a.words = t->d_words;
  a.trial = t->d_trial;
  a.mimg = t->d_mimg;
  a.plan = r->d_plan;
  a.hdr = r->d_hdr;
  a.counts = r->d_counts;
  a.npairs = r->d_npairs;
  a.surv = r->d_surv;
  a.surv_range = r->d_surv_range;
  a.surv_cap = r->surv_cap;
  a.n_primes = t->n;
  a.n_smem_primes = L.n_smem;
  a.smem_words = L.smem_words;
  a.n_trial = t->n_trial;
  a.range_first = first;
  a.range_count = count;
  fill_hot(a, t, L);
  return a;
}

static VerifyArgs verify_args(cuboid_result* r, bool clear_other) {
  VerifyArgs v;
  v.surv = r->d_surv;
  v.surv_range = r->d_surv_range;
  v.surv_cap = r->surv_cap;
  v.hdr = r->d_hdr;
  v.roots = r->d_roots;
  v.root_range = r->d_root_range;
  v.root_cap = r->root_cap;
  if (clear_other) {  // what a single-range run uses: header, pair total 0, counts of range 0
    unsigned char* other = r->d_blocks[r->cur ^ 1];
    v.zero_block = reinterpret_cast<unsigned long long*>(other);
    v.zero_words = (uint32_t)((kHdrBytes + 8) / 8);
    v.zero_block2 = reinterpret_cast<unsigned long long*>(other + kHdrBytes) + r->max_ranges;
    v.zero_words2 = r->t->n;
  }
  return v;
}

static uint32_t verify_blocks(const cuboid_tables* t) { return (uint32_t)t->sms * 2; }

// Kernels of one batched run: plan (all ranges, count read on the device), sieve, verify.
static cudaError_t timing_events(cuboid_result* r, uint32_t launches) {
  while (r->tev.size() < 2 * (size_t)launches) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    r->tev.push_back(ev);
  }
  return cudaSuccess;
}

// Captured into a graph: the timing events become event-record nodes (External flag).
// Without them the sieve and the root test are programmatic dependents of the kernel
// before them, so each is scheduled while that kernel finishes.
static cudaError_t enqueue_batched(cuboid_result* r, const LaunchShape& L, bool steps, bool timed,
                                   cudaStream_t s) {
  cudaError_t e = launch_plan(r->d_ranges, 0, 0xFFFFFFFFu, r->d_hdr, r->d_plan, r->d_counts, r->d_npairs,
                              r->t->n, L.target_tiles, s, false, L.row_lanes);
  if (e == cudaSuccess && timed) e = cudaEventRecordWithFlags(r->tev[0], s, cudaEventRecordExternal);
  if (e == cudaSuccess)
    e = launch_sieve(sieve_args(r, L, 0, 0xFFFFFFFFu), steps, L.blocks, L.threads, L.smem, s, !timed);
  if (e == cudaSuccess && timed) e = cudaEventRecordWithFlags(r->tev[1], s, cudaEventRecordExternal);
  if (e == cudaSuccess) e = launch_verify(verify_args(r, false), verify_blocks(r->t), s, !timed);
  return e;
}

// Batched: reset + one graph (plan, persistent sieve, root test).  Plain: per range a
// plan and a sieve launch (the first plan also clears the header), then one root test.
// h_ranges (plain runs from host ranges): each plan launch takes its range by value.
static cudaError_t run_kernels(cuboid_result* r, const cuboid_range* d_ranges, const cuboid_range* h_ranges,
                               uint32_t n, uint32_t mode, cudaStream_t s) {
  const bool steps = mode & CUBOID_MODE_COUNT_STEPS;
  const bool timed = mode & CUBOID_MODE_TIME_SIEVE;
  const bool stage_fail = mode & CUBOID_MODE_STAGE_TIMEOUT;
  const bool batched = (mode & 0xFu) == CUBOID_MODE_BATCHED;
  const LaunchShape L = launch_shape(r->t, steps);
  cudaError_t e = sieve_set_smem_limit(steps, L.smem);
  if (e != cudaSuccess) return e;
  r->timed_launches = 0;
  if (timed) {
    e = timing_events(r, batched ? 1 : n);
    if (e != cudaSuccess) return e;
  }
  if (batched) {
    e = launch_reset(r->d_hdr, n, s);  // zero the header, n_ranges = n
    if (e != cudaSuccess) return e;
    const int gi = (steps ? 1 : 0) + (timed ? 2 : 0) + 4 * r->cur;  // graphs hold the block's address
    cudaGraphExec_t& g = r->graph[gi];
    if (g && std::memcmp(&r->graph_tuning[gi], &r->t->tuning, sizeof(cuboid_tuning)) != 0) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
    if (timed) r->timed_launches = 1;
    if (!g) {
      r->graph_tuning[gi] = r->t->tuning;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return e;
      cudaError_t ek = enqueue_batched(r, L, steps, timed, r->cap_stream);
      e = cudaStreamEndCapture(r->cap_stream, &graph);
      if (ek != cudaSuccess) e = ek;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&g, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        g = nullptr;
        return e;
      }
    }
    return cudaGraphLaunch(g, s);
  }
  if (n == 1) {
    // One range: no plan kernel.  The run works in the block the last run did not use
    // (whose header, first pair total and first counts that run's root test cleared, or
    // which is still clear from the start), every CTA plans the range itself, and this
    // run's root test clears the same parts of the other block for the next such run.
    use_block(r, r->cur ^ 1);
    SieveArgs sa = sieve_args(r, L, 0, 1);
    sa.self_plan = 1;
    sa.target_tiles = L.target_tiles;
    sa.self_range = h_ranges ? nullptr : d_ranges;
    if (h_ranges) sa.self_range_val = h_ranges[0];
    if (stage_fail) sa.stage_spins = 0;
    if (timed) e = cudaEventRecord(r->tev[0], s);
    if (e == cudaSuccess) e = launch_sieve(sa, steps, L.blocks, L.threads, L.smem, s, false);
    if (e == cudaSuccess && timed) e = cudaEventRecord(r->tev[1], s);
    VerifyArgs v = verify_args(r, true);
    v.max_bits = h_ranges ? ranges_max_bits(h_ranges, 1) : 0u;
    if (e == cudaSuccess) e = launch_verify(v, verify_blocks(r->t), s, !timed);
    if (timed) r->timed_launches = 1;
    return e;
  }
  for (uint32_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = launch_plan(d_ranges, i, 1, r->d_hdr, r->d_plan, r->d_counts, r->d_npairs, r->t->n, L.target_tiles, s,
                    i == 0, L.row_lanes, h_ranges ? h_ranges + i : nullptr);
    if (e == cudaSuccess && timed) e = cudaEventRecord(r->tev[2 * i], s);
    SieveArgs sa = sieve_args(r, L, i, 1);
    if (stage_fail) sa.stage_spins = 0;
    if (e == cudaSuccess) e = launch_sieve(sa, steps, L.blocks, L.threads, L.smem, s, !timed);
    if (e == cudaSuccess && timed) e = cudaEventRecord(r->tev[2 * i + 1], s);
  }
  VerifyArgs v = verify_args(r, false);
  v.max_bits = h_ranges ? ranges_max_bits(h_ranges, n) : 0u;
  if (e == cudaSuccess) e = launch_verify(v, verify_blocks(r->t), s, !timed);
  if (timed) r->timed_launches = n;
  return e;
}

static int validate_ranges(const cuboid_range* rg, uint32_t n) {
  for (uint32_t i = 0; i < n; ++i) {
    const cuboid_range& R = rg[i];
    if (R.p_lo == 0 || R.q_lo == 0 || R.p_lo > R.p_hi || R.q_lo > R.q_hi) return CUBOID_ERANGE;
    if (R.reserved != 0 || (R.flags & ~0xFu)) return CUBOID_EINVAL;
    if ((R.flags & CUBOID_ROWS_P) && (R.flags & CUBOID_ROWS_Q)) return CUBOID_EINVAL;
  }
  return CUBOID_OK;
}

static int check_device(const cuboid_result* r) {
  int dev = -1;
  cudaGetDevice(&dev);
  return dev == r->device ? CUBOID_OK : CUBOID_EINVAL;
}

static void result_release(cuboid_result* r) {
  if (!r) return;
  if (!r->host_only) {
    if (r->done) cudaEventSynchronize(r->done);
    for (auto& g : r->graph)
      if (g) cudaGraphExecDestroy(g);
    for (auto ev : r->tev) cudaEventDestroy(ev);
    if (r->cap_stream) cudaStreamDestroy(r->cap_stream);
    if (r->done) cudaEventDestroy(r->done);
    cudaFree(r->d_blocks[0]);
    cudaFree(r->d_ranges);
    cudaFree(r->d_plan);
    cudaFree(r->d_surv);
    cudaFree(r->d_surv_range);
    cudaFree(r->d_roots);
    cudaFree(r->d_root_range);
    cudaFree(r->d_base);
    cudaFreeHost(r->h_block);
    cudaFreeHost(r->h_ranges);
  }
  delete r;
}

int result_create(const cuboid_tables* t, uint32_t max_ranges, uint64_t surv_cap, uint64_t root_cap,
                  cuboid_result** out) {
  if (!t) return CUBOID_ENOTABLES;
  if (!out || max_ranges == 0) return CUBOID_EINVAL;
  cuboid_result* r = new (std::nothrow) cuboid_result();
  if (!r) return CUBOID_ENOMEM;
  r->t = t;
  r->device = t->device;
  r->max_ranges = max_ranges;
  r->surv_cap = surv_cap ? surv_cap : kDefaultSurvCap;
  r->root_cap = root_cap ? root_cap : kDefaultRootCap;
  const size_t nc = (size_t)max_ranges * t->n;
  cudaError_t e = cudaSuccess;
#define AL(call)                                      \
  if (e == cudaSuccess) {                             \
    e = (call);                                       \
  }
  const size_t block = result_block_bytes(max_ranges, nc);
  r->block_bytes = block;
  AL(cudaMalloc(&r->d_blocks[0], 2 * block));
  AL(cudaMallocHost(&r->h_block, block));
  AL(cudaMemset(r->d_blocks[0], 0, 2 * block));
  if (e == cudaSuccess) {
    r->d_blocks[1] = r->d_blocks[0] + block;
    use_block(r, 0);
    r->h_hdr = reinterpret_cast<DevHeader*>(r->h_block);
    r->h_npairs = reinterpret_cast<unsigned long long*>(r->h_block + kHdrBytes);
    r->h_counts = r->h_npairs + max_ranges;
  }
  AL(cudaMalloc(&r->d_ranges, max_ranges * sizeof(cuboid_range)));
  AL(cudaMalloc(&r->d_plan, max_ranges * sizeof(TilePlan)));
  AL(cudaMalloc(&r->d_surv, r->surv_cap * sizeof(unsigned long long)));
  AL(cudaMalloc(&r->d_surv_range, r->surv_cap * sizeof(uint32_t)));
  AL(cudaMalloc(&r->d_roots, r->root_cap * sizeof(cuboid_root)));
  AL(cudaMalloc(&r->d_root_range, r->root_cap * sizeof(uint32_t)));
  AL(cudaMallocHost(&r->h_ranges, max_ranges * sizeof(cuboid_range)));
  AL(cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming));
  AL(cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking));
  AL(cudaMemset(r->d_hdr, 0, sizeof(DevHeader)));
#undef AL
  if (e != cudaSuccess) {
    result_release(r);
    return status_from_cuda(e);
  }
  *out = r;
  return CUBOID_OK;
}

// Bytes of the result block that one run fills: header, pair totals, counts of n ranges.
static size_t used_block_bytes(const cuboid_result* r) {
  return result_block_bytes(r->max_ranges, (size_t)r->n_ranges * r->t->n);
}

static int enqueue_download(cuboid_result* r, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(r->h_block, r->d_block, used_block_bytes(r), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(r->done, s);
  if (e == cudaSuccess) r->downloaded = true;
  return status_from_cuda(e);
}

int sieve_into(cuboid_result* r, const cuboid_range* ranges, uint32_t n, uint32_t mode, cudaStream_t s,
               bool device_ranges, bool download) {
  if (!r) return CUBOID_EINVAL;
  if (!r->t) return CUBOID_ENOTABLES;
  if (r->host_only || !ranges || n == 0 || n > r->max_ranges) return CUBOID_EINVAL;
  if ((mode & ~(0xFu | CUBOID_MODE_COUNT_STEPS | CUBOID_MODE_TIME_SIEVE | CUBOID_MODE_STAGE_TIMEOUT)) ||
      (mode & 0xFu) > CUBOID_MODE_BATCHED)
    return CUBOID_EINVAL;
  if ((mode & CUBOID_MODE_STAGE_TIMEOUT) && (mode & 0xFu) != CUBOID_MODE_PLAIN) return CUBOID_EINVAL;
  if (check_device(r) != CUBOID_OK) return CUBOID_EINVAL;
  cudaError_t e = cudaSuccess;
  const bool batched = (mode & 0xFu) == CUBOID_MODE_BATCHED;
  const cuboid_range* d_ranges = r->d_ranges;
  const cuboid_range* h_ranges = nullptr;
  if (!device_ranges && !batched) {
    const int st = validate_ranges(ranges, n);
    if (st != CUBOID_OK) return st;
    h_ranges = ranges;  // plain launches take each range as a kernel argument: no copy
  } else if (!device_ranges) {
    const int st = validate_ranges(ranges, n);
    if (st != CUBOID_OK) return st;
    cudaEventSynchronize(r->done);  // the pinned staging may still feed an earlier copy
    std::memcpy(r->h_ranges, ranges, n * sizeof(cuboid_range));
    e = cudaMemcpyAsync(r->d_ranges, r->h_ranges, n * sizeof(cuboid_range), cudaMemcpyHostToDevice, s);
  } else if (batched) {
    // the captured graph reads the result's own copy
    e = cudaMemcpyAsync(r->d_ranges, ranges, n * sizeof(cuboid_range), cudaMemcpyDeviceToDevice, s);
  } else {
    d_ranges = ranges;  // plain launches read the caller's device ranges in stream order
  }
  if (e != cudaSuccess) return status_from_cuda(e);
  r->n_ranges = n;
  r->downloaded = false;
  r->fetched = false;
  r->wide = false;
  e = run_kernels(r, d_ranges, h_ranges, n, mode, s);
  if (e != cudaSuccess) return status_from_cuda(e);
  if (download) return enqueue_download(r, s);
  e = cudaEventRecord(r->done, s);
  return status_from_cuda(e);
}

// ---- 64-bit ranges

constexpr uint64_t k2p32 = 1ull << 32;

// The pieces of a 64-bit range (cuboid.h, "64-bit ranges"): 32-bit ranges whose
// coordinates are relative to bases (two per piece: added to p, added to q).
static int wide_pieces(const cuboid_range_wide& R, std::vector<cuboid_range>& pieces,
                       std::vector<unsigned long long>& bases) {
  const uint32_t fl = R.flags;
  if (R.reserved != 0 || (fl & ~0xFu) || ((fl & CUBOID_ROWS_P) && (fl & CUBOID_ROWS_Q))) return CUBOID_EINVAL;
  if (R.p_lo == 0 || R.q_lo == 0 || R.p_lo > R.p_hi || R.q_lo > R.q_hi || R.p_hi >= CUBOID_WIDE_LIMIT ||
      R.q_hi >= CUBOID_WIDE_LIMIT)
    return CUBOID_ERANGE;
  bool rows_q;
  if (fl & CUBOID_ROWS_P) {
    if (R.p_hi >= k2p32) return CUBOID_ERANGE;
    rows_q = false;
  } else if (fl & CUBOID_ROWS_Q) {
    if (R.q_hi >= k2p32) return CUBOID_ERANGE;
    rows_q = true;
  } else if (R.p_hi < k2p32 && R.q_hi < k2p32) {  // a 32-bit range
    pieces.push_back(cuboid_range{(uint32_t)R.p_lo, (uint32_t)R.p_hi, (uint32_t)R.q_lo, (uint32_t)R.q_hi, fl, 0u});
    bases.push_back(0ull);
    bases.push_back(0ull);
    return CUBOID_OK;
  } else if (R.p_hi < k2p32) {
    rows_q = false;
  } else if (R.q_hi < k2p32) {
    rows_q = true;
  } else {
    return CUBOID_ERANGE;  // no coordinate below 2^32 to index the rows
  }
  const uint32_t x_lo = (uint32_t)(rows_q ? R.q_lo : R.p_lo), x_hi = (uint32_t)(rows_q ? R.q_hi : R.p_hi);
  const uint64_t y_lo = rows_q ? R.p_lo : R.q_lo, y_hi = rows_q ? R.p_hi : R.q_hi;
  const uint32_t row_flag = rows_q ? CUBOID_ROWS_Q : CUBOID_ROWS_P;
  auto add = [&](uint64_t lo, uint64_t hi, uint64_t base, uint32_t flags) {
    const uint32_t a = (uint32_t)(lo - base), b = (uint32_t)(hi - base);
    pieces.push_back(rows_q ? cuboid_range{a, b, x_lo, x_hi, flags, 0u} : cuboid_range{x_lo, x_hi, a, b, flags, 0u});
    bases.push_back(rows_q ? base : 0ull);
    bases.push_back(rows_q ? 0ull : base);
  };
  // the values below 2^32: a 32-bit piece with the range's own restrictions
  if (y_lo < k2p32)
    add(y_lo, std::min<uint64_t>(y_hi, k2p32 - 1), 0ull, (fl & (CUBOID_Q_LT_P | CUBOID_ALLOW_DIAGONAL)) | row_flag);
  // above 2^32 every y exceeds every row value: no diagonal pair, and q < p holds on all of
  // a piece (rows of q, y = p) or on none of it (rows of p, y = q)
  if ((fl & CUBOID_Q_LT_P) && !rows_q) return CUBOID_OK;
  for (uint64_t start = std::max<uint64_t>(y_lo, k2p32); start <= y_hi;) {
    const uint64_t base = (start & ~63ull) - 64;  // relative start in [64, 128)
    const uint64_t end = std::min<uint64_t>(y_hi, base + 0xFFFFFFFFull);
    add(start, end, base, row_flag);
    start = end + 1;
  }
  return CUBOID_OK;
}

// Per piece a plan and a sieve launch (the first plan clears the header), then one root
// test whose records are offset by the pieces' bases.
static cudaError_t run_kernels_wide(cuboid_result* r, const std::vector<cuboid_range>& pieces, cudaStream_t s) {
  const LaunchShape L = launch_shape(r->t, false, true);
  cudaError_t e = sieve_set_smem_limit(false, L.smem);
  if (e != cudaSuccess) return e;
  const uint32_t n = (uint32_t)pieces.size();
  if (n == 0) return launch_reset(r->d_hdr, 0, s);
  r->timed_launches = 0;
  for (uint32_t i = 0; i < n && e == cudaSuccess; ++i) {
    e = launch_plan(nullptr, i, 1, r->d_hdr, r->d_plan, r->d_counts, r->d_npairs, r->t->n, L.target_tiles, s,
                    i == 0, L.row_lanes, &pieces[i]);
    SieveArgs sa = sieve_args(r, L, i, 1);
    sa.y_base = r->h_base[2 * (size_t)i] + r->h_base[2 * (size_t)i + 1];  // one of the two is 0
    if (e == cudaSuccess) e = launch_sieve(sa, false, L.blocks, L.threads, L.smem, s, true);
  }
  if (e == cudaSuccess) {
    VerifyArgs v = verify_args(r, false);
    v.base = r->d_base;
    e = launch_verify(v, verify_blocks(r->t), s, true);
  }
  return e;
}

// Per 64-bit range: counts and pair totals summed over its pieces, records made absolute.
static void wide_collect(cuboid_result* r) {
  const uint32_t np = r->t->n;
  r->wcounts.assign((size_t)r->n_wide * np, 0);
  r->wnpairs.assign(r->n_wide, 0);
  r->wsurv.assign(r->n_wide, {});
  r->wroots.assign(r->n_wide, {});
  std::vector<std::vector<std::pair<uint64_t, uint64_t>>> sv(r->n_wide);
  for (uint32_t k = 0; k < r->n_ranges; ++k) {
    const uint32_t u = r->piece_of[k];
    const uint64_t bp = r->h_base[2 * (size_t)k], bq = r->h_base[2 * (size_t)k + 1];
    for (uint32_t i = 0; i < np; ++i) r->wcounts[(size_t)u * np + i] += r->counts[(size_t)k * np + i];
    r->wnpairs[u] += r->npairs[k];
    for (uint64_t rec : r->surv[k]) sv[u].push_back({(rec >> 32) + bp, (uint32_t)rec + bq});
    for (const cuboid_root& x : r->roots[k])
      r->wroots[u].push_back(cuboid_root_wide{x.p + bp, x.q + bq, x.t_lo, x.t_hi});
  }
  for (uint32_t u = 0; u < r->n_wide; ++u) {
    std::sort(sv[u].begin(), sv[u].end());
    r->wsurv[u].reserve(2 * sv[u].size());
    for (const auto& pq : sv[u]) {
      r->wsurv[u].push_back(pq.first);
      r->wsurv[u].push_back(pq.second);
    }
    std::sort(r->wroots[u].begin(), r->wroots[u].end(), [](const cuboid_root_wide& a, const cuboid_root_wide& b) {
      if (a.p != b.p) return a.p < b.p;
      if (a.q != b.q) return a.q < b.q;
      if (a.t_hi != b.t_hi) return a.t_hi < b.t_hi;
      return a.t_lo < b.t_lo;
    });
  }
}

int result_wait(cuboid_result* r) {
  if (!r) return CUBOID_EINVAL;
  if (r->host_only || r->fetched) return r->wait_status;
  if (check_device(r) != CUBOID_OK) return CUBOID_EINVAL;
  cudaError_t e = cudaEventSynchronize(r->done);
  if (e != cudaSuccess) return status_from_cuda(e);
  const cuboid_tables* t = r->t;
  const uint32_t n = r->n_ranges;
  const size_t nc = (size_t)n * t->n;
  if (!r->downloaded) {
    e = cudaMemcpy(r->h_block, r->d_block, used_block_bytes(r), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status_from_cuda(e);
  }
  const DevHeader H = *r->h_hdr;
  r->counts.assign(nc, 0);
  for (uint32_t k = 0; k < n; ++k)
    for (uint32_t eidx = 0; eidx < t->n; ++eidx)
      r->counts[(size_t)k * t->n + t->order[eidx]] = r->h_counts[(size_t)k * t->n + eidx];
  r->npairs.assign(r->h_npairs, r->h_npairs + n);
  r->surv.assign(n, {});
  r->roots.assign(n, {});
  const uint64_t ns = std::min<uint64_t>(H.n_surv, r->surv_cap);
  if (ns) {
    std::vector<unsigned long long> sv(ns);
    std::vector<uint32_t> sr(ns);
    e = cudaMemcpy(sv.data(), r->d_surv, ns * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(sr.data(), r->d_surv_range, ns * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status_from_cuda(e);
    for (uint64_t i = 0; i < ns; ++i)
      if (sr[i] < n) r->surv[sr[i]].push_back(sv[i]);
  }
  const uint64_t nr = std::min<uint64_t>(H.n_roots, r->root_cap);
  if (nr) {
    std::vector<cuboid_root> rv(nr);
    std::vector<uint32_t> rr(nr);
    e = cudaMemcpy(rv.data(), r->d_roots, nr * sizeof(cuboid_root), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(rr.data(), r->d_root_range, nr * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status_from_cuda(e);
    for (uint64_t i = 0; i < nr; ++i)
      if (rr[i] < n) r->roots[rr[i]].push_back(rv[i]);
  }
  for (auto& v : r->surv) std::sort(v.begin(), v.end());
  auto key = [](const cuboid_root& a, const cuboid_root& b) {
    if (a.p != b.p) return a.p < b.p;
    if (a.q != b.q) return a.q < b.q;
    if (a.t_hi != b.t_hi) return a.t_hi < b.t_hi;
    return a.t_lo < b.t_lo;
  };
  for (auto& v : r->roots) std::sort(v.begin(), v.end(), key);
  r->sieve_ms = 0.f;
  for (uint32_t i = 0; i < r->timed_launches; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r->tev[2 * i], r->tev[2 * i + 1]) == cudaSuccess) r->sieve_ms += ms;
  }
  r->stats.words = H.stats[0];
  r->stats.word_steps = H.stats[1];
  r->stats.warp_steps = H.stats[2];
  r->stats.tiles = H.stats[3];
  int st = CUBOID_OK;
  if (H.status & kStatusDebugIndex) st = CUBOID_EINDEX;
  else if (H.status & kStatusStageTimeout) st = CUBOID_ETIMEOUT;
  else if (H.status & kStatusVerifyFail) st = CUBOID_EVERIFY;
  else if (H.status & kStatusBadRange) st = CUBOID_ERANGE;
  else if (H.status & (kStatusSurvOverflow | kStatusRootOverflow)) st = CUBOID_EOVERFLOW;
  if (r->wide) wide_collect(r);
  r->wait_status = st;
  r->fetched = true;
  return st;
}

int result_snapshot(cuboid_result* r, std::vector<unsigned long long>& counts,
                    std::vector<unsigned long long>& npairs, unsigned long long& n_surv,
                    unsigned long long& n_roots) {
  if (!r || !r->fetched) return CUBOID_EINVAL;
  counts.assign(r->counts.begin(), r->counts.end());
  npairs.assign(r->npairs.begin(), r->npairs.end());
  n_surv = r->h_hdr ? r->h_hdr->n_surv : 0;
  n_roots = r->h_hdr ? r->h_hdr->n_roots : 0;
  return CUBOID_OK;
}

bool result_event_done(cuboid_result* r) { return cudaEventQuery(r->done) != cudaErrorNotReady; }

cuboid_result* result_host_only(const cuboid_tables* t, uint64_t npairs, const uint64_t* counts,
                                const uint64_t* surv, uint64_t n_surv, const cuboid_root* roots,
                                uint64_t n_roots, int status) {
  cuboid_result* r = new (std::nothrow) cuboid_result();
  if (!r) return nullptr;
  r->t = t;
  r->device = t->device;
  r->host_only = true;
  r->fetched = true;
  r->n_ranges = 1;
  r->max_ranges = 1;
  r->counts.assign(counts, counts + t->n);
  r->npairs.assign(1, npairs);
  r->surv.assign(1, std::vector<uint64_t>(surv, surv + n_surv));
  r->roots.assign(1, std::vector<cuboid_root>(roots, roots + n_roots));
  r->wait_status = status;
  return r;
}

}  // namespace cuboid

// ------------------------------------------------------------------ C ABI

extern "C" int cuboid_result_create(const cuboid_tables* t, uint32_t max_ranges, uint64_t surv_cap,
                                    uint64_t root_cap, cuboid_result** out) {
  return result_create(t, max_ranges, surv_cap, root_cap, out);
}

extern "C" int cuboid_sieve(const cuboid_tables* t, uint32_t p_lo, uint32_t p_hi, uint32_t q_lo,
                            uint32_t q_hi, uint32_t flags, void* stream, cuboid_result** out) {
  if (!t) return CUBOID_ENOTABLES;
  if (!out) return CUBOID_EINVAL;
  cuboid_range R{p_lo, p_hi, q_lo, q_hi, flags, 0};
  int st = validate_ranges(&R, 1);
  if (st != CUBOID_OK) return st;
  cuboid_result* r = nullptr;
  st = result_create(t, 1, 0, 0, &r);
  if (st != CUBOID_OK) return st;
  st = sieve_into(r, &R, 1, CUBOID_MODE_PLAIN, (cudaStream_t)stream, false, true);
  if (st != CUBOID_OK) {
    result_release(r);
    return st;
  }
  *out = r;
  return CUBOID_OK;
}

extern "C" int cuboid_sieve_batch(const cuboid_tables* t, const cuboid_range* ranges, uint32_t n,
                                  void* stream, cuboid_result** out) {
  if (!t) return CUBOID_ENOTABLES;
  if (!out || !ranges || n == 0) return CUBOID_EINVAL;
  int st = validate_ranges(ranges, n);
  if (st != CUBOID_OK) return st;
  cuboid_result* r = nullptr;
  st = result_create(t, n, 0, 0, &r);
  if (st != CUBOID_OK) return st;
  st = sieve_into(r, ranges, n, CUBOID_MODE_BATCHED, (cudaStream_t)stream, false, true);
  if (st != CUBOID_OK) {
    result_release(r);
    return st;
  }
  *out = r;
  return CUBOID_OK;
}

extern "C" int cuboid_sieve_into(cuboid_result* res, const cuboid_range* ranges, uint32_t n, uint32_t mode,
                                 void* stream) {
  return sieve_into(res, ranges, n, mode, (cudaStream_t)stream, false, true);
}

extern "C" int cuboid_sieve_device(cuboid_result* res, const cuboid_range* ranges_dev, uint32_t n,
                                   uint32_t mode, void* stream) {
  return sieve_into(res, ranges_dev, n, mode, (cudaStream_t)stream, true, false);
}

extern "C" int cuboid_result_download(cuboid_result* res, void* stream) {
  if (!res || res->host_only) return CUBOID_EINVAL;
  return enqueue_download(res, (cudaStream_t)stream);
}

extern "C" int cuboid_result_wait(cuboid_result* res) { return result_wait(res); }

extern "C" int cuboid_result_get(const cuboid_result* res, uint32_t range_idx, uint64_t* n_pairs,
                                 uint64_t* counts, uint64_t* n_surv, const uint64_t** surv,
                                 uint64_t* n_roots, const cuboid_root** roots) {
  if (!res || !res->fetched || res->wide) return CUBOID_EINVAL;
  if (range_idx >= res->n_ranges) return CUBOID_EINVAL;
  const uint32_t np = res->t ? res->t->n : (uint32_t)(res->counts.size() / std::max<uint32_t>(res->n_ranges, 1));
  if (n_pairs) *n_pairs = res->npairs[range_idx];
  if (counts) std::memcpy(counts, res->counts.data() + (size_t)range_idx * np, np * sizeof(uint64_t));
  if (n_surv) *n_surv = res->surv[range_idx].size();
  if (surv) *surv = res->surv[range_idx].data();
  if (n_roots) *n_roots = res->roots[range_idx].size();
  if (roots) *roots = res->roots[range_idx].data();
  return CUBOID_OK;
}

extern "C" int cuboid_wide_pieces(const cuboid_range_wide* r, cuboid_range* pieces, uint64_t* bases, uint32_t cap,
                                  uint32_t* n) {
  if (!r || !n || (cap && (!pieces || !bases))) return CUBOID_EINVAL;
  std::vector<cuboid_range> pc;
  std::vector<unsigned long long> bs;
  const int st = wide_pieces(*r, pc, bs);
  if (st != CUBOID_OK) return st;
  *n = (uint32_t)pc.size();
  if (pc.size() > cap) return CUBOID_EOVERFLOW;
  if (!pc.empty()) {
    std::memcpy(pieces, pc.data(), pc.size() * sizeof(cuboid_range));
    for (size_t i = 0; i < bs.size(); ++i) bases[i] = bs[i];
  }
  return CUBOID_OK;
}

namespace cuboid {

// Sieve n 64-bit ranges on an existing result object (enough ranges for their pieces),
// enqueued on s with the copies back.  ETOOLARGE: more pieces than r holds.
int sieve_wide_into(cuboid_result* r, const cuboid_range_wide* ranges, uint32_t n, cudaStream_t s) {
  if (!r || !r->t || r->host_only || !ranges || n == 0) return CUBOID_EINVAL;
  if (check_device(r) != CUBOID_OK) return CUBOID_EINVAL;
  std::vector<cuboid_range> pieces;
  std::vector<unsigned long long> bases;
  std::vector<uint32_t> owner;
  for (uint32_t i = 0; i < n; ++i) {
    const size_t before = pieces.size();
    const int st = wide_pieces(ranges[i], pieces, bases);
    if (st != CUBOID_OK) return st;
    owner.insert(owner.end(), pieces.size() - before, i);
  }
  if (pieces.size() > r->max_ranges) return CUBOID_ETOOLARGE;
  cudaError_t e = cudaSuccess;
  const size_t nb = std::max<size_t>(bases.size(), 2);
  if (r->d_base_cap < nb) {
    cudaFree(r->d_base);
    r->d_base = nullptr;
    r->d_base_cap = 0;
    e = cudaMalloc(&r->d_base, nb * sizeof(unsigned long long));
    if (e != cudaSuccess) return status_from_cuda(e);
    r->d_base_cap = nb;
  }
  cudaEventSynchronize(r->done);  // h_base may still feed the copy of an earlier run
  r->wide = true;
  r->n_wide = n;
  r->piece_of = owner;
  r->h_base = bases;
  if (!bases.empty())
    e = cudaMemcpyAsync(r->d_base, r->h_base.data(), bases.size() * sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, s);
  r->n_ranges = (uint32_t)pieces.size();
  r->downloaded = false;
  r->fetched = false;
  if (e == cudaSuccess) e = run_kernels_wide(r, pieces, s);
  return e == cudaSuccess ? enqueue_download(r, s) : status_from_cuda(e);
}

}  // namespace cuboid

extern "C" int cuboid_sieve_wide(const cuboid_tables* t, const cuboid_range_wide* ranges, uint32_t n, void* stream,
                                 cuboid_result** out) {
  if (!t) return CUBOID_ENOTABLES;
  if (!out || !ranges || n == 0) return CUBOID_EINVAL;
  uint64_t total = 0;
  for (uint32_t i = 0; i < n; ++i) {
    uint32_t k = 0;
    const int st = cuboid_wide_pieces(&ranges[i], nullptr, nullptr, 0, &k);
    if (st != CUBOID_OK && st != CUBOID_EOVERFLOW) return st;
    total += k;
  }
  if (total >= 0xFFFFFFFFull) return CUBOID_ETOOLARGE;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != t->device) return CUBOID_EINVAL;
  cuboid_result* r = nullptr;
  int st = result_create(t, std::max<uint32_t>((uint32_t)total, 1u), 0, 0, &r);
  if (st != CUBOID_OK) return st;
  st = sieve_wide_into(r, ranges, n, (cudaStream_t)stream);
  if (st != CUBOID_OK) {
    result_release(r);
    return st;
  }
  *out = r;
  return CUBOID_OK;
}

extern "C" int cuboid_result_get_wide(const cuboid_result* res, uint32_t range_idx, uint64_t* n_pairs,
                                      uint64_t* counts, uint64_t* n_surv, const uint64_t** surv, uint64_t* n_roots,
                                      const cuboid_root_wide** roots) {
  if (!res || !res->fetched || !res->wide || range_idx >= res->n_wide) return CUBOID_EINVAL;
  const uint32_t np = res->t->n;
  if (n_pairs) *n_pairs = res->wnpairs[range_idx];
  if (counts) std::memcpy(counts, res->wcounts.data() + (size_t)range_idx * np, np * sizeof(uint64_t));
  if (n_surv) *n_surv = res->wsurv[range_idx].size() / 2;
  if (surv) *surv = res->wsurv[range_idx].data();
  if (n_roots) *n_roots = res->wroots[range_idx].size();
  if (roots) *roots = res->wroots[range_idx].data();
  return CUBOID_OK;
}

extern "C" int cuboid_result_sieve_ms(const cuboid_result* res, float* ms, uint32_t* launches) {
  if (!res || !res->fetched || res->timed_launches == 0) return CUBOID_EINVAL;
  if (ms) *ms = res->sieve_ms;
  if (launches) *launches = res->timed_launches;
  return CUBOID_OK;
}

extern "C" int cuboid_result_stats(const cuboid_result* res, cuboid_stats* out) {
  if (!res || !out || !res->fetched) return CUBOID_EINVAL;
  *out = res->stats;
  return CUBOID_OK;
}

extern "C" int cuboid_result_free(cuboid_result* res) {
  if (!res) return CUBOID_EINVAL;
  result_release(res);
  return CUBOID_OK;
}

// ------------------------------------------------------------------ exact root test on given pairs

namespace cuboid {

// The root test of n records (p << 32 | q) on the device, synchronous on s.  rng (or null):
// each record's range index; base (or null): per range the values added to p and q.  Roots
// come back unsorted with their range indices; fail: a survivor the test could not settle.
static int verify_records(const std::vector<unsigned long long>& rec, const std::vector<uint32_t>* rng,
                          const std::vector<unsigned long long>* base, cudaStream_t s,
                          std::vector<cuboid_root>& out, std::vector<uint32_t>& out_range, bool& fail) {
  const size_t n = rec.size();
  cudaError_t e = verify_init_device();
  if (e != cudaSuccess) return status_from_cuda(e);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t rcap = 5ull * n;  // at most five roots u of the quintic per pair
  DevHeader* d_hdr = nullptr;
  unsigned long long* d_surv = nullptr;
  unsigned long long* d_base = nullptr;
  uint32_t* d_rng = nullptr;
  cuboid_root* d_roots = nullptr;
  uint32_t* d_rr = nullptr;
  e = cudaMalloc(&d_hdr, sizeof(DevHeader));
  if (e == cudaSuccess) e = cudaMalloc(&d_surv, n * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&d_roots, rcap * sizeof(cuboid_root));
  if (e == cudaSuccess) e = cudaMalloc(&d_rr, rcap * sizeof(uint32_t));
  if (e == cudaSuccess && rng) e = cudaMalloc(&d_rng, n * sizeof(uint32_t));
  if (e == cudaSuccess && base) e = cudaMalloc(&d_base, base->size() * sizeof(unsigned long long));
  DevHeader H{};
  H.n_surv = n;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_hdr, &H, sizeof(H), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_surv, rec.data(), n * sizeof(unsigned long long), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && rng)
    e = cudaMemcpyAsync(d_rng, rng->data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && base)
    e = cudaMemcpyAsync(d_base, base->data(), base->size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    VerifyArgs v;
    v.surv = d_surv;
    v.surv_range = d_rng;
    v.surv_cap = n;
    v.hdr = d_hdr;
    v.roots = d_roots;
    v.root_range = d_rr;
    v.root_cap = rcap;
    v.base = d_base;
    unsigned long long m = 0;  // the largest coordinate of any record
    for (uint32_t i = 0; i < n; ++i) {
      const uint32_t k = rng ? (*rng)[i] : 0u;
      const unsigned long long bp = base ? (*base)[2 * (size_t)k] : 0ull, bq = base ? (*base)[2 * (size_t)k + 1] : 0ull;
      m |= ((rec[i] >> 32) + bp) | ((rec[i] & 0xFFFFFFFFull) + bq);
    }
    while (m) {
      ++v.max_bits;
      m >>= 1;
    }
    e = launch_verify(v, (uint32_t)sms * 2, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&H, d_hdr, sizeof(H), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  out.clear();
  out_range.clear();
  if (e == cudaSuccess && H.n_roots) {
    out.resize(std::min<uint64_t>(H.n_roots, rcap));
    out_range.resize(out.size());
    e = cudaMemcpy(out.data(), d_roots, out.size() * sizeof(cuboid_root), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(out_range.data(), d_rr, out.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  }
  cudaFree(d_hdr);
  cudaFree(d_surv);
  cudaFree(d_roots);
  cudaFree(d_rr);
  cudaFree(d_rng);
  cudaFree(d_base);
  if (e != cudaSuccess) return status_from_cuda(e);
  fail = (H.status & kStatusVerifyFail) != 0;
  return CUBOID_OK;
}

}  // namespace cuboid

extern "C" int cuboid_verify_pairs(const uint32_t* p, const uint32_t* q, uint32_t n, void* stream,
                                   cuboid_root* roots_out, uint64_t cap, uint64_t* n_roots) {
  if (!p || !q || !n_roots || (cap && !roots_out)) return CUBOID_EINVAL;
  for (uint32_t i = 0; i < n; ++i)
    if (p[i] == 0 || q[i] == 0) return CUBOID_EINVAL;
  *n_roots = 0;
  if (n == 0) return CUBOID_OK;
  std::vector<unsigned long long> rec(n);
  for (uint32_t i = 0; i < n; ++i) rec[i] = ((unsigned long long)p[i] << 32) | q[i];
  std::vector<cuboid_root> out;
  std::vector<uint32_t> rr;
  bool fail = false;
  const int st = verify_records(rec, nullptr, nullptr, (cudaStream_t)stream, out, rr, fail);
  if (st != CUBOID_OK) return st;
  std::sort(out.begin(), out.end(), [](const cuboid_root& a, const cuboid_root& b) {
    if (a.p != b.p) return a.p < b.p;
    if (a.q != b.q) return a.q < b.q;
    if (a.t_hi != b.t_hi) return a.t_hi < b.t_hi;
    return a.t_lo < b.t_lo;
  });
  *n_roots = out.size();
  if (fail) return CUBOID_EVERIFY;
  if (out.size() > cap) return CUBOID_EOVERFLOW;
  if (!out.empty()) std::memcpy(roots_out, out.data(), out.size() * sizeof(cuboid_root));
  return CUBOID_OK;
}

static bool wide_root_less(const cuboid_root_wide& a, const cuboid_root_wide& b) {
  if (a.p != b.p) return a.p < b.p;
  if (a.q != b.q) return a.q < b.q;
  if (a.t_hi != b.t_hi) return a.t_hi < b.t_hi;
  return a.t_lo < b.t_lo;
}

extern "C" int cuboid_verify_pairs_wide(const uint64_t* p, const uint64_t* q, uint32_t n, void* stream,
                                        cuboid_root_wide* roots_out, uint64_t cap, uint64_t* n_roots) {
  if (!p || !q || !n_roots || (cap && !roots_out)) return CUBOID_EINVAL;
  for (uint32_t i = 0; i < n; ++i) {
    if (p[i] == 0 || q[i] == 0) return CUBOID_EINVAL;
    if (p[i] >= CUBOID_WIDE_LIMIT || q[i] >= CUBOID_WIDE_LIMIT) return CUBOID_ERANGE;
  }
  *n_roots = 0;
  if (n == 0) return CUBOID_OK;
  // each pair is its own "range" whose base is the pair itself (records are zero)
  std::vector<unsigned long long> rec(n, 0ull), base(2 * (size_t)n);
  std::vector<uint32_t> rng(n);
  for (uint32_t i = 0; i < n; ++i) {
    rng[i] = i;
    base[2 * (size_t)i] = p[i];
    base[2 * (size_t)i + 1] = q[i];
  }
  std::vector<cuboid_root> out;
  std::vector<uint32_t> rr;
  bool fail = false;
  const int st = verify_records(rec, &rng, &base, (cudaStream_t)stream, out, rr, fail);
  if (st != CUBOID_OK) return st;
  std::vector<cuboid_root_wide> w(out.size());
  for (size_t i = 0; i < out.size(); ++i)
    w[i] = cuboid_root_wide{out[i].p + p[rr[i]], out[i].q + q[rr[i]], out[i].t_lo, out[i].t_hi};
  std::sort(w.begin(), w.end(), wide_root_less);
  *n_roots = w.size();
  if (fail) return CUBOID_EVERIFY;
  if (w.size() > cap) return CUBOID_EOVERFLOW;
  if (!w.empty()) std::memcpy(roots_out, w.data(), w.size() * sizeof(cuboid_root_wide));
  return CUBOID_OK;
}

// ------------------------------------------------------------------ sharding

namespace {

typedef unsigned __int128 u128;

// Lattice points of the triangle rows x = p_lo..p (p >= p_lo - 1): row x holds the q in
// [q_lo, min(q_hi, x - 1 + diag)].
u128 tri_points(const cuboid_range& R, uint64_t p) {
  const int64_t diag = (R.flags & CUBOID_ALLOW_DIAGONAL) ? 1 : 0;
  const int64_t W = (int64_t)R.q_hi - R.q_lo + 1;
  const int64_t z = (int64_t)R.q_lo - diag;  // row x holds min(W, max(0, x - z)) points
  auto F = [&](int64_t x) -> u128 {           // sum over rows <= x
    if (x <= z) return 0;
    const int64_t k = x - z;
    if (k <= W) return (u128)k * (u128)(k + 1) / 2;
    return (u128)W * (u128)(W + 1) / 2 + (u128)(k - W) * (u128)W;
  };
  return F((int64_t)p) - F((int64_t)R.p_lo - 1);
}

}  // namespace

extern "C" int cuboid_shard_range(const cuboid_range* r, uint32_t k, uint32_t i, cuboid_range* out,
                                  uint64_t* points) {
  if (!r || !out || k == 0 || i >= k) return CUBOID_EINVAL;
  const cuboid_range R = *r;
  if (validate_ranges(&R, 1) != CUBOID_OK) return CUBOID_ERANGE;
  cuboid_range S = R;
  if (R.flags & CUBOID_Q_LT_P) {
    const u128 total = tri_points(R, R.p_hi);
    auto cut = [&](uint32_t j) -> uint64_t {  // first row of shard j
      if (j == 0) return R.p_lo;
      if (j == k) return (uint64_t)R.p_hi + 1;
      const u128 want = total * j / k;
      uint64_t lo = R.p_lo, hi = (uint64_t)R.p_hi + 1;  // smallest p with points(p_lo..p-1) >= want
      while (lo < hi) {
        const uint64_t mid = (lo + hi) / 2;
        if (tri_points(R, mid - 1) >= want) hi = mid; else lo = mid + 1;
      }
      return lo;
    };
    const uint64_t a = cut(i), b = cut(i + 1);
    if (a >= b) {
      S.p_lo = 1;
      S.p_hi = 0;
    } else {
      S.p_lo = (uint32_t)a;
      S.p_hi = (uint32_t)(b - 1);
    }
    if (points) *points = a < b ? (uint64_t)(tri_points(R, b - 1) - tri_points(R, a - 1)) : 0;
  } else {
    const bool along_p = (uint64_t)(R.p_hi - R.p_lo) >= (uint64_t)(R.q_hi - R.q_lo);
    const uint64_t lo = along_p ? R.p_lo : R.q_lo, n = (uint64_t)(along_p ? R.p_hi - R.p_lo : R.q_hi - R.q_lo) + 1;
    const uint64_t a = lo + n * i / k, b = lo + n * (i + 1) / k;  // rows [a, b)
    const uint64_t other = (uint64_t)(along_p ? R.q_hi - R.q_lo : R.p_hi - R.p_lo) + 1;
    uint32_t& slo = along_p ? S.p_lo : S.q_lo;
    uint32_t& shi = along_p ? S.p_hi : S.q_hi;
    if (a >= b) {
      slo = 1;
      shi = 0;
    } else {
      slo = (uint32_t)a;
      shi = (uint32_t)(b - 1);
    }
    if (points) *points = (b - a) * other;
  }
  *out = S;
  return CUBOID_OK;
}

// ------------------------------------------------------------------ measurement helpers

namespace {

// One instruction of each kind per step of 16 independent chains (inline PTX, so the
// compiler emits that instruction and nothing else in the chain): kinds 2-7.
__device__ __forceinline__ uint32_t op_lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t op_shf(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("shf.r.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t op_popc_mad(uint32_t a, uint32_t k) {  // popc, then one mad
  uint32_t d;
  asm volatile("{\n .reg .b32 t;\n popc.b32 t, %1;\n mad.lo.u32 %0, t, %2, %1;\n}" : "=r"(d) : "r"(a), "r"(k));
  return d;
}
__device__ __forceinline__ uint32_t op_mad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ unsigned long long op_madwide(uint32_t a, uint32_t b, unsigned long long c) {
  unsigned long long d;
  asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint32_t op_madhi(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// kind 0: 16 independent chains of add / shift / xor (three 32-bit integer ops each).
// kind 1: the sieve's lookup mix: shared-memory load pair, funnel shift, and, popc, xor.
// kinds 2-7: one instruction per chain step: lop3, funnel shift, popc (+ one mad.lo),
// mad.lo, mad.wide (32 x 32 + 64), mad.hi; kind 8: the add-then-minimum min(a + b, c) of
// __viaddmin_u32 (one instruction on GPUs with the DPX instructions).
__global__ void k_probe(uint32_t kind, uint32_t iters, uint32_t* sink) {
  __shared__ uint32_t tab[1024];
  for (uint32_t i = threadIdx.x; i < 1024; i += blockDim.x) tab[i] = i * 2654435761u;
  __syncthreads();
  uint32_t a[16];
  const uint32_t seed = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = seed * (i + 1);
  if (kind == 0) {
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 16; ++i) a[i] = (a[i] + it) ^ (a[i] >> 1);
    }
  } else if (kind == 1) {
    uint32_t acc = 0;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const uint32_t wi = a[i] & 1022u;
        const uint32_t win = __funnelshift_r(tab[wi], tab[wi + 1], a[i]);
        acc += __popc(win & a[i]);
        a[i] ^= win;
      }
    }
    a[0] += acc;
  } else {
    const uint32_t k1 = seed | 1u, k2 = seed ^ 0x9E3779B9u;
    unsigned long long w[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = a[i];
#define CUBOID_PROBE_LOOP(stmt)            \
  for (uint32_t it = 0; it < iters; ++it) { \
    _Pragma("unroll") for (int i = 0; i < 16; ++i) { stmt; } \
  }
    if (kind == 2) {
      CUBOID_PROBE_LOOP(a[i] = op_lop3(a[i], k1, it))
    } else if (kind == 3) {
      CUBOID_PROBE_LOOP(a[i] = op_shf(a[i], k2, it))
    } else if (kind == 4) {
      CUBOID_PROBE_LOOP(a[i] = op_popc_mad(a[i], k1))
    } else if (kind == 5) {
      CUBOID_PROBE_LOOP(a[i] = op_mad(a[i], k1, k2))
    } else if (kind == 6) {
      CUBOID_PROBE_LOOP(w[i] = op_madwide((uint32_t)w[i], k1, w[i]))
    } else if (kind == 8) {
      CUBOID_PROBE_LOOP(a[i] = __viaddmin_u32(a[i], k1, k2))
    } else {
      CUBOID_PROBE_LOOP(a[i] = op_madhi(a[i], k1, k2))
    }
#undef CUBOID_PROBE_LOOP
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] ^= (uint32_t)w[i] ^ (uint32_t)(w[i] >> 32);
  }
  uint32_t x = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) x ^= a[i];
  sink[seed] = x;
}

}  // namespace

extern "C" int cuboid_probe_int_issue(uint32_t kind, uint32_t blocks, uint32_t threads, uint32_t iters,
                                      uint32_t* sink_dev, void* stream) {
  if (kind > 8 || blocks == 0 || threads == 0 || threads > 1024 || threads % 32 || !sink_dev)
    return CUBOID_EINVAL;
  k_probe<<<blocks, threads, 0, (cudaStream_t)stream>>>(kind, iters, sink_dev);
  return status_from_cuda(cudaGetLastError());
}

extern "C" int cuboid_device_sms(uint32_t* sms) {
  if (!sms) return CUBOID_EINVAL;
  int dev = 0, v = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return status_from_cuda(e);
  *sms = (uint32_t)v;
  return CUBOID_OK;
}

extern "C" const char* cuboid_version(void) { return "libcuboid 0.1 (sm_103a)"; }
