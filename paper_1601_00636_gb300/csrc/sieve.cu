// K2 + K3: the bit sieve of section 2 / the search loop of section 5, on the device.
//
// Work unit ("subtile"): one row value x (p, or q when the rectangle is narrow in q) and
// a chunk of consecutive 64-value words of the other coordinate y; a warp takes 32 / G
// subtiles at a time (G lanes per row).  Each lane sieves two adjacent 64-bit words of y
// values at a time (y0 = 64 w .. 64 w + 127) and carries an "alive" mask of the pairs
// still in play:
//   alive = in-range bits & ~(bits of y sharing a prime factor with x) & ~diagonal,
// then for each prime of the effective order
//   rej   = window(u_r row x mod r, starting at y0 mod r) & alive
//   count[prime] += popc(rej);  alive &= ~rej
// The 128-bit window of a pair of words is four funnel shifts of five 32-bit words of
// the window-row table (see cuboid_internal.cuh).  The first K primes ("hot") are applied
// to every word without an early-exit test, with their moduli in the constant bank and
// their counts kept as per-lane sums; words still alive afterwards go to a per-warp queue
// and are finished 32 at a time with a warp-uniform early exit.  Survivors (alive bits
// after the last prime) are compacted with a warp prefix sum and one atomic per warp.
// Tiles come from a device queue (each warp's first tile fixed, then one atomic per tile),
// so one kernel serves one range per launch and thousands of ranges per launch.
#include <mutex>
#include <type_traits>

#include "cuboid_internal.cuh"

namespace cuboid {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr unsigned long long FULL64 = ~0ull;
constexpr uint32_t kNoRange = 0xFFFFFFFFu;
constexpr uint32_t kFlushTiles = 256;       // per-warp uint32 counters are flushed at least this often
constexpr uint32_t kQueue = 96;             // per-warp queue of words that outlive the hot primes (below 32
                                            // after a drain, plus up to 64 from one pair of words per lane)
constexpr int kFacRegs = 4;                 // odd factors whose per-lane offsets sit in registers
constexpr uint32_t kMobiusIters = 8;        // subtiles whose lanes take this many iterations count their
                                            // pairs by Moebius inversion instead of per-word popcounts

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}

// ------------------------------------------------------------------ sieve kernel

// Coprimality masks come from the mask image built with the tables (see
// cuboid_internal.cuh), staged into shared memory with the table prefix.
constexpr uint32_t kTrialSmem = 256;  // leading trial primes staged in shared memory

struct WarpState {
  uint32_t cur_range;
  uint32_t imax;            // deepest prime index reached since the last flush
  uint32_t tiles_since_flush;
  unsigned long long npairs;
  unsigned long long qbits;  // alive pairs of the words queued after the hot primes (since the last fold)
};

__device__ __forceinline__ void flush_counts(WarpState& ws, uint32_t* wcnt, const SieveArgs& a,
                                             uint32_t lane) {
  __syncwarp();
  if (ws.cur_range != kNoRange) {
    unsigned long long* dst = a.counts + (unsigned long long)ws.cur_range * a.n_primes;
    for (uint32_t i = lane; i <= ws.imax && i < a.n_primes; i += 32) {
      const uint32_t c = wcnt[i];
      if (c) {
        atomicAdd(dst + i, (unsigned long long)c);
        wcnt[i] = 0;
      }
    }
    if (lane == 0 && ws.npairs) atomicAdd(a.npairs + ws.cur_range, ws.npairs);
  }
  ws.npairs = 0;
  ws.imax = 0;
  ws.tiles_since_flush = 0;
  __syncwarp();
}


// Poll an mbarrier phase at most `spins` times (each poll may suspend the thread for a
// short, hardware-chosen time); true once the phase has completed.
__device__ __forceinline__ bool mbar_wait_parity(uint32_t bar, uint32_t parity, uint32_t spins) {
  for (uint32_t it = 0; it < spins; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Integer adds and address arithmetic issued on the FMA pipe: x * one + y with one == 1
// at run time (the compiler cannot fold the multiply, so the add does not take a slot of
// the ALU pipe, which the shifts, logic ops and minima keep busy).
__device__ __forceinline__ uint32_t fma_add(uint32_t x, uint32_t y, uint32_t one) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one), "r"(y));
  return d;
}
__device__ __forceinline__ uint32_t fma_sub(uint32_t x, uint32_t y, uint32_t one) {  // x - y
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(y), "r"(0u - one), "r"(x));
  return d;
}
__device__ __forceinline__ uint32_t fma_mad(uint32_t x, uint32_t k, uint32_t y) {  // x k + y
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(k), "r"(y));
  return d;
}
__device__ __forceinline__ uint32_t mulhi_fma(uint32_t x, uint32_t k) {  // (x k) >> 32
  uint32_t d;
  asm("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(x), "r"(k));
  return d;
}
// Five consecutive 32-bit words of shared memory from byte address ad.  The staged
// tables do not change while the kernel sieves, so the loads are pure (no volatile, no
// memory clobber) and the compiler may move them ahead of the arithmetic that uses them.
__device__ __forceinline__ void lds5(uint32_t ad, uint32_t& w0, uint32_t& w1, uint32_t& w2, uint32_t& w3,
                                     uint32_t& w4) {
  asm("ld.shared.u32 %0, [%5];\n ld.shared.u32 %1, [%5+4];\n ld.shared.u32 %2, [%5+8];\n"
      " ld.shared.u32 %3, [%5+12];\n ld.shared.u32 %4, [%5+16];"
      : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3), "=r"(w4)
      : "r"(ad));
}

// n mod r for any 32-bit n, with magic = floor(2^32 / r): n - floor(n*magic/2^32) r is
// n mod r or n mod r + r, and the unsigned minimum with itself minus r (one add-and-minimum)
// picks the residue.
__device__ __forceinline__ uint32_t mod_min(uint32_t n, uint32_t r, uint32_t magic) {
  const uint32_t e = n - __umulhi(n, magic) * r;
  return __viaddmin_u32(e, 0u - r, e);
}

// Up to 32 queued words {x, y0, alive lo, alive hi} (one per lane) of range `range` go
// through the primes [first, n) with a warp-uniform early exit; then the survivors are
// compacted.  kWide: y0 is relative to the piece's base, whose residues are s_ybr.
template <bool kSteps, bool kWide>
__device__ __forceinline__ void cold_batch(const SieveArgs& a, const PrimeInfo* s_info, const uint32_t* s_tab,
                                           const uint32_t* s_ybr, uint32_t* wcnt, const uint4* q, uint32_t cnt,
                                           uint32_t first, bool rows_q, uint32_t range, uint32_t lane,
                                           WarpState& ws, unsigned long long& st_wsteps,
                                           unsigned long long& st_warpsteps) {
  const uint4 e = lane < cnt ? q[lane] : make_uint4(0u, 0u, 0u, 0u);
  const uint32_t x = e.x, y0 = e.y;
  uint32_t al = e.z, ah = e.w;
  // the pairs these words carry out of the hot primes: the last hot prime's count is the
  // pairs alive before it minus these (see fold)
  ws.qbits += __reduce_add_sync(FULL, __popc(al) + __popc(ah));
  const uint32_t n = a.n_primes;
  uint32_t i = first;
  for (; i < n; ++i) {
    if (!__any_sync(FULL, (al | ah) != 0u)) break;
    const PrimeInfo pi = s_info[i];
    const uint32_t ro = pi.off + mod_min(x, pi.r, pi.magic) * pi.W;
    uint32_t s = mod_min(y0, pi.r, pi.magic);
    if constexpr (kWide) {  // (y_base + y0) mod r
      s += s_ybr[i];
      s = min(s, s - pi.r);
    }
    const uint32_t wi = ro + (s >> 5);
    uint32_t w0 = 0, w1 = 0, w2 = 0;
    // the window stays inside row (x mod r): s < r and its last word before the row's end
    const bool in_row = s < pi.r && (s >> 5) + 2 < pi.W;
    if (i < a.n_smem_primes) {
      if (CUBOID_IDX_OK(in_row && wi + 2 < a.smem_words, a.hdr, 2u)) {
        w0 = s_tab[wi];
        w1 = s_tab[wi + 1];
        w2 = s_tab[wi + 2];
      }
    } else if (CUBOID_IDX_OK(in_row && wi + 2 < a.total_words, a.hdr, 3u)) {
      w0 = __ldg(a.words + wi);
      w1 = __ldg(a.words + wi + 1);
      w2 = __ldg(a.words + wi + 2);
    }
    const uint32_t rl = __funnelshift_r(w0, w1, s) & al, rh = __funnelshift_r(w1, w2, s) & ah;
    const uint32_t c = __reduce_add_sync(FULL, __popc(rl) + __popc(rh));
    if (kSteps) {
      st_wsteps += (al | ah) ? 1 : 0;
      st_warpsteps++;
    }
    if (lane == 0 && c) wcnt[i] += c;
    al ^= rl;
    ah ^= rh;
  }
  const uint32_t reached = i < n ? i : n - 1;
  if (reached > ws.imax) ws.imax = reached;
  if (__any_sync(FULL, (al | ah) != 0u)) {
    const uint32_t kk = __popc(al) + __popc(ah);
    uint32_t incl = kk;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(FULL, incl, d);
      if (lane >= (uint32_t)d) incl += o;
    }
    const uint32_t tot = __shfl_sync(FULL, incl, 31);
    unsigned long long basepos = 0;
    if (lane == 31) basepos = atomicAdd(&a.hdr->n_surv, (unsigned long long)tot);
    basepos = __shfl_sync(FULL, basepos, 31);
    unsigned long long pos = basepos + incl - kk;
    bool over = false;
    unsigned long long alive = ((unsigned long long)ah << 32) | al;
    while (alive) {
      const uint32_t b = (uint32_t)__ffsll((long long)alive) - 1;
      alive &= alive - 1;
      const uint32_t y = y0 + b;
      const unsigned long long p = rows_q ? y : x, qq = rows_q ? x : y;
      if (pos < a.surv_cap) {
        a.surv[pos] = (p << 32) | qq;
        a.surv_range[pos] = range;
      } else {
        over = true;
      }
      ++pos;
    }
    if (over) atomicOr(&a.hdr->status, kStatusSurvOverflow);
  }
}

// Process full batches of 32 queued words (all of them when `all`).
template <bool kSteps, bool kWide>
__device__ __forceinline__ void drain(const SieveArgs& a, const PrimeInfo* s_info, const uint32_t* s_tab,
                                      const uint32_t* s_ybr, uint32_t* wcnt, uint4* q, uint32_t& qn,
                                      uint32_t first, bool rows_q, uint32_t range, uint32_t lane, WarpState& ws,
                                      unsigned long long& st_wsteps, unsigned long long& st_warpsteps, bool all) {
  while (qn >= 32 || (all && qn > 0)) {
    const uint32_t cnt = qn < 32 ? qn : 32;
    cold_batch<kSteps, kWide>(a, s_info, s_tab, s_ybr, wcnt, q, cnt, first, rows_q, range, lane, ws, st_wsteps,
                              st_warpsteps);
    const uint32_t rest = qn - cnt;  // below 64: entries 32 .. 32 + rest move to the front
    uint4 e0 = make_uint4(0u, 0u, 0u, 0u), e1 = e0;
    const bool mv0 = lane < rest && CUBOID_IDX_OK(32 + lane < kQueue, a.hdr, 7u);
    const bool mv1 = lane + 32 < rest && CUBOID_IDX_OK(64 + lane < kQueue, a.hdr, 7u);
    if (mv0) e0 = q[32 + lane];
    if (mv1) e1 = q[64 + lane];
    __syncwarp();
    if (mv0) q[lane] = e0;
    if (mv1) q[32 + lane] = e1;
    __syncwarp();
    qn = rest;
  }
}

// K: number of "hot" primes (the first K of the effective order, all resident in shared
// memory).
// kMaxThreads: 1024 keeps every kernel at <= 64 registers (two 512-thread CTAs per SM);
// 640 allows 96 (20 warps per SM, e.g. two 320-thread CTAs); 512 lets 512 threads per SM
// use up to 128 registers.
// G: lanes per row.  A warp takes one tile = 32 / G consecutive subtiles of a range (a
// subtile is one row and one chunk of its 64-value words); each group of G lanes sieves
// one subtile, each lane a pair of adjacent words at a time, lanes on pairs G apart.  G = 32 is one subtile per warp; smaller groups
// share the per-row setup (factors of the row value, residues of the hot primes) among
// fewer words, which pays on short rows.
// kWide: the launch sieves one piece of a 64-bit range (SieveArgs::y_base): the residues of
// y_base modulo the table primes (per CTA) and modulo the row's factors (per row) are added
// to those of the relative y; whole-warp rows only.
template <bool kSteps, int K, int kMaxThreads, int G, bool kWide = false>
__global__ void __launch_bounds__(kMaxThreads, 1) k_sieve(SieveArgs a) {
  static_assert(!kWide || G == 32, "64-bit pieces use whole-warp rows");
  static_assert(G == 8 || G == 16 || G == 32, "lanes per row");
  constexpr uint32_t NG = 32 / G;                 // subtiles per tile (groups per warp)
  constexpr uint32_t kStride = 128u * G;          // a lane's next pair of words starts 2 G words further on
  extern __shared__ uint4 smem_raw[];
  const uint32_t n = a.n_primes;
  const uint32_t warps = blockDim.x >> 5;
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  const uint32_t g = lane / G, gl = lane % G;     // group and lane in the group
  const uint32_t gshift = g * G;
  const uint32_t gmask = G == 32 ? FULL : ((1u << G) - 1u) << gshift;
  // Dynamic shared memory: the table prefix, the prime records, the leading trial primes
  // and the coprimality mask image (each staged by one bulk copy), then the per-warp
  // working arrays.
  const uint32_t tab_bytes = (a.smem_words * 4u + 15u) & ~15u;  // the table buffer has 16 B of slack
  const uint32_t n_trial_s = a.n_trial < kTrialSmem ? a.n_trial : kTrialSmem;
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem_raw);                                 // [smem_words]
  PrimeInfo* s_info = reinterpret_cast<PrimeInfo*>(smem_raw + tab_bytes / 16);             // [n]
  TrialPrime* s_trial = reinterpret_cast<TrialPrime*>(s_info + n);                         // [kTrialSmem]
  uint4* s_fac_all = reinterpret_cast<uint4*>(s_trial + kTrialSmem);                       // [warps][NG][kMaxFactors]
  uint4* s_queue_all = s_fac_all + warps * NG * kMaxFactors;                               // [warps][kQueue]
  uint4* s_mtab = s_queue_all + warps * kQueue;                                             // [kMaskTab]
  uint32_t* s_foff = reinterpret_cast<uint32_t*>(s_mtab + kMaskTab);                       // [kPeriodicBelow]
  uint32_t* s_fmag_all = s_foff + kPeriodicBelow;                                                       // [warps][NG][kMaxFactors]
  uint32_t* s_cnt_all = s_fmag_all + warps * NG * kMaxFactors;                              // [warps][n]
  uint32_t* s_ybr = s_cnt_all + warps * n;                  // [n] (kWide): y_base mod r
  uint32_t* s_fyb_all = s_ybr + n;                          // [warps][NG][kMaxFactors] (kWide): y_base mod f
  __shared__ __align__(8) unsigned long long s_bar;  // completion of the bulk copies
  __shared__ TilePlan s_self_plan;                    // the single range's plan (self_plan)
  __shared__ unsigned long long s_self_total;

  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&s_bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // TMA bulk copies global -> shared (16-byte aligned, sizes multiples of 16); the
    // tables and prime records were written when the tables were built
    const uint32_t info_bytes = n * (uint32_t)sizeof(PrimeInfo);
    const uint32_t trial_bytes = n_trial_s * (uint32_t)sizeof(TrialPrime);
    const uint32_t mimg_bytes = kMaskImageWords * 4u;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"(tab_bytes + info_bytes + trial_bytes + mimg_bytes)
                 : "memory");
    if (tab_bytes)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(s_tab)),
                   "l"(a.words), "r"(tab_bytes), "r"(bar)
                   : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(s_info)),
                 "l"(a.info), "r"(info_bytes), "r"(bar)
                 : "memory");
    if (trial_bytes)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(s_trial)),
                   "l"(a.trial), "r"(trial_bytes), "r"(bar)
                   : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(s_mtab)),
                 "l"(a.mimg), "r"(mimg_bytes), "r"(bar)
                 : "memory");
  }
  if (a.self_plan && threadIdx.x == 0) {
    const cuboid_range R = a.self_range ? *a.self_range : a.self_range_val;
    TilePlan P;
    unsigned long long words;
    const bool ok = plan_orient(R, P, words);
    const unsigned long long tiles = plan_tiles(P, plan_chunk(words, a.target_tiles, NG), NG);
    P.tile_end = tiles;
    s_self_plan = P;
    s_self_total = tiles;
    if (!ok && blockIdx.x == 0) atomicOr(&a.hdr->status, kStatusBadRange);
  }
  for (uint32_t i = threadIdx.x; i < warps * n; i += blockDim.x) s_cnt_all[i] = 0;
  // bounded wait for the staging: on time-out the CTA records it and leaves once its
  // copies have landed (or a second bounded wait ends)
  const bool staged = mbar_wait_parity(bar, 0u, a.stage_spins);
  if (__syncthreads_or(!staged)) {
    pdl_wait();
    if (threadIdx.x == 0) atomicOr(&a.hdr->status, kStatusStageTimeout);
    mbar_wait_parity(bar, 0u, kStageSpins);
    return;
  }
  if constexpr (kWide) {  // residues of the piece's base, effective order (hot primes first)
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) s_ybr[i] = (uint32_t)(a.y_base % s_info[i].r);
    __syncthreads();
  }
  pdl_wait();     // the plan (header, tile plans, zeroed counts) is complete from here on
  pdl_trigger();  // the root-test grid may be scheduled as CTAs of this grid retire

  uint4* s_fac = s_fac_all + (wid * NG + g) * kMaxFactors;        // this group's factors
  uint32_t* s_fmag = s_fmag_all + (wid * NG + g) * kMaxFactors;
  uint32_t* s_fyb = s_fyb_all + (wid * NG + g) * kMaxFactors;
  uint4* s_queue = s_queue_all + wid * kQueue;
  uint32_t* wcnt = s_cnt_all + wid * n;
  const uint32_t count = a.self_plan ? 1u : (a.range_count == kNoRange ? a.hdr->n_ranges : a.range_count);
  const unsigned long long total = a.self_plan ? s_self_total : a.hdr->total_tiles;

  WarpState ws{kNoRange, 0, 0, 0, 0};
  unsigned long long st_words = 0, st_wsteps = 0, st_warpsteps = 0, st_tiles = 0;
  uint32_t qn = 0;       // queued words (warp-uniform), all of range ws.cur_range
  bool q_rows = false;   // orientation of the queued words

  // Per-lane sums of the pairs still alive: tile_pairs before the hot primes, hs[h] after
  // hot prime h.  Hot prime h rejected the difference of the sums before and after it (a
  // pair leaves the alive set once).  Folded into the warp's counters at each flush: at
  // most kFlushTiles tiles of at most kMaxChunkWords / G + 1 words a lane, 64 pairs a
  // word, so below 2^27.
  uint32_t hs[K > 0 ? K : 1];
#pragma unroll
  for (int h = 0; h < (K > 0 ? K : 1); ++h) hs[h] = 0;
  uint32_t tile_pairs = 0;
  // Call with the queue drained: the pairs alive after the last hot prime are then those
  // counted into ws.qbits, so its per-lane sum is not kept in the word loop.
  auto fold = [&]() {
    uint32_t before = tile_pairs;
#pragma unroll
    for (int h = 0; h + 1 < K; ++h) {
      const uint32_t c = __reduce_add_sync(FULL, before - hs[h]);
      if (lane == 0 && c) wcnt[h] += c;
      before = hs[h];
      hs[h] = 0;
    }
    if constexpr (K > 0) {
      const uint32_t c = (uint32_t)(__reduce_add_sync(FULL, before) - ws.qbits);
      if (lane == 0 && c) wcnt[K - 1] += c;
    }
    ws.qbits = 0;
    ws.npairs += __reduce_add_sync(FULL, tile_pairs);
    tile_pairs = 0;
    __syncwarp();
  };

  // The first tile of every warp is fixed (tile CTA x warps + warp: no atomic on the
  // shared cursor at the start, when every warp would ask at once); the cursor hands out
  // the tiles after those.
  const unsigned long long first_tiles = (unsigned long long)gridDim.x * warps;
  unsigned long long next = (unsigned long long)blockIdx.x * warps + wid;
  TilePlan P1{};  // a single-range launch reads its plan once
  if (a.self_plan) P1 = s_self_plan;
  else if (count == 1) P1 = a.plan[a.range_first];

  for (;;) {
    const unsigned long long tile = next;
    if (tile >= total) break;
    if (lane == 0) next = first_tiles + atomicAdd(&a.hdr->cursor, 1ull);  // prefetch the next tile

    uint32_t k = a.range_first;
    if (count > 1) {  // first range with tile_end > tile
      uint32_t lo = a.range_first, hi = a.range_first + count - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.plan[mid].tile_end > tile) hi = mid; else lo = mid + 1;
      }
      k = lo;
    }
    const TilePlan P = count == 1 ? P1 : a.plan[k];
    const unsigned long long tbeg = (k == a.range_first) ? 0ull : a.plan[k - 1].tile_end;
    if (k != ws.cur_range || ws.tiles_since_flush >= kFlushTiles) {
      drain<kSteps, kWide>(a, s_info, s_tab, s_ybr, wcnt, s_queue, qn, K, q_rows, ws.cur_range, lane, ws,
                           st_wsteps, st_warpsteps, true);
      fold();
      flush_counts(ws, wcnt, a, lane);
      ws.cur_range = k;
    }
    ws.tiles_since_flush++;

    const bool rows_q = P.flags & kRowsQ;
    q_rows = rows_q;
    const bool tri = !kWide && (P.flags & CUBOID_Q_LT_P);  // a 64-bit piece lies above every row value
    const uint32_t diag = (P.flags & CUBOID_ALLOW_DIAGONAL) ? 1u : 0u;
    const uint32_t wbox_lo = P.y_lo >> 6;
    const uint32_t nw = (P.y_hi >> 6) - wbox_lo + 1;
    const uint32_t chunks = (nw + P.chunk_words - 1) / P.chunk_words;
    const unsigned long long n_rows = (unsigned long long)(P.x_hi - P.x_lo) + 1;
    // this group's subtile: row and chunk
    const unsigned long long sub = (tile - tbeg) * NG + g;
    unsigned long long row_idx;
    uint32_t chunk;
    if (chunks == 1) {
      row_idx = sub;
      chunk = 0;
    } else {
      row_idx = sub / chunks;
      chunk = (uint32_t)(sub - row_idx * chunks);
    }
    bool live = row_idx < n_rows;  // the last tile of a range may have idle groups
    // triangles with p rows: longest rows (largest p) first
    const uint32_t x = !live ? 1u
                             : ((tri && !rows_q) ? P.x_hi - (uint32_t)row_idx : P.x_lo + (uint32_t)row_idx);

    // y range of this row
    unsigned long long ylo = P.y_lo, yhi = P.y_hi;
    if (tri) {
      if (!rows_q) {
        const unsigned long long lim = (unsigned long long)x - 1 + diag;  // q < p (q <= p)
        if (lim < yhi) yhi = lim;
      } else {
        const unsigned long long lim = (unsigned long long)x + 1 - diag;  // p > q (p >= q)
        if (lim > ylo) ylo = lim;
      }
    }
    const uint32_t wlo = (uint32_t)(ylo >> 6), whi = (uint32_t)(yhi >> 6);
    const uint32_t c0 = wbox_lo + chunk * P.chunk_words;
    const uint32_t c1 = c0 + P.chunk_words - 1;
    const uint32_t wbeg = c0 > wlo ? c0 : wlo;
    const uint32_t wend = c1 < whi ? c1 : whi;
    if (ylo > yhi || wbeg > wend) live = false;
    if (G == 32) {
      if (!live) {
        next = __shfl_sync(FULL, next, 0);
        continue;
      }
    } else if (!__any_sync(FULL, live)) {
      next = __shfl_sync(FULL, next, 0);
      continue;
    }
    if (kSteps) st_tiles++;
    const unsigned long long lo_mask = FULL64 << (uint32_t)(ylo & 63);
    const unsigned long long hi_mask = FULL64 >> (63 - (uint32_t)(yhi & 63));
    const uint32_t dword = kWide ? 0xFFFFFFFFu : x >> 6;  // past every word: no diagonal in a 64-bit piece
    const uint32_t dbit_lo = (x & 32) ? 0u : 1u << (x & 31), dbit_hi = (x & 32) ? 1u << (x & 31) : 0u;

    // ---- distinct odd prime factors of x (trial division shared by the group's lanes)
    // Each lane tests one trial prime per batch; a lane that divides x writes its factor
    // entry {f - y, -y, mask table base, base + cap} (y = (128 G) mod f) and its reciprocal, and
    // divides its prime power out of the cofactor through a product over the group.
    uint32_t nfo = 0;  // uniform in the group
    bool has2 = false;
    uint32_t big = 1;  // a prime factor above 2^31 left out of the masks (x itself), or 1
    {
      uint32_t m = x;
      if ((m & 1u) == 0) {
        has2 = true;
        m >>= __ffs(m) - 1;
      }
      bool act = live;
      for (uint32_t base = 0;; base += G) {
        if (act) {
          if (base >= a.n_trial) {
            act = false;
          } else {
            const uint32_t f0 = base < n_trial_s ? s_trial[base].f : __ldg(&a.trial[base].f);
            if ((unsigned long long)f0 * f0 > m) act = false;
          }
        }
        if (G == 32) {
          if (!act) break;
        } else if (!__any_sync(FULL, act)) {
          break;
        }
        const uint32_t idx = base + gl;
        const TrialPrime tp = !(act && idx < a.n_trial) ? TrialPrime{1u, 1u, 0u, 0u}
                              : (idx < n_trial_s ? s_trial[idx] : a.trial[idx]);
        const bool hit = act && idx < a.n_trial && m * tp.inv <= tp.lim;
        const uint32_t wbal = __ballot_sync(FULL, hit);
        if (!wbal) continue;
        const uint32_t bal = wbal & gmask;  // this group's hits
        uint32_t pw = 1u;                   // the power of this lane's prime in m
        if (hit) {
          uint32_t mm = m * tp.inv;  // m / f, exact
          pw = tp.f;
          while (mm * tp.inv <= tp.lim) {
            mm *= tp.inv;
            pw *= tp.f;
          }
          const uint32_t pos = nfo + __popc(bal & lanemask_lt);
          const uint32_t f = tp.f;
          if (CUBOID_IDX_OK(pos < kMaxFactors, a.hdr, 5u)) {
            const uint32_t y = mod_min(kStride, f, tp.lim);
            const uint32_t base = f < kPeriodicBelow ? s_foff[f] : kBitTab;
            s_fac[pos] = make_uint4(f - y, 0u - y, base, base + (f < kPeriodicBelow ? f - 1 : 128u));
            s_fmag[pos] = tp.lim;  // floor(2^32 / f) for odd f > 1
            if constexpr (kWide) s_fyb[pos] = (uint32_t)(a.y_base % f);
          }
        }
#pragma unroll
        for (int d = G / 2; d; d >>= 1) pw *= __shfl_xor_sync(FULL, pw, d);  // within the group
        uint32_t inv = pw;  // pw^-1 mod 2^32 (pw odd) by Newton's iteration
#pragma unroll
        for (int it = 0; it < 4; ++it) inv *= 2u - pw * inv;
        m *= inv;  // exact: pw divides m
        nfo += __popc(bal);
      }
      // the cofactor is a prime: above every trial prime tested, or below 9 if no batch ran.
      // A prime factor above 2^31 is x itself, whose only multiple below 2^32 is the
      // diagonal y = x (handled with the range edges), so 32-bit ranges leave it out.
      if (live && m > 1 && (kWide || m <= 0x80000000u)) {
        if (gl == 0 && CUBOID_IDX_OK(nfo < kMaxFactors, a.hdr, 5u)) {
          const uint32_t mag = 0xFFFFFFFFu / m;
          const uint32_t y = mod_min(kStride, m, mag);
          const uint32_t base = m < kPeriodicBelow ? s_foff[m] : kBitTab;
          s_fac[nfo] = make_uint4(m - y, 0u - y, base, base + (m < kPeriodicBelow ? m - 1 : 128u));
          s_fmag[nfo] = mag;
          if constexpr (kWide) s_fyb[nfo] = (uint32_t)(a.y_base % m);
        }
        ++nfo;
      } else if (live && m > 1) {
        big = m;
      }
      // inert entries up to kFacRegs: offset 128 that never moves, empty mask
      if (gl < (uint32_t)kFacRegs && gl >= nfo) s_fac[gl] = make_uint4(1u, 0u, kBitTab, kBitTab + 128u);
      __syncwarp();
    }
    // Each lane sieves pairs of adjacent words (128 values): pair p of the subtile covers
    // words wbeg + 2 p and wbeg + 2 p + 1, and lane gl takes the pairs gl, gl + G, ....
    // Per-lane offset of the first multiple of each odd factor in the lane's first pair.
    const uint32_t y0f = (wbeg + 2 * gl) << 6;
    uint32_t tf[kFacRegs];
#pragma unroll
    for (int i = 0; i < kFacRegs; ++i) {
      tf[i] = 128u;  // inert entry
      if ((uint32_t)i < nfo) {
        const uint32_t f = s_fac[i].x - s_fac[i].y;
        uint32_t r = mod_min(y0f, f, s_fmag[i]);
        if constexpr (kWide) {  // (y_base + y0) mod f; f may exceed 2^31
          const unsigned long long rr = (unsigned long long)r + s_fyb[i];
          r = (uint32_t)(rr >= f ? rr - f : rr);
        }
        tf[i] = r ? f - r : 0u;
      }
    }

    // ---- row offsets of the hot primes (word index, and shared byte address)
    uint32_t rb[K > 0 ? K : 1];
    uint32_t rb4[K > 0 ? K : 1];
    uint32_t sh[K > 0 ? K : 1];  // y0 mod r of the lane's current word, advanced per slot
    const uint32_t tab_addr = (uint32_t)__cvta_generic_to_shared(s_tab);
#pragma unroll
    for (int h = 0; h < K; ++h) {
      rb[h] = a.hot_off[h] + mod_min(x, a.hot_r[h], a.hot_magic[h]) * a.hot_W[h];
      rb4[h] = tab_addr + 4u * rb[h];
      uint32_t s0 = mod_min(y0f, a.hot_r[h], a.hot_magic[h]);
      if constexpr (kWide) {
        s0 += s_ybr[h];
        s0 = min(s0, s0 - a.hot_r[h]);
      }
      sh[h] = s0;
    }

    const uint32_t npairs_sub = live ? (wend - wbeg) / 2 + 1 : 0u;  // pairs of words of the subtile
    const uint32_t nit = (npairs_sub + G - 1) / G;                 // iterations of this lane's group
    const uint32_t maxit = G == 32 ? nit : __reduce_max_sync(FULL, nit);
    const uint32_t one = a.one;  // 1 at run time: x * one + y issues on the FMA pipe
    // Pairs of the subtile when its lanes take many iterations (instead of a popcount per
    // word): Moebius inversion over the prime factors of x,
    //   #{y in [Y0, Y1] : gcd(x, y) = 1} = sum over sets S of them of (-1)^|S| (floor(Y1 / d)
    //   - floor((Y0 - 1) / d)), d the product of S,
    // then the diagonal y = x (coprime only for x = 1; the range flag admits it).  Lane gl
    // of the group takes every G-th set; the warp's sums add up the lanes' parts.
    const bool mob = !kWide && maxit >= kMobiusIters;  // uniform in the warp
    if (mob && live) {
      const uint32_t Y0 = (uint32_t)max((unsigned long long)ylo, (unsigned long long)wbeg << 6);
      const uint32_t Y1 = (uint32_t)min(yhi, ((unsigned long long)wend << 6) + 63);
      const uint32_t np = nfo + (has2 ? 1u : 0u) + (big > 1 ? 1u : 0u);
      uint32_t part = 0;  // modulo 2^32: the warp's total is what counts
      for (uint32_t set = gl; set < (1u << np); set += G) {
        unsigned long long d = 1;
        uint32_t sign = 0;
        for (uint32_t b = 0; b < np && d <= Y1; ++b) {
          if (!((set >> b) & 1u)) continue;
          const uint32_t f = b < nfo ? s_fac[b].x - s_fac[b].y : (b == nfo && has2 ? 2u : big);
          d *= f;
          sign ^= 1u;
        }
        if (d > Y1) continue;
        const uint32_t t = Y1 / (uint32_t)d - (Y0 - 1) / (uint32_t)d;
        part += sign ? 0u - t : t;
      }
      if (gl == 0 && x >= Y0 && x <= Y1) {
        if (x == 1 && !diag) part -= 1;
        if (x > 1 && diag) part += 1;
      }
      tile_pairs += part;
    }
    // x even: y0 is even, so the even y (excluded) sit at the even bits
    const uint32_t even_bits = has2 ? 0x55555555u : 0u;
    // Interior pairs of words (neither word on a range edge, both in the subtile) have
    // their first word in [int_base, int_base + int_span]; the others take the edge path,
    // as do the pairs holding the diagonal word.
    const long long int_hi = (long long)(wend < whi ? wend + 1 : whi) - 2;  // last interior first word
    const long long int_lo = (long long)wlo + 1;
    // no interior: base 2^32 - 1 and span 0 make every pair an edge (word indices < 2^26)
    const bool has_interior = live && int_hi >= int_lo;
    const uint32_t int_span = has_interior ? (uint32_t)(int_hi - int_lo) : 0u;
    const uint32_t int_base = has_interior ? (uint32_t)int_lo : 0xFFFFFFFFu;
    const bool diag_in = dword >= wbeg && dword <= wend;
    // one word's exclusions beyond coprimality: bits outside the range, the diagonal
    // (unless the range admits it: then it is kept whatever the masks say)
    auto edge_word = [&](uint32_t w, bool on, uint32_t& ml, uint32_t& mh) {
      if (!on) {
        ml = mh = FULL;
        return;
      }
      unsigned long long rm = FULL64;
      if (w == wlo) rm &= lo_mask;
      if (w == whi) rm &= hi_mask;
      const uint32_t rml = (uint32_t)rm, rmh = (uint32_t)(rm >> 32);
      ml |= ~rml;
      mh |= ~rmh;
      if (w == dword) {
        ml |= dbit_lo;
        mh |= dbit_hi;
        if (diag) {
          ml &= ~(dbit_lo & rml);
          mh &= ~(dbit_hi & rmh);
        }
      }
    };
    // queue the words of the lanes' pairs still alive (the warp's A words, then its B
    // words, in lane order) and finish full batches of 32 through the rest of the primes
    auto enqueue2 = [&](uint32_t alA, uint32_t ahA, uint32_t alB, uint32_t ahB, uint32_t y0) {
      const bool liveA = (alA | ahA) != 0u, liveB = (alB | ahB) != 0u;
      const uint32_t balA = __ballot_sync(FULL, liveA), balB = __ballot_sync(FULL, liveB);
      if (balA | balB) {
        const uint32_t nA = __popc(balA);
        const uint32_t slotA = qn + __popc(balA & lanemask_lt);
        const uint32_t slotB = qn + nA + __popc(balB & lanemask_lt);
        if (liveA && CUBOID_IDX_OK(slotA < kQueue, a.hdr, 6u)) s_queue[slotA] = make_uint4(x, y0, alA, ahA);
        if (liveB && CUBOID_IDX_OK(slotB < kQueue, a.hdr, 6u)) s_queue[slotB] = make_uint4(x, y0 + 64u, alB, ahB);
        qn += nA + __popc(balB);
        __syncwarp();
        drain<kSteps, kWide>(a, s_info, s_tab, s_ybr, wcnt, s_queue, qn, K, rows_q, k, lane, ws, st_wsteps,
                             st_warpsteps, false);
      }
    };
    // The same window in iterations: this lane's pairs start at words wb0 + 2 G j, the
    // interior ones for j in [j_lo, j_lo + j_span] (none: j_lo = 2^32 - 1, j_span = 0), and
    // the pair holding the diagonal word is iteration j_d (none: 2^32 - 1), so the word
    // loop tests its iteration number instead of the words.
    const uint32_t wb0 = wbeg + 2 * gl;
    uint32_t j_lo = 0xFFFFFFFFu, j_span = 0u;
    if (has_interior && int_base + int_span >= wb0) {
      const uint32_t first = int_base > wb0 ? (int_base - wb0 + 2 * G - 1) / (2 * G) : 0u;
      const uint32_t last = (int_base + int_span - wb0) / (2 * G);
      if (first <= last) {
        j_lo = first;
        j_span = last - first;
      }
    }
    uint32_t j_d = 0xFFFFFFFFu;
    if (diag_in && dword >= wb0 && (dword - wb0) % (2 * G) <= 1u) j_d = (dword - wb0) / (2 * G);
    // The word loop, compiled twice: with the pair totals left to the Moebius count above,
    // or counted per pair of words (a flag tested in every iteration cost 2 %).
    auto word_loop = [&](auto by_mobius) {
    constexpr bool kMob = decltype(by_mobius)::value;
    uint32_t wb = wb0;
    for (uint32_t j = 0; j < maxit; ++j, wb += 2 * G) {
      const uint32_t wA = wb, wB = wb + 1;  // the lane's pair of adjacent words
      // bits to exclude: y sharing a prime factor with x (128-bit masks from the image for
      // both words at once), even y for even x, then the range edges and the diagonal.  A
      // lane whose pair lies past the subtile computes masks the edge path then overwrites.
      uint4 m = make_uint4(even_bits, even_bits, even_bits, even_bits);
      {
#pragma unroll
        for (int i = 0; i < kFacRegs; ++i) {  // inert entries give an empty mask
          // whole-warp rows (nfo is the warp's): the second pair of slots only for rows with
          // three or more odd factors (a test per slot costs more than the inert slot it saves)
          if (G == 32 && i == 2 && nfo <= 2u) break;
          const uint4 fc = s_fac[i];          // {f - y, -y, table base, base + cap}, y = (128 G) mod f
          // base + min(t, cap) as one add-and-minimum, min(t + base, base + cap): in 32-bit
          // ranges t < f <= 2^31, so t + base does not wrap
          const uint32_t mi = kWide ? fc.z + min(tf[i], fc.w - fc.z) : __viaddmin_u32(tf[i], fc.z, fc.w);
          const uint4 mk = CUBOID_IDX_OK(mi < kMaskTab, a.hdr, 4u) ? s_mtab[mi] : make_uint4(0u, 0u, 0u, 0u);
          m.x |= mk.x;
          m.y |= mk.y;
          m.z |= mk.z;
          m.w |= mk.w;
          // the lane's next pair starts 128 G further on: t <- (t - y) mod f, the smaller
          // of t - y (wraps when t < y) and t - y + f (f <= 2^31, so no wrap)
          if constexpr (kWide)  // a factor above 2^31 (x itself) has multiples 2x, 3x, ... here
            tf[i] = tf[i] >= 0u - fc.y ? tf[i] + fc.y : tf[i] + fc.x;
          else
            tf[i] = __viaddmin_u32(tf[i], fc.y, fma_add(tf[i], fc.x, one));
        }
        for (uint32_t i = kFacRegs; i < nfo; ++i) {
          const uint4 fc = s_fac[i];
          const uint32_t f = fc.x - fc.y;
          uint32_t s = mod_min(wA << 6, f, s_fmag[i]);
          if constexpr (kWide) {
            const unsigned long long ss = (unsigned long long)s + s_fyb[i];
            s = (uint32_t)(ss >= f ? ss - f : ss);
          }
          const uint32_t t = s ? f - s : 0u;
          const uint32_t mi = kWide ? fc.z + min(t, fc.w - fc.z) : __viaddmin_u32(t, fc.z, fc.w);
          const uint4 mk = CUBOID_IDX_OK(mi < kMaskTab, a.hdr, 4u) ? s_mtab[mi] : make_uint4(0u, 0u, 0u, 0u);
          m.x |= mk.x;
          m.y |= mk.y;
          m.z |= mk.z;
          m.w |= mk.w;
        }
      }
      // (a pair with a word outside the subtile, or of an idle group, is an edge pair too)
      if (j - j_lo > j_span || j == j_d) {
        // (whole-warp rows: every lane runs nit = maxit iterations)
        const bool onA = (G == 32 || j < nit) && wA <= wend, onB = (G == 32 || j < nit) && wB <= wend;
        edge_word(wA, onA, m.x, m.y);
        edge_word(wB, onB, m.z, m.w);
      }
      uint32_t alA = ~m.x, ahA = ~m.y, alB = ~m.z, ahB = ~m.w;
      if constexpr (!kMob) {  // pairs of this pair of words: 128 minus the excluded bits
        tile_pairs = fma_add(tile_pairs, 128u, one);
        tile_pairs = fma_sub(tile_pairs, __popc(m.x), one);
        tile_pairs = fma_sub(tile_pairs, __popc(m.y), one);
        tile_pairs = fma_sub(tile_pairs, __popc(m.z), one);
        tile_pairs = fma_sub(tile_pairs, __popc(m.w), one);
      }
      if (kSteps) st_words += ((alA | ahA) ? 1 : 0) + ((alB | ahB) ? 1 : 0);
      // hot primes: no early-exit test; one 128-bit window serves both words
#pragma unroll
      for (int h = 0; h < K; ++h) {
        if (kSteps) st_wsteps += ((alA | ahA) ? 1 : 0) + ((alB | ahB) ? 1 : 0);
        const uint32_t s = sh[h];
        // next pair: + (128 G) mod r; the smaller of s + step and s + step - r (which
        // wraps when s + step < r) is the residue
        sh[h] = __viaddmin_u32(s, a.hot_step[h], fma_add(s, a.hot_step_m[h], one));
        // shared byte address of word s / 32 of the row (s >> 5 by a multiply-high)
        const uint32_t ad = fma_mad(mulhi_fma(s, 1u << 27), 4u, rb4[h]);
        uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0;
        // the window stays inside row (x mod r): s < r, its last word before the row's end
        if (CUBOID_IDX_OK(s < a.hot_r[h] && (s >> 5) + 4 < a.hot_W[h] && rb[h] + (s >> 5) + 4 < a.smem_words,
                          a.hdr, 1u))
          lds5(ad, w0, w1, w2, w3, w4);
        alA &= ~__funnelshift_r(w0, w1, s);  // the window of u_r(x mod r, y0 mod r ...)
        ahA &= ~__funnelshift_r(w1, w2, s);
        alB &= ~__funnelshift_r(w2, w3, s);
        ahB &= ~__funnelshift_r(w3, w4, s);
        if (h + 1 < K)  // the last hot prime's count comes from the queued words
          hs[h] += (__popc(alA) + __popc(ahA)) + (__popc(alB) + __popc(ahB));
      }
      if (kSteps) st_warpsteps += 2 * K;
      enqueue2(alA, ahA, alB, ahB, wA << 6);
    }
    };
    if (mob) word_loop(std::true_type{});
    else word_loop(std::false_type{});
    if constexpr (K > 0) {
      if ((uint32_t)(K - 1) > ws.imax) ws.imax = (uint32_t)(K - 1);
    }
    next = __shfl_sync(FULL, next, 0);
  }
  drain<kSteps, kWide>(a, s_info, s_tab, s_ybr, wcnt, s_queue, qn, K, q_rows, ws.cur_range, lane, ws, st_wsteps,
                       st_warpsteps, true);
  fold();
  flush_counts(ws, wcnt, a, lane);
  if (kSteps) {
    const unsigned long long w = warp_sum_u64(st_words), s = warp_sum_u64(st_wsteps);
    if (lane == 0) {
      atomicAdd(&a.hdr->stats[0], w);
      atomicAdd(&a.hdr->stats[1], s);
      atomicAdd(&a.hdr->stats[2], st_warpsteps);
      atomicAdd(&a.hdr->stats[3], st_tiles);
    }
  }
}

template <bool S, int M, int G, bool W>
cudaError_t set_attr_g(size_t bytes) {
  const int b = (int)bytes;
  cudaError_t e = cudaFuncSetAttribute(k_sieve<S, 0, M, G, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sieve<S, 2, M, G, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sieve<S, 4, M, G, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sieve<S, 5, M, G, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sieve<S, 6, M, G, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

// The step-counting build exists for whole-warp rows only (the counts do not depend on
// the lanes per row), and so does the build for pieces of 64-bit ranges.
template <bool S>
cudaError_t set_attr_all(size_t bytes) {
  cudaError_t e = set_attr_g<S, 1024, 32, false>(bytes);
  if (e == cudaSuccess) e = set_attr_g<S, 512, 32, false>(bytes);
  if constexpr (!S) {
    if (e == cudaSuccess) e = set_attr_g<S, 640, 32, false>(bytes);
    if (e == cudaSuccess) e = set_attr_g<S, 640, 16, false>(bytes);
    if (e == cudaSuccess) e = set_attr_g<S, 640, 8, false>(bytes);
    if (e == cudaSuccess) e = set_attr_g<S, 1024, 16, false>(bytes);
    if (e == cudaSuccess) e = set_attr_g<S, 512, 16, false>(bytes);
    if (e == cudaSuccess) e = set_attr_g<S, 1024, 8, false>(bytes);
    if (e == cudaSuccess) e = set_attr_g<S, 512, 8, false>(bytes);
    if (e == cudaSuccess) e = set_attr_g<S, 1024, 32, true>(bytes);
    if (e == cudaSuccess) e = set_attr_g<S, 512, 32, true>(bytes);
  }
  return e;
}

template <bool S, int M, int G, bool W>
cudaError_t launch_g(const SieveArgs& a, uint32_t blocks, uint32_t threads, size_t smem, cudaStream_t s, bool pdl) {
  switch (a.n_hot) {
    case 6: return launch_ex(k_sieve<S, 6, M, G, W>, blocks, threads, smem, s, pdl, a);
    case 5: return launch_ex(k_sieve<S, 5, M, G, W>, blocks, threads, smem, s, pdl, a);
    case 4: return launch_ex(k_sieve<S, 4, M, G, W>, blocks, threads, smem, s, pdl, a);
    case 2: return launch_ex(k_sieve<S, 2, M, G, W>, blocks, threads, smem, s, pdl, a);
    default: return launch_ex(k_sieve<S, 0, M, G, W>, blocks, threads, smem, s, pdl, a);
  }
}

template <bool S, int M>
cudaError_t launch_m(const SieveArgs& a, uint32_t blocks, uint32_t threads, size_t smem, cudaStream_t s, bool pdl) {
  if constexpr (!S && M != 640) {  // 64-bit pieces: the 512- and 1024-thread builds
    if (a.y_base) return launch_g<S, M, 32, true>(a, blocks, threads, smem, s, pdl);
  }
  if constexpr (!S) {
    if (a.row_lanes == 8) return launch_g<S, M, 8, false>(a, blocks, threads, smem, s, pdl);
    if (a.row_lanes == 16) return launch_g<S, M, 16, false>(a, blocks, threads, smem, s, pdl);
  }
  return launch_g<S, M, 32, false>(a, blocks, threads, smem, s, pdl);
}

// The 128-register variant serves shapes with at most 512 threads per SM.
template <bool S>
cudaError_t launch_k(const SieveArgs& a, uint32_t blocks, uint32_t threads, uint32_t per_sm, size_t smem,
                     cudaStream_t s, bool pdl) {
  if (threads * per_sm <= 512) return launch_m<S, 512>(a, blocks, threads, smem, s, pdl);
  if constexpr (!S) {
    if (threads * per_sm <= 640 && !a.y_base) return launch_m<S, 640>(a, blocks, threads, smem, s, pdl);
  }
  return launch_m<S, 1024>(a, blocks, threads, smem, s, pdl);
}

// Exhaustive check of mod_min: every 32-bit n against the % operator for modulus
// mods[blockIdx.y] (2 <= r < 2^32) with the reciprocal floor(2^32 / r) the tables use
// (floor((2^32 - 1) / r) for the factors, the same value for every r that is not a
// power of two).  bad[y] counts the mismatches.
__global__ void k_probe_mod_min(const uint32_t* mods, unsigned long long* bad) {
  const uint32_t r = mods[blockIdx.y];
  const uint32_t magic = (uint32_t)((1ull << 32) / r);
  unsigned long long miss = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long n = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; n < (1ull << 32);
       n += stride)
    miss += mod_min((uint32_t)n, r, magic) != (uint32_t)n % r;
  miss = warp_sum_u64(miss);
  if ((threadIdx.x & 31) == 0 && miss) atomicAdd(bad + blockIdx.y, miss);
}

}  // namespace

size_t sieve_smem_bytes(uint32_t smem_words, uint32_t n_primes, uint32_t threads, uint32_t row_lanes, bool wide) {
  const uint32_t warps = threads / 32;
  const uint32_t groups = 32 / (row_lanes ? row_lanes : 32);
  const size_t wide_bytes =
      wide ? (size_t)n_primes * sizeof(uint32_t) + (size_t)warps * groups * kMaxFactors * sizeof(uint32_t) : 0;
  return (((size_t)smem_words * 4 + 15) & ~(size_t)15) + (size_t)n_primes * sizeof(PrimeInfo) +
         (size_t)kTrialSmem * sizeof(TrialPrime) +
         (size_t)warps * groups * kMaxFactors * sizeof(uint4) +
         (size_t)warps * kQueue * sizeof(uint4) + kMaskTab * sizeof(uint4) + kPeriodicBelow * sizeof(uint32_t) +
         (size_t)warps * groups * kMaxFactors * sizeof(uint32_t) +
         (size_t)warps * n_primes * sizeof(uint32_t) + wide_bytes;
}

// The dynamic shared-memory limit is a per-device function attribute: raise it only when
// a launch needs more than what was set before (each call costs host time).
cudaError_t sieve_set_smem_limit(bool count_steps, size_t bytes) {
  static std::mutex mu;
  static size_t set_bytes[64][2];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return count_steps ? set_attr_all<true>(bytes) : set_attr_all<false>(bytes);
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set_bytes[dev][count_steps ? 1 : 0];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = count_steps ? set_attr_all<true>(bytes) : set_attr_all<false>(bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaError_t launch_sieve(const SieveArgs& a, bool count_steps, uint32_t blocks, uint32_t threads,
                         size_t smem, cudaStream_t s, bool pdl) {
  if (a.y_base && (count_steps || a.row_lanes != 32 || a.self_plan)) return cudaErrorInvalidValue;
  const uint32_t per_sm = a.n_sms ? (blocks + a.n_sms - 1) / a.n_sms : 2;
  const cudaError_t e = count_steps ? launch_k<true>(a, blocks, threads, per_sm, smem, s, pdl)
                                    : launch_k<false>(a, blocks, threads, per_sm, smem, s, pdl);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace cuboid

extern "C" int cuboid_probe_mod_min(const uint32_t* mods, uint32_t n, uint64_t* mismatches, void* stream) {
  using namespace cuboid;
  if (!mods || !mismatches || n == 0 || n > 65535) return CUBOID_EINVAL;
  for (uint32_t i = 0; i < n; ++i)
    if (mods[i] < 2) return CUBOID_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* d_mods = nullptr;
  unsigned long long* d_bad = nullptr;
  cudaError_t e = cudaMalloc(&d_mods, n * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&d_bad, n * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_mods, mods, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, n * sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_probe_mod_min<<<dim3((unsigned)sms * 8, n), 256, 0, s>>>(d_mods, d_bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(mismatches, d_bad, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_mods);
  cudaFree(d_bad);
  return status_from_cuda(e);
}
