// K2 + K3: the bit sieve of section 2 / the search loop of section 5, on the device.
//
// Work unit ("tile"): one row value x (p, or q when the rectangle is narrow in q) and a
// chunk of consecutive 32-value words of the other coordinate y.  Each lane owns one
// 32-bit word of y values (y0 = 32 w .. 32 w + 31) and carries an "alive" mask of the
// pairs still in play:
//   alive = in-range bits & ~(bits of y sharing a prime factor with x) & ~diagonal,
// then for each prime of the effective order
//   rej   = window(u_r row x mod r, starting at y0 mod r) & alive
//   count[prime] += popc(rej);  alive &= ~rej
// until every lane of the warp is empty (warp-uniform early exit).  The window is one
// funnel shift of two 32-bit words of the window-row table (see cuboid_internal.cuh).
// Survivors (alive bits after the last prime) are compacted with a warp prefix sum and
// one atomic per warp.  Tiles come from a device queue (one atomic per tile), so the
// same kernel serves one range per launch and thousands of ranges per launch.
#include "cuboid_internal.cuh"

namespace cuboid {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t kNoRange = 0xFFFFFFFFu;
constexpr uint32_t kFlushTiles = 256;  // per-warp uint32 counters are flushed at least this often

// n mod r for any 32-bit n, with magic = floor(2^32 / r): the estimate n*magic/2^32 is
// floor(n/r) or one less, so one conditional subtraction finishes the residue.
__device__ __forceinline__ uint32_t fast_mod(uint32_t n, uint32_t r, uint32_t magic) {
  const uint32_t qt = __umulhi(n, magic);
  const uint32_t rem = n - qt * r;
  return rem >= r ? rem - r : rem;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}

// ------------------------------------------------------------------ plan kernel

__global__ void k_reset(DevHeader* hdr, uint32_t n_ranges) {
  DevHeader h = {};
  h.n_ranges = n_ranges;
  *hdr = h;
}

__global__ void __launch_bounds__(1024) k_plan(const cuboid_range* ranges, uint32_t first,
                                               uint32_t count_arg, DevHeader* hdr, TilePlan* plan,
                                               unsigned long long* counts, unsigned long long* npairs,
                                               uint32_t n_primes, uint32_t target_tiles) {
  __shared__ unsigned long long s_words;
  __shared__ unsigned long long s_carry;
  __shared__ unsigned long long s_warp[32];
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t count = count_arg == kNoRange ? hdr->n_ranges : count_arg;
  if (tid == 0) {
    s_words = 0;
    s_carry = 0;
  }
  __syncthreads();
  unsigned long long my_words = 0;
  for (uint32_t k = tid; k < count; k += blockDim.x) {
    const cuboid_range R = ranges[first + k];
    const uint32_t fl = R.flags;
    const bool bad = R.p_lo == 0 || R.q_lo == 0 || R.p_lo > R.p_hi || R.q_lo > R.q_hi ||
                     R.reserved != 0 || (fl & ~0xFu) ||
                     ((fl & CUBOID_ROWS_P) && (fl & CUBOID_ROWS_Q));
    TilePlan P;
    if (bad) {
      atomicOr(&hdr->status, kStatusBadRange);
      P.x_lo = 1;
      P.x_hi = 0;
      P.y_lo = 1;
      P.y_hi = 0;
      P.flags = 0;
    } else {
      const bool rows_q = (fl & CUBOID_ROWS_Q) ||
                          (!(fl & CUBOID_ROWS_P) && (R.p_hi - R.p_lo) > (R.q_hi - R.q_lo));
      P.x_lo = rows_q ? R.q_lo : R.p_lo;
      P.x_hi = rows_q ? R.q_hi : R.p_hi;
      P.y_lo = rows_q ? R.p_lo : R.q_lo;
      P.y_hi = rows_q ? R.p_hi : R.q_hi;
      P.flags = (fl & (CUBOID_Q_LT_P | CUBOID_ALLOW_DIAGONAL)) | (rows_q ? kRowsQ : 0u);
      my_words += ((unsigned long long)(P.x_hi - P.x_lo) + 1) * ((P.y_hi >> 5) - (P.y_lo >> 5) + 1);
    }
    P.chunk_words = 32;
    P.tile_end = 0;
    plan[first + k] = P;
  }
  my_words = warp_sum_u64(my_words);
  if (lane == 0) atomicAdd(&s_words, my_words);
  __syncthreads();
  unsigned long long cw = (s_words + target_tiles - 1) / (target_tiles ? target_tiles : 1);
  cw = (cw + 31) & ~31ull;
  if (cw < 32) cw = 32;
  if (cw > 65536) cw = 65536;  // keeps a warp's uint32 counters below 2^32 between flushes

  for (uint32_t base = 0; base < count; base += blockDim.x) {
    const uint32_t k = base + tid;
    unsigned long long tiles = 0;
    TilePlan P;
    if (k < count) {
      P = plan[first + k];
      if (P.x_lo <= P.x_hi) {
        const unsigned long long nw = (P.y_hi >> 5) - (P.y_lo >> 5) + 1;
        unsigned long long chunk = (nw + 31) & ~31ull;
        if (chunk > cw) chunk = cw;
        P.chunk_words = (uint32_t)chunk;
        tiles = ((unsigned long long)(P.x_hi - P.x_lo) + 1) * ((nw + chunk - 1) / chunk);
      }
    }
    // block inclusive scan of tiles
    unsigned long long v = tiles;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(FULL, v, d);
      if (lane >= (uint32_t)d) v += o;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
      unsigned long long w = lane < (blockDim.x >> 5) ? s_warp[lane] : 0;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long o = __shfl_up_sync(FULL, w, d);
        if (lane >= (uint32_t)d) w += o;
      }
      s_warp[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    const unsigned long long incl = v + (wid ? s_warp[wid - 1] : 0) + s_carry;
    if (k < count) {
      P.tile_end = incl;
      plan[first + k] = P;
    }
    __syncthreads();
    if (tid == blockDim.x - 1) s_carry = incl;
    __syncthreads();
  }
  const unsigned long long nc = (unsigned long long)count * n_primes;
  for (unsigned long long j = tid; j < nc; j += blockDim.x) counts[(unsigned long long)first * n_primes + j] = 0;
  for (uint32_t k = tid; k < count; k += blockDim.x) npairs[first + k] = 0;
  if (tid == 0) {
    hdr->cursor = 0;
    hdr->total_tiles = s_carry;
  }
}

// ------------------------------------------------------------------ sieve kernel

constexpr uint32_t kQueue = 64;    // per-warp queue of words that outlive the hot primes
constexpr int kFacRegs = 4;        // odd factors of the row whose per-lane offsets sit in registers

struct WarpState {
  uint32_t cur_range;
  uint32_t imax;            // deepest prime index reached since the last flush
  uint32_t tiles_since_flush;
  unsigned long long npairs;
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

// Words that outlived the hot primes: up to 32 queued (y0, alive) entries, one per lane,
// go through the remaining primes with a warp-uniform early exit; survivors are
// compacted with a warp prefix sum and one atomic per warp.
template <bool kSteps>
__device__ __forceinline__ void cold_batch(const SieveArgs& a, const PrimeInfo* s_info, const uint32_t* s_tab,
                                           uint32_t* wcnt, const uint2* q, uint32_t cnt, uint32_t first,
                                           uint32_t x, bool rows_q, uint32_t range, uint32_t rowoff_lane,
                                           uint32_t lane, WarpState& ws, unsigned long long& st_wsteps,
                                           unsigned long long& st_warpsteps) {
  const uint2 e = lane < cnt ? q[lane] : make_uint2(0u, 0u);
  const uint32_t y0 = e.x;
  uint32_t alive = e.y;
  const uint32_t n = a.n_primes;
  uint32_t i = first;
  for (; i < a.n_smem_primes; ++i) {
    if (!__any_sync(FULL, alive)) break;
    const PrimeInfo pi = s_info[i];
    const uint32_t ro = (i < 32) ? __shfl_sync(FULL, rowoff_lane, i) : pi.off + fast_mod(x, pi.r, pi.magic) * pi.W;
    const uint32_t s = fast_mod(y0, pi.r, pi.magic);
    const uint32_t wi = ro + (s >> 5);
    const uint32_t win = __funnelshift_r(s_tab[wi], s_tab[wi + 1], s);
    const uint32_t rej = win & alive;
    const uint32_t c = __reduce_add_sync(FULL, __popc(rej));
    if (kSteps) {
      st_wsteps += alive ? 1 : 0;
      st_warpsteps++;
    }
    if (lane == 0 && c) wcnt[i] += c;
    alive ^= rej;
  }
  for (; i < n; ++i) {
    if (!__any_sync(FULL, alive)) break;
    const PrimeInfo pi = s_info[i];
    const uint32_t ro = (i < 32) ? __shfl_sync(FULL, rowoff_lane, i) : pi.off + fast_mod(x, pi.r, pi.magic) * pi.W;
    const uint32_t s = fast_mod(y0, pi.r, pi.magic);
    const uint32_t wi = ro + (s >> 5);
    const uint32_t win = __funnelshift_r(__ldg(a.words + wi), __ldg(a.words + wi + 1), s);
    const uint32_t rej = win & alive;
    const uint32_t c = __reduce_add_sync(FULL, __popc(rej));
    if (kSteps) {
      st_wsteps += alive ? 1 : 0;
      st_warpsteps++;
    }
    if (lane == 0 && c) wcnt[i] += c;
    alive ^= rej;
  }
  const uint32_t reached = i < n ? i : n - 1;
  if (reached > ws.imax) ws.imax = reached;
  if (__any_sync(FULL, alive)) {
    const uint32_t kk = __popc(alive);
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
    while (alive) {
      const uint32_t b = __ffs(alive) - 1;
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

// K: number of "hot" primes (the first K of the effective order, all resident in shared
// memory).  Every word goes through them without an early-exit test, their moduli are
// kernel parameters (constant bank) and their counts accumulate in registers; words
// still alive afterwards are queued and finished by cold_batch.
template <bool kSteps, int K>
__global__ void __launch_bounds__(1024) k_sieve(SieveArgs a) {
  extern __shared__ uint4 smem_raw[];
  const uint32_t n = a.n_primes;
  const uint32_t warps = blockDim.x >> 5;
  const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t lanemask_lt = (1u << lane) - 1u;
  PrimeInfo* s_info = reinterpret_cast<PrimeInfo*>(smem_raw);
  uint4* s_fac_all = smem_raw + n;                                                   // [warps][kMaxFactors]
  uint2* s_queue_all = reinterpret_cast<uint2*>(s_fac_all + warps * kMaxFactors);    // [warps][kQueue]
  uint32_t* s_pat = reinterpret_cast<uint32_t*>(s_queue_all + warps * kQueue);       // [32]
  uint32_t* s_cnt_all = s_pat + 32;                                                  // [warps][n]
  uint32_t* s_tab = s_cnt_all + warps * n;                                           // [smem_words]

  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) s_info[i] = a.info[i];
  for (uint32_t i = threadIdx.x; i < warps * n; i += blockDim.x) s_cnt_all[i] = 0;
  if (threadIdx.x < 32) {  // bits 0, f, 2f, ... of a 32-bit word, for odd f < 32
    uint32_t pat = 0;
    const uint32_t f = threadIdx.x;
    if (f >= 3 && (f & 1))
      for (uint32_t j = 0; j < 32; j += f) pat |= 1u << j;
    s_pat[f] = pat;
  }
  for (uint32_t i = threadIdx.x; i < a.smem_words; i += blockDim.x) s_tab[i] = __ldg(a.words + i);
  __syncthreads();

  uint4* s_fac = s_fac_all + wid * kMaxFactors;
  uint2* s_queue = s_queue_all + wid * kQueue;
  uint32_t* wcnt = s_cnt_all + wid * n;
  const uint32_t count = a.range_count == kNoRange ? a.hdr->n_ranges : a.range_count;
  const unsigned long long total = a.hdr->total_tiles;

  WarpState ws{kNoRange, 0, 0, 0};
  unsigned long long st_words = 0, st_wsteps = 0, st_warpsteps = 0, st_tiles = 0;

  for (;;) {
    unsigned long long tile = 0;
    if (lane == 0) tile = atomicAdd(&a.hdr->cursor, 1ull);
    tile = __shfl_sync(FULL, tile, 0);
    if (tile >= total) break;

    uint32_t k = a.range_first;
    if (count > 1) {  // first range with tile_end > tile
      uint32_t lo = a.range_first, hi = a.range_first + count - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a.plan[mid].tile_end > tile) hi = mid; else lo = mid + 1;
      }
      k = lo;
    }
    const TilePlan P = a.plan[k];
    const unsigned long long tbeg = (k == a.range_first) ? 0ull : a.plan[k - 1].tile_end;
    if (k != ws.cur_range || ws.tiles_since_flush >= kFlushTiles) {
      flush_counts(ws, wcnt, a, lane);
      ws.cur_range = k;
    }
    ws.tiles_since_flush++;

    const bool rows_q = P.flags & kRowsQ;
    const bool tri = P.flags & CUBOID_Q_LT_P;
    const uint32_t diag = (P.flags & CUBOID_ALLOW_DIAGONAL) ? 1u : 0u;
    const uint32_t wbox_lo = P.y_lo >> 5;
    const uint32_t nw = (P.y_hi >> 5) - wbox_lo + 1;
    const uint32_t chunks = (nw + P.chunk_words - 1) / P.chunk_words;
    const unsigned long long local = tile - tbeg;
    unsigned long long row_idx;
    uint32_t chunk;
    if (chunks == 1) {
      row_idx = local;
      chunk = 0;
    } else {
      row_idx = local / chunks;
      chunk = (uint32_t)(local - row_idx * chunks);
    }
    // triangles with p rows: longest rows (largest p) first
    const uint32_t x = (tri && !rows_q) ? P.x_hi - (uint32_t)row_idx : P.x_lo + (uint32_t)row_idx;

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
    if (ylo > yhi) continue;
    const uint32_t wlo = (uint32_t)(ylo >> 5), whi = (uint32_t)(yhi >> 5);
    const uint32_t c0 = wbox_lo + chunk * P.chunk_words;
    const uint32_t c1 = c0 + P.chunk_words - 1;
    const uint32_t wbeg = c0 > wlo ? c0 : wlo;
    const uint32_t wend = c1 < whi ? c1 : whi;
    if (wbeg > wend) continue;
    if (kSteps) st_tiles++;
    const uint32_t lo_mask = FULL << (uint32_t)(ylo & 31);
    const uint32_t hi_mask = FULL >> (31 - (uint32_t)(yhi & 31));
    const uint32_t dword = x >> 5, dbit = 1u << (x & 31);

    // ---- distinct odd prime factors of x (warp-cooperative trial division)
    uint32_t nfo = 0;
    bool has2 = false;
    {
      uint32_t m = x;
      if ((m & 1u) == 0) {
        has2 = true;
        m >>= __ffs(m) - 1;
      }
      for (uint32_t base = 0; base < a.n_trial; base += 32) {
        const uint32_t f0 = __ldg(&a.trial[base].f);
        if ((unsigned long long)f0 * f0 > m) break;
        const uint32_t idx = base + lane;
        const TrialPrime tp = idx < a.n_trial ? a.trial[idx] : TrialPrime{1u, 1u, 0u, 0u};
        const bool hit = idx < a.n_trial && m * tp.inv <= tp.lim;
        uint32_t bal = __ballot_sync(FULL, hit);
        while (bal) {
          const uint32_t b = __ffs(bal) - 1;
          bal &= bal - 1;
          const uint32_t f = __shfl_sync(FULL, tp.f, b);
          const uint32_t inv = __shfl_sync(FULL, tp.inv, b);
          const uint32_t lim = __shfl_sync(FULL, tp.lim, b);
          while (m * inv <= lim) m *= inv;   // exact division by f
          if (lane == 0) s_fac[nfo] = make_uint4(f, 0xFFFFFFFFu / f, f < 32 ? s_pat[f] : 1u, 1024u % f);
          ++nfo;
        }
      }
      if (m > 1) {
        if (lane == 0) s_fac[nfo] = make_uint4(m, 0xFFFFFFFFu / m, m < 32 ? s_pat[m] : 1u, 1024u % m);
        ++nfo;
      }
      __syncwarp();
    }
    // per-lane offset of the first multiple of each odd factor in the lane's first word
    uint32_t tf[kFacRegs];
    {
      const uint32_t y0f = (wbeg + lane) << 5;
#pragma unroll
      for (int i = 0; i < kFacRegs; ++i) {
        tf[i] = 0;
        if ((uint32_t)i < nfo) {
          const uint4 fc = s_fac[i];
          const uint32_t s = fast_mod(y0f, fc.x, fc.y);
          tf[i] = s ? fc.x - s : 0u;
        }
      }
    }

    // ---- row offsets: hot primes in registers, the first 32 primes one per lane
    uint32_t rb[K > 0 ? K : 1];
#pragma unroll
    for (int h = 0; h < K; ++h) rb[h] = a.hot_off[h] + fast_mod(x, a.hot_r[h], a.hot_magic[h]) * a.hot_W[h];
    uint32_t rowoff_lane = 0;
    if (lane < n) {
      const PrimeInfo pi = s_info[lane];
      rowoff_lane = pi.off + fast_mod(x, pi.r, pi.magic) * pi.W;
    }

    uint32_t hcnt[K > 0 ? K : 1];
#pragma unroll
    for (int h = 0; h < (K > 0 ? K : 1); ++h) hcnt[h] = 0;
    uint32_t tile_pairs = 0;
    uint32_t qn = 0;

    for (uint32_t wb = wbeg; wb <= wend; wb += 32) {
      const uint32_t w = wb + lane;
      const uint32_t y0 = w << 5;
      uint32_t alive = 0;
      if (w <= wend) {
        uint32_t rm = FULL;
        if (w == wlo) rm &= lo_mask;
        if (w == whi) rm &= hi_mask;
        alive = has2 ? (rm & 0xAAAAAAAAu) : rm;  // y0 is even: even y at even bit positions
#pragma unroll
        for (int i = 0; i < kFacRegs; ++i) {
          if ((uint32_t)i < nfo) {
            const uint4 fc = s_fac[i];
            if (tf[i] < 32) alive &= ~(fc.z << tf[i]);
            const uint32_t tn = tf[i] - fc.w;  // the lane's next word starts 1024 further on
            tf[i] = (int)tn < 0 ? tn + fc.x : tn;
          }
        }
        for (uint32_t i = kFacRegs; i < nfo; ++i) {
          const uint4 fc = s_fac[i];
          const uint32_t s = fast_mod(y0, fc.x, fc.y);
          const uint32_t j0 = s ? fc.x - s : 0u;
          if (j0 < 32) alive &= ~(fc.z << j0);
        }
        if (w == dword) {
          alive &= ~dbit;
          if (diag) alive |= dbit & rm;
        }
        tile_pairs += __popc(alive);
        if (kSteps) st_words += alive ? 1 : 0;
      }
      // hot primes: no early-exit test
#pragma unroll
      for (int h = 0; h < K; ++h) {
        if (kSteps) st_wsteps += alive ? 1 : 0;
        const uint32_t s = fast_mod(y0, a.hot_r[h], a.hot_magic[h]);
        const uint32_t wi = rb[h] + (s >> 5);
        const uint32_t win = __funnelshift_r(s_tab[wi], s_tab[wi + 1], s);
        const uint32_t rej = win & alive;
        hcnt[h] += __popc(rej);
        alive ^= rej;
      }
      if (kSteps) st_warpsteps += K;
      // queue the words still alive
      const uint32_t bal = __ballot_sync(FULL, alive != 0u);
      if (bal) {
        if (alive) s_queue[qn + __popc(bal & lanemask_lt)] = make_uint2(y0, alive);
        qn += __popc(bal);
        __syncwarp();
        if (qn >= 32) {
          cold_batch<kSteps>(a, s_info, s_tab, wcnt, s_queue, 32, K, x, rows_q, k, rowoff_lane, lane, ws,
                             st_wsteps, st_warpsteps);
          const uint32_t rest = qn - 32;
          uint2 e = make_uint2(0u, 0u);
          if (lane < rest) e = s_queue[32 + lane];
          __syncwarp();
          if (lane < rest) s_queue[lane] = e;
          __syncwarp();
          qn = rest;
        }
      }
    }
    if (qn)
      cold_batch<kSteps>(a, s_info, s_tab, wcnt, s_queue, qn, K, x, rows_q, k, rowoff_lane, lane, ws, st_wsteps,
                         st_warpsteps);
    // tile totals
#pragma unroll
    for (int h = 0; h < K; ++h) {
      const uint32_t c = __reduce_add_sync(FULL, hcnt[h]);
      if (lane == 0 && c) wcnt[h] += c;
    }
    if constexpr (K > 0) {
      if ((uint32_t)(K - 1) > ws.imax) ws.imax = (uint32_t)(K - 1);
    }
    ws.npairs += __reduce_add_sync(FULL, tile_pairs);
    __syncwarp();
  }
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

}  // namespace

size_t sieve_smem_bytes(uint32_t smem_words, uint32_t n_primes, uint32_t threads) {
  const uint32_t warps = threads / 32;
  return (size_t)n_primes * sizeof(PrimeInfo) + (size_t)warps * kMaxFactors * sizeof(uint4) +
         (size_t)warps * kQueue * sizeof(uint2) + 32 * sizeof(uint32_t) +
         (size_t)warps * n_primes * sizeof(uint32_t) + (size_t)smem_words * sizeof(uint32_t);
}

namespace {
template <bool S>
cudaError_t set_attr_all(size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_sieve<S, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sieve<S, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sieve<S, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sieve<S, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}
template <bool S>
void launch_k(const SieveArgs& a, uint32_t blocks, uint32_t threads, size_t smem, cudaStream_t s) {
  switch (a.n_hot) {
    case 6: k_sieve<S, 6><<<blocks, threads, smem, s>>>(a); break;
    case 4: k_sieve<S, 4><<<blocks, threads, smem, s>>>(a); break;
    case 2: k_sieve<S, 2><<<blocks, threads, smem, s>>>(a); break;
    default: k_sieve<S, 0><<<blocks, threads, smem, s>>>(a); break;
  }
}
}  // namespace

cudaError_t sieve_set_smem_limit(bool count_steps, size_t bytes) {
  return count_steps ? set_attr_all<true>(bytes) : set_attr_all<false>(bytes);
}

cudaError_t launch_reset(DevHeader* hdr, uint32_t n_ranges, cudaStream_t s) {
  k_reset<<<1, 1, 0, s>>>(hdr, n_ranges);
  return cudaGetLastError();
}

cudaError_t launch_plan(const cuboid_range* ranges, uint32_t first, uint32_t count, DevHeader* hdr,
                        TilePlan* plan, unsigned long long* counts, unsigned long long* npairs,
                        uint32_t n_primes, uint32_t target_tiles, cudaStream_t s) {
  k_plan<<<1, 1024, 0, s>>>(ranges, first, count, hdr, plan, counts, npairs, n_primes, target_tiles);
  return cudaGetLastError();
}

cudaError_t launch_sieve(const SieveArgs& a, bool count_steps, uint32_t blocks, uint32_t threads,
                         size_t smem, cudaStream_t s) {
  if (count_steps)
    launch_k<true>(a, blocks, threads, smem, s);
  else
    launch_k<false>(a, blocks, threads, smem, s);
  return cudaGetLastError();
}

}  // namespace cuboid
