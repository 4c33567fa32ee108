// Internal declarations shared by the translation units of libcuboid.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "cuboid.h"

namespace cuboid {

constexpr uint32_t kMaxPrimes = 1280;       // every prime below the Eq. 2.7 bound (1196 of them) fits
constexpr uint32_t kPrimeLimit = 9697;     // r < 9697: the bound derived below Eq. 2.7
constexpr uint32_t kStageSpins = 1u << 22;    // polls of a CTA's staging barrier before it gives up
constexpr uint32_t kMaxChunkWords = 32768;   // 64-value words per subtile: at most 2^21 pairs
constexpr uint32_t kMaxFactors = 10;       // distinct primes of a 32-bit integer <= 9
constexpr uint32_t kSieveRevision = 22;    // part of the autotuner's cache key: bump when the kernel changes

// Coprimality mask image: for each odd prime f < 128 and offset t in [0, f) the 128-bit
// mask of bits t, t + f, t + 2f, ... (as four uint32 quarters: two adjacent 64-value
// words), then the single bits 1 << t for t in [0, 128) and an empty mask at index 128 (a
// factor f >= 128 hits a pair of words at most once); then, for each n < 128, the index of
// n's first mask if n is an odd prime, else the single-bit block.  Built once with the
// tables; staged into each CTA's shared memory.
constexpr uint32_t kPeriodicBelow = 128;  // factors below this get periodic masks
constexpr uint32_t odd_prime_sum_below(uint32_t lim) {
  uint32_t s = 0;
  for (uint32_t f = 3; f < lim; f += 2) {
    bool prime = true;
    for (uint32_t d = 3; d * d <= f; d += 2) prime = prime && (f % d != 0);
    if (prime) s += f;
  }
  return s;
}
constexpr uint32_t kBitTab = odd_prime_sum_below(kPeriodicBelow);  // 1718: periodic masks
constexpr uint32_t kMaskTab = kBitTab + 129;                       // 128-bit entries of the mask table
static_assert(kBitTab == 1718, "mask table layout");
constexpr uint32_t kMaskImageWords = 4 * kMaskTab + kPeriodicBelow;  // masks, then the offsets
static_assert((kMaskImageWords * 4) % 16 == 0, "bulk-copy size");

// Per-prime sieve constants, one entry per prime in the effective order.  16 bytes.
struct PrimeInfo {
  uint32_t r;      // the prime
  uint32_t magic;  // floor(2^32 / r): residue of a 32-bit n by one mul.hi and one fix-up
  uint32_t off;    // first word of row 0 in the window-row blob
  uint32_t W;      // words per row: floor((r - 1) / 32) + 5
};

// Window-row layout: row a of prime r holds W 32-bit words; bit j (0 <= j < 32 W) is
// u_r(a, j mod r).  The 128 bits u_r(a, s), ..., u_r(a, s + 127 mod r) for any s < r (two
// adjacent 64-value words) are four funnel shifts of words s/32 ... s/32 + 4; the first
// 64 of them are two funnel shifts of words s/32 ... s/32 + 2.
__host__ __device__ inline uint32_t row_words(uint32_t r) { return (r - 1) / 32 + 5; }

// One planned range.  32 bytes.
struct TilePlan {
  uint32_t x_lo, x_hi;   // row variable bounds (p, or q when kRowsQ)
  uint32_t y_lo, y_hi;   // word-dimension bounds of the rectangle
  uint32_t flags;        // range flags | kRowsQ
  uint32_t chunk_words;  // words per tile (multiple of 32)
  uint64_t tile_end;     // tiles of ranges [first, this] (inclusive prefix sum)
};
constexpr uint32_t kRowsQ = 0x80000000u;

// Device header of a result object.
struct DevHeader {
  unsigned long long cursor;       // tiles handed out after each warp's first (fixed) tile
  unsigned long long total_tiles;  // tiles of the running launch
  unsigned long long n_surv;       // survivors found (may exceed the capacity)
  unsigned long long n_roots;      // roots found (may exceed the capacity)
  unsigned int status;             // kStatus* bits
  unsigned int n_ranges;           // ranges of a batched launch
  unsigned long long stats[4];     // cuboid_stats fields
  unsigned int debug_code;         // CUBOID_DEBUG builds: the first failed index check (0: none)
  unsigned int debug_pad;
};
constexpr unsigned kStatusSurvOverflow = 1u;
constexpr unsigned kStatusRootOverflow = 2u;
constexpr unsigned kStatusBadRange = 4u;
constexpr unsigned kStatusVerifyFail = 8u;
constexpr unsigned kStatusStageTimeout = 16u;  // a CTA's shared-memory staging did not complete
constexpr unsigned kStatusDebugIndex = 32u;    // CUBOID_DEBUG builds: an index check failed

// Index checks of the CUBOID_DEBUG build: CUBOID_IDX_OK(cond, hdr, code) is true in a
// release build; in a debug build it is cond, and when cond is false it records
// kStatusDebugIndex and the first failing check's code in the header, and the caller skips
// the access (no trap, no assert: the kernel finishes and the host reads the status).
// Codes: 1 hot-prime window (shared), 2 cold window (shared), 3 cold window (global),
// 4 coprimality mask entry, 5 factor record, 6 per-warp queue slot, 7 queue refill slot.
#ifdef CUBOID_DEBUG
__device__ __forceinline__ bool debug_index_ok(bool ok, DevHeader* hdr, unsigned code) {
  if (!ok) {
    atomicOr(&hdr->status, kStatusDebugIndex);
    atomicCAS(&hdr->debug_code, 0u, code);
  }
  return ok;
}
#define CUBOID_IDX_OK(cond, hdr, code) ::cuboid::debug_index_ok((cond), (hdr), (code))
#else
#define CUBOID_IDX_OK(cond, hdr, code) true
#endif

// Odd trial-division primes below 2^16 with the exact-divisibility constants
// inv = f^-1 mod 2^32 and lim = floor((2^32 - 1) / f):  f | n  <=>  n * inv <= lim.
// ---- planning of one range (shared by the plan kernel and the single-range sieve)

// Orientation and word count of a range: rows of p, or of q when the rectangle is narrow
// in q (or forced by the flags).  Returns false for an invalid range (P is then empty).
__host__ __device__ inline bool plan_orient(const cuboid_range& R, TilePlan& P, unsigned long long& words) {
  const uint32_t fl = R.flags;
  const bool bad = R.p_lo == 0 || R.q_lo == 0 || R.p_lo > R.p_hi || R.q_lo > R.q_hi || R.reserved != 0 ||
                   (fl & ~0xFu) || ((fl & CUBOID_ROWS_P) && (fl & CUBOID_ROWS_Q));
  P.chunk_words = 1;
  P.tile_end = 0;
  words = 0;
  if (bad) {
    P.x_lo = 1;
    P.x_hi = 0;
    P.y_lo = 1;
    P.y_hi = 0;
    P.flags = 0;
    return false;
  }
  const bool rows_q = (fl & CUBOID_ROWS_Q) || (!(fl & CUBOID_ROWS_P) && (R.p_hi - R.p_lo) > (R.q_hi - R.q_lo));
  P.x_lo = rows_q ? R.q_lo : R.p_lo;
  P.x_hi = rows_q ? R.q_hi : R.p_hi;
  P.y_lo = rows_q ? R.p_lo : R.q_lo;
  P.y_hi = rows_q ? R.p_hi : R.q_hi;
  P.flags = (fl & (CUBOID_Q_LT_P | CUBOID_ALLOW_DIAGONAL)) | (rows_q ? kRowsQ : 0u);
  words = ((unsigned long long)(P.x_hi - P.x_lo) + 1) * ((P.y_hi >> 6) - (P.y_lo >> 6) + 1);
  return true;
}

// Words per subtile from the total words of a launch and its target number of tiles.
__host__ __device__ inline unsigned long long plan_chunk(unsigned long long total_words, uint32_t target_tiles,
                                                         uint32_t subtiles_per_tile) {
  const unsigned long long target_sub = (unsigned long long)(target_tiles ? target_tiles : 1) * subtiles_per_tile;
  unsigned long long cw = (total_words + target_sub - 1) / target_sub;
  if (cw < 1) cw = 1;
  if (cw > kMaxChunkWords) cw = kMaxChunkWords;
  return cw;
}

// Sets P.chunk_words and returns the range's tiles (subtiles_per_tile subtiles each).
__host__ __device__ inline unsigned long long plan_tiles(TilePlan& P, unsigned long long cw,
                                                         uint32_t subtiles_per_tile) {
  if (P.x_lo > P.x_hi) return 0;
  const unsigned long long nw = (P.y_hi >> 6) - (P.y_lo >> 6) + 1;
  const unsigned long long chunk = nw < cw ? nw : cw;
  P.chunk_words = (uint32_t)chunk;
  const unsigned long long subtiles = ((unsigned long long)(P.x_hi - P.x_lo) + 1) * ((nw + chunk - 1) / chunk);
  return (subtiles + subtiles_per_tile - 1) / subtiles_per_tile;
}

struct TrialPrime {
  uint32_t f, inv, lim, pad;
};

}  // namespace cuboid

struct cuboid_tables {
  int device = 0;
  uint32_t n = 0;
  uint32_t flags = 0;
  std::vector<uint32_t> primes;     // caller order
  std::vector<uint32_t> order;      // effective order -> caller index
  std::vector<uint32_t> unsolvable; // per caller index: number of k with v_r(k) = 1
  std::vector<cuboid::PrimeInfo> info;  // effective order
  uint64_t total_words = 0;
  cuboid::PrimeInfo* d_info = nullptr;
  uint32_t* d_words = nullptr;      // window rows, effective order
  uint8_t* d_vbytes = nullptr;      // v_r bytes, caller order, at vbyte_off[i]
  std::vector<uint64_t> vbyte_off;
  cuboid::TrialPrime* d_trial = nullptr;
  uint32_t* d_mimg = nullptr;       // coprimality mask image (kMaskImageWords)
  uint32_t n_trial = 0;
  cuboid_tuning tuning{};
  std::atomic<int> users{0};        // servers and searches holding the tables
  bool searching = false;           // a region search runs on these tables
  int sms = 0;
  int smem_per_sm = 0;              // device limits read once at build time
  int smem_per_block = 0;
};

namespace cuboid {

// Launch parameters of the sieve kernel.
struct SieveArgs {
  const PrimeInfo* info;
  const uint32_t* words;
  const TrialPrime* trial;
  const uint32_t* mimg;          // coprimality mask image
  const TilePlan* plan;
  DevHeader* hdr;
  unsigned long long* counts;   // [range][prime, effective order]
  unsigned long long* npairs;   // [range]
  unsigned long long* surv;     // (p << 32 | q)
  uint32_t* surv_range;
  unsigned long long surv_cap;
  uint32_t n_primes;
  uint32_t n_smem_primes;
  uint32_t smem_words;
  uint32_t n_trial;
  uint32_t range_first;
  uint32_t range_count;         // UINT32_MAX: read hdr->n_ranges
  uint32_t n_hot;               // hot primes (0, 2, 4, 5, 6 or 8): the first n_hot of the effective order
  uint32_t hot_r[8], hot_magic[8], hot_off[8], hot_W[8];
  uint32_t hot_step[8];          // (128 row_lanes) mod r: a lane's stride between pairs of words
  uint32_t hot_step_m[8];        // hot_step - r (mod 2^32)
  uint32_t one = 1;              // the multiplier of the adds the sieve issues on the FMA pipe
  uint32_t row_lanes;            // lanes per row (8, 16, 32)
  uint32_t stage_spins;          // polls of the staging barrier before a time-out
  // Single-range launch without a plan kernel (self_plan = 1): every CTA plans the range
  // itself (read from self_range, or self_range_val when that is null) for target_tiles
  // tiles; the header, counts and pair total start at zero (the previous run cleared them).
  uint32_t self_plan = 0;
  uint32_t target_tiles = 0;
  const cuboid_range* self_range = nullptr;
  cuboid_range self_range_val = {};
  uint32_t n_sms;               // SMs of the device (picks the register budget of the variant)
  unsigned long long total_words = 0;  // window-row words of the tables (index checks of debug builds)
  // Piece of a 64-bit range: the planned y (word) coordinates are relative to y_base, a
  // multiple of 64 at or above 2^32 - 64, and every y of the piece is at least 2^32, above
  // any 32-bit row value x (so the piece holds no diagonal pair and no triangle edge).
  // 0: a 32-bit range.
  unsigned long long y_base = 0;
};
constexpr uint32_t kMaxHot = 8;

struct VerifyArgs {
  const unsigned long long* surv;
  const uint32_t* surv_range;
  unsigned long long surv_cap;
  DevHeader* hdr;
  cuboid_root* roots;
  uint32_t* root_range;
  unsigned long long root_cap;
  // 64-bit ranges (may be null): per range index k, base[2 k] and base[2 k + 1] are added
  // to the record's p and q (the sieve writes them relative to the piece's base)
  const unsigned long long* base = nullptr;
  // cleared by block 0 after the sieve (may be null): the header and first pair total,
  // and the first range's counts, of the result block the next single-range run uses
  unsigned long long* zero_block = nullptr;
  uint32_t zero_words = 0;
  unsigned long long* zero_block2 = nullptr;
  uint32_t zero_words2 = 0;
  // bits of the largest p or q any record can hold (picks the root test's moduli budget);
  // 0: unknown (32-bit pairs, or pairs below 2^40 when base is set)
  uint32_t max_bits = 0;
};

// Bits of the largest coordinate of n host ranges (0 for none).
inline uint32_t ranges_max_bits(const cuboid_range* r, uint32_t n) {
  uint32_t m = 0;
  for (uint32_t i = 0; i < n; ++i) m |= r[i].p_hi | r[i].q_hi;
  uint32_t b = 0;
  while (m) {
    ++b;
    m >>= 1;
  }
  return b;
}

// Launchers (each checks its own launch and returns cudaError_t).
cudaError_t launch_plan(const cuboid_range* ranges, uint32_t first, uint32_t count,
                        DevHeader* hdr, TilePlan* plan, unsigned long long* counts,
                        unsigned long long* npairs, uint32_t n_primes, uint32_t target_tiles,
                        cudaStream_t s, bool reset, uint32_t row_lanes,
                        const cuboid_range* inline_range = nullptr);  // host range passed by value (count 1)
cudaError_t launch_reset(DevHeader* hdr, uint32_t n_ranges, cudaStream_t s);
// pdl: launch as a programmatic dependent of the kernel just before it in the stream (the
// grid is scheduled while that kernel runs and waits on griddepcontrol.wait before it
// reads what that kernel wrote).  Only when the previous stream operation is that kernel.
cudaError_t launch_sieve(const SieveArgs& a, bool count_steps, uint32_t blocks,
                         uint32_t threads, size_t smem, cudaStream_t s, bool pdl = false);
size_t sieve_smem_bytes(uint32_t smem_words, uint32_t n_primes, uint32_t threads, uint32_t row_lanes,
                        bool wide = false);
cudaError_t sieve_set_smem_limit(bool count_steps, size_t bytes);
cudaError_t launch_verify(const VerifyArgs& a, uint32_t blocks, cudaStream_t s, bool pdl = false);

// Programmatic dependent launch: a dependent grid waits here until the grid before it has
// completed and its writes are visible (a no-op in a grid launched without the attribute);
// a primary grid lets its dependent be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// cudaLaunchKernelEx with the programmatic-serialization attribute when pdl is set.
template <class... KArgs, class... Args>
cudaError_t launch_ex(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                      Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
cudaError_t verify_init_device();   // upload the 62-bit moduli (once per device)

// Sieve launch shape chosen from the tables' tuning (runtime.cu).
struct LaunchShape {
  uint32_t threads, blocks, n_smem, smem_words, target_tiles, n_hot, row_lanes;
  size_t smem;
};
void fill_hot(SieveArgs& a, const cuboid_tables* t, const LaunchShape& L);
// count_steps: the step-counting build, which exists for whole-warp rows only.  wide: the
// build for pieces of 64-bit ranges (whole-warp rows, more shared memory).
LaunchShape launch_shape(const cuboid_tables* t, bool count_steps = false, bool wide = false);

// packed: NULL (tables from the definition), or per caller index the host address of the
// prime's Eq. 2.6 bytes (ceil(r^2 / 8)), which become the full tables as they are.
int build_tables(const uint32_t* primes, uint32_t n, uint32_t flags, cudaStream_t s, cuboid_tables** out,
                 const uint8_t* const* packed);

int status_from_cuda(cudaError_t e);

}  // namespace cuboid
