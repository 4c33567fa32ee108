/*
 * cuboid.h -- C ABI of libcuboid: the modulo-primes sieve for the second cuboid
 * conjecture on one GB300 (sm_103a).
 *
 * Method (arXiv:1601.00636, Gallyamov, Kadyrov, Kashelevskiy, Kutlugallyamov, Sharipov):
 *   For coprime p != q the tenth-degree polynomial Q_pq(t) of Eq. 1.1 can only have an
 *   integer root if, for every prime r, the residue pair (p mod r, q mod r) is
 *   "solvable" (Definition 1.1, section 2).  The unsolvability bits u_r (Eq. 2.3) of a
 *   list of primes form a bit sieve (section 2); a pair is rejected by the first prime
 *   of the list whose bit is 1, and the search of section 5 walks (p, q) through it.
 *   Pairs that no prime rejects ("survivors") get an exact test for integer roots.
 *
 * Conventions shared by every call:
 *   - Every function returns an int status (CUBOID_OK or a CUBOID_E* code below).
 *     Misuse is reported by the status and never crashes (section 5 gives the same
 *     contract for the paper's DLL).  Output arguments are written only on CUBOID_OK
 *     unless a call says otherwise.
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Calls that enqueue device work return without waiting unless they say so.
 *   - Objects are bound to the CUDA device that was current when they were created;
 *     use them with that device current.  The library owns every device and pinned
 *     host buffer it allocates; handles are freed by the matching *_free/_destroy.
 *   - Ranges are inclusive on both ends; p and q are 32-bit (1 <= p, q <= 2^32 - 1),
 *     except in the calls of the "64-bit ranges" section (p, q < 2^40).
 *   - Counts are indexed by the caller's prime list.  counts[i] is the number of pairs
 *     whose FIRST rejecting prime, in the effective order, is primes[i].
 */
#ifndef CUBOID_H
#define CUBOID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
/* 0, 1, 2 and 6 follow the codes of the paper's Start_searching / Release calls
 * (section 5): 0 success, 1 busy, 2..5 out-of-range start values, 6 tables missing. */
#define CUBOID_OK          0
#define CUBOID_EBUSY       1  /* object in use (tables held by a server; no free slot) */
#define CUBOID_ERANGE      2  /* a bound is 0, lo > hi, or p, q outside 32 bits; search: p < 152 */
#define CUBOID_EPMAX       3  /* search: p > 72796055, so 59 p leaves 32 bits (section 5) */
#define CUBOID_EQLOW       4  /* search: q below the region of Eq. 5.2 */
#define CUBOID_EQHIGH      5  /* search: q above 59 p (Eq. 5.2) */
#define CUBOID_ENOTABLES   6  /* NULL tables handle */
#define CUBOID_EINVAL      7  /* invalid argument (NULL pointer, bad prime list, ...) */
#define CUBOID_ENOMEM      8  /* device or pinned allocation failed */
#define CUBOID_ETIMEOUT    9  /* a bounded wait expired */
#define CUBOID_ECUDA      10  /* a CUDA runtime call failed */
#define CUBOID_EOVERFLOW  11  /* an output buffer was too small (counts stay exact) */
#define CUBOID_EAGAIN     12  /* not finished yet (server poll) */
#define CUBOID_EVERIFY    13  /* the exact root test could not settle a survivor */
#define CUBOID_ETOOLARGE  14  /* more ranges than the fixed capacity of cuboid_sieve_noalloc */
#define CUBOID_EINDEX     15  /* CUBOID_DEBUG build only: a kernel's index check failed (the access was skipped) */

/* ------------------------------------------------------------ build flags */
#define CUBOID_ORDER_AS_GIVEN    0x0u /* sieve the primes in the caller's order */
#define CUBOID_ORDER_BY_DENSITY  0x1u /* decreasing unsolvable fraction, ties: smaller r */
#define CUBOID_ORDER_BY_RATE     0x4u /* decreasing rejection rate of a coprime pair: the
                                         number of unsolvable k over r + 1; ties: smaller r */
#define CUBOID_BUILD_REDUCED     0x0u /* u_r from v_r(k)=u_r(k,1) by homogeneity (default) */
#define CUBOID_BUILD_FULL        0x2u /* u_r by trying every t for every (p~, q~) */
#define CUBOID_TABLES_IMPORTED   0x10u /* info flag: the tables came from paper-format files */
#define CUBOID_IMPORT_CHECK      0x8u /* import: compare every table with the definition */

/* ------------------------------------------------------------ range flags */
#define CUBOID_Q_LT_P            0x1u /* only q < p (q <= p with ALLOW_DIAGONAL) */
#define CUBOID_ALLOW_DIAGONAL    0x2u /* also sieve p == q, whatever gcd(p, p) (tests) */
#define CUBOID_ROWS_P            0x4u /* force tiles with one p per row */
#define CUBOID_ROWS_Q            0x8u /* force tiles with one q per row */

/* ------------------------------------------------------------ sieve modes */
#define CUBOID_MODE_PLAIN        0x0u /* one kernel launch sequence per range */
#define CUBOID_MODE_BATCHED      0x1u /* all ranges in one persistent launch (CUDA graph) */
#define CUBOID_MODE_COUNT_STEPS  0x100u /* also count sieve steps (cuboid_result_stats) */
#define CUBOID_MODE_TIME_SIEVE   0x200u /* time the sieve kernel(s) with CUDA events */
#define CUBOID_MODE_STAGE_TIMEOUT 0x400u /* failure test: every CTA's bounded wait for its
                                            shared-memory staging gives up at once; the
                                            CTAs leave once their copies land and the run
                                            reports CUBOID_ETIMEOUT (plain mode only) */

typedef struct cuboid_tables cuboid_tables;
typedef struct cuboid_result cuboid_result;
typedef struct cuboid_server cuboid_server;

/* One rectangle [p_lo, p_hi] x [q_lo, q_hi] with CUBOID_Q_LT_P / ALLOW_DIAGONAL /
 * ROWS_* flags; reserved must be 0.  24 bytes. */
typedef struct cuboid_range {
  uint32_t p_lo, p_hi, q_lo, q_hi;
  uint32_t flags;
  uint32_t reserved;
} cuboid_range;

/* An integer root t > 0 of Q_pq (t may exceed 64 bits: t = t_hi * 2^64 + t_lo). */
typedef struct cuboid_root {
  uint32_t p, q;
  uint64_t t_lo, t_hi;
} cuboid_root;

/* Kernel shape.  Any field 0 means "library default".  Results never depend on it. */
typedef struct cuboid_tuning {
  uint32_t block_threads;   /* threads per CTA of the sieve kernel (multiple of 32) */
  uint32_t ctas_per_sm;     /* persistent CTAs per SM */
  uint32_t smem_primes;     /* how many leading primes (effective order) sit in shared memory */
  uint32_t tiles_per_warp;  /* target number of work tiles per warp (sets the tile size) */
  uint32_t hot_primes;      /* leading primes tested without an early-exit check (0..8) */
  uint32_t row_lanes;       /* lanes sieving one row: 8, 16 or 32 (a warp then takes 4, 2 or
                               1 rows at a time; fewer lanes share a row's setup among fewer
                               words, which pays on short rows) */
} cuboid_tuning;

/* Instrumentation filled by runs with CUBOID_MODE_COUNT_STEPS. */
typedef struct cuboid_stats {
  uint64_t words;        /* 32-q words that held at least one sieved pair */
  uint64_t word_steps;   /* sum over words of primes tried until the word was all rejected */
  uint64_t warp_steps;   /* prime steps executed per warp (times 32 = lane slots issued) */
  uint64_t tiles;        /* non-empty tiles */
} cuboid_stats;

/* ================================================================ tables (section 2) */

/* Build the unsolvability tables u_r (Eq. 2.3, Definition 1.1) for n primes on the
 * current device.
 *   primes: host array of n distinct primes, 2 <= r < 9697 (the bound below Eq. 2.7),
 *           1 <= n <= 1280 (every prime below 9697 fits: the full list from 11 is 1192
 *           primes, whose tables take 4.4 GB of device memory).
 *   flags:  one CUBOID_ORDER_* | CUBOID_BUILD_*.
 *   stream: work is enqueued on it; the call synchronises the stream before returning
 *           (the effective order is needed on the host).
 *   out:    receives the handle; free with cuboid_tables_free.
 * Errors: EINVAL (NULL, n out of range, r not a prime, r >= 9697, duplicates),
 *         ENOMEM, ECUDA. */
int cuboid_tables_build(const uint32_t* primes, uint32_t n, uint32_t flags, void* stream,
                        cuboid_tables** out);

/* Number of primes, bytes of device table memory, build flags (any pointer may be NULL). */
int cuboid_tables_info(const cuboid_tables* t, uint32_t* n_primes, uint64_t* device_bytes,
                       uint32_t* flags);

/* The effective sieve order: order_out[k] = index (into the caller's list) of the k-th
 * prime tried.  order_out holds n entries. */
int cuboid_tables_order(const cuboid_tables* t, uint32_t* order_out);

/* Copy the table of primes[prime_idx] in the byte layout of Eq. 2.6: bit i = p~ r + q~
 * at byte i/8, bit position i%8 (least significant first), last byte zero-padded;
 * ceil(r^2/8) bytes.  *written (may be NULL) receives that size.  Synchronous.
 * Errors: EINVAL (index), EOVERFLOW (dst NULL or cap too small; *written still set). */
int cuboid_tables_copy_bits(const cuboid_tables* t, uint32_t prime_idx, uint8_t* dst,
                            size_t cap, size_t* written);

/* Copy v_r(k) = u_r(k, 1), k = 0..r-1, one byte (0/1) per k, for primes[prime_idx].
 * Synchronous.  Errors: EINVAL, EOVERFLOW (cap < r). */
int cuboid_tables_copy_reduced(const cuboid_tables* t, uint32_t prime_idx, uint8_t* dst,
                               size_t cap);

/* The paper's two table files (section 2; written by Write_pq_file_stream, section 3,
 * and loaded by Load_Cuboid_Binaries, section 5):
 *   bit tables file: for each prime in the caller's order, its r x r table u_r in the
 *     Eq. 2.6 byte layout (ceil(r^2 / 8) bytes: bit p~ r + q~, least significant bit
 *     first, last byte zero-padded), tables back to back;
 *   primes file: one 8-byte little-endian record per prime, the C struct
 *     {short prime; unsigned int offset;} -- int16 prime, 2 zero padding bytes, uint32
 *     byte offset of the prime's table in the bit tables file (Eq. 2.7 keeps the offsets
 *     below 2^32).
 * Export writes both files (overwriting them) and returns the bit tables' size in
 * *bytes_written.  Host-synchronous.  Errors: ENOTABLES; EINVAL (NULL path, file not
 * writable); ERANGE (a prime above 32767 or offsets past 2^32). */
int cuboid_tables_export(const cuboid_tables* t, const char* bit_tables_path, const char* primes_path,
                         uint64_t* bytes_written);

/* Build tables from the two files: the file's bits become the device tables as they are
 * (the reduced table v_r is read from them, v_r(k) = u_r(k, 1)), in the order given by
 * flags (CUBOID_ORDER_*).  With CUBOID_IMPORT_CHECK every table is also compared with a
 * table built from the definition, and a difference gives CUBOID_EVERIFY.  *bytes_loaded
 * receives the primes file's size (the value the paper's loader returns).  cuboid_tables_info
 * reports CUBOID_TABLES_IMPORTED among the flags.  Synchronous on stream.  Errors: EINVAL
 * (unreadable file, primes file not a whole number of records, a record's prime not a
 * prime in [2, 9697), repeated, or a table's padding bits not zero); ERANGE (a table past
 * the end of the bit tables file); those of cuboid_tables_build; EVERIFY. */
int cuboid_tables_import(const char* bit_tables_path, const char* primes_path, uint32_t flags, void* stream,
                         cuboid_tables** out, uint64_t* bytes_loaded);

/* Set / read the kernel shape used by later sieve calls on these tables. */
int cuboid_tables_set_tuning(cuboid_tables* t, const cuboid_tuning* tune);
int cuboid_tables_get_tuning(const cuboid_tables* t, cuboid_tuning* tune);

/* Autotuner: time kernel shapes (hot primes, tiles per warp, threads per CTA, CTAs per
 * SM, primes in shared memory, lanes per row) by coordinate descent on these very ranges (host array,
 * n >= 1, mode CUBOID_MODE_PLAIN or CUBOID_MODE_BATCHED), set the fastest on the tables
 * and return it with its time in milliseconds (either pointer may be NULL).  Every
 * candidate must give the same counts, pair totals and survivor/root totals; otherwise
 * the tables keep their previous shape and EVERIFY is returned.  cache_path (may be
 * NULL): a text file of earlier results keyed by device name, prime list, ranges and
 * mode; a hit skips the search, a new result is appended.  Synchronous on stream. */
int cuboid_autotune(cuboid_tables* t, const cuboid_range* ranges, uint32_t n, uint32_t mode, void* stream,
                    const char* cache_path, cuboid_tuning* best, float* best_ms);

/* Free the tables.  Returns EBUSY (and frees nothing) while a server uses them, like
 * the paper's Release call that refuses while a search runs (section 5). */
int cuboid_tables_free(cuboid_tables* t);

/* ================================================================ sieving (sections 2, 5) */

/* Allocate a reusable result object for up to max_ranges ranges, surv_cap survivor
 * records and root_cap root records (0 = defaults 2^20 and 2^16). */
int cuboid_result_create(const cuboid_tables* t, uint32_t max_ranges, uint64_t surv_cap,
                         uint64_t root_cap, cuboid_result** out);

/* Sieve one range: every coprime pair p != q with p_lo <= p <= p_hi, q_lo <= q <= q_hi
 * (and the flags' restrictions) goes through the bit sieve of section 2 in the
 * effective order; survivors get the exact integer-root test of Q_pq.  Creates *out
 * (default capacities) and enqueues the work and the copies back on stream; call
 * cuboid_result_wait before cuboid_result_get.  Errors: ENOTABLES, ERANGE, ENOMEM. */
int cuboid_sieve(const cuboid_tables* t, uint32_t p_lo, uint32_t p_hi, uint32_t q_lo,
                 uint32_t q_hi, uint32_t flags, void* stream, cuboid_result** out);

/* Sieve n ranges (host array) in one persistent launch with a device work queue,
 * replayed from a captured CUDA graph.  Creates *out with max_ranges = n. */
int cuboid_sieve_batch(const cuboid_tables* t, const cuboid_range* ranges, uint32_t n,
                       void* stream, cuboid_result** out);

/* Reuse an existing result: copy n host ranges in (n <= max_ranges), run them with
 * mode CUBOID_MODE_PLAIN (one launch sequence per range) or CUBOID_MODE_BATCHED (one
 * persistent launch), optionally | CUBOID_MODE_COUNT_STEPS, and enqueue the copies
 * back.  The previous use of res must have been waited for.  Errors: ERANGE (a bad
 * range; nothing is launched), EINVAL. */
int cuboid_sieve_into(cuboid_result* res, const cuboid_range* ranges, uint32_t n,
                      uint32_t mode, void* stream);

/* As cuboid_sieve_into with device-resident ranges (a device pointer to n ranges) and
 * no copy back: results stay on the device until cuboid_result_download.  Invalid
 * ranges are skipped on the device and reported by cuboid_result_wait as ERANGE.
 * CUBOID_MODE_BATCHED copies the ranges in stream order; the plain mode reads them where
 * they are, so they must stay valid and unchanged until the work on stream completes. */
int cuboid_sieve_device(cuboid_result* res, const cuboid_range* ranges_dev, uint32_t n,
                        uint32_t mode, void* stream);

/* Enqueue the copy of counts, pair totals and record counts to pinned host memory. */
int cuboid_result_download(cuboid_result* res, void* stream);

/* Wait for the last enqueued work of res, fetch survivor and root records and sort
 * them.  Returns CUBOID_OK, or EOVERFLOW (a record buffer was too small: counts and
 * pair totals are still exact), ERANGE (a device-side range was invalid), EVERIFY, or
 * ETIMEOUT (a CTA's bulk staging of the tables into shared memory did not complete within
 * its bounded wait; the results are then incomplete). */
int cuboid_result_wait(cuboid_result* res);

/* Results of range range_idx (valid after cuboid_result_wait):
 *   n_pairs:  coprime pairs sieved (= sum of counts + n_surv);
 *   counts:   n_primes entries, caller order (may be NULL);
 *   surv:     n_surv records (p << 32 | q), ascending; owned by res;
 *   roots:    n_roots records, ascending by (p, q, t); owned by res.
 * Any output pointer may be NULL. */
int cuboid_result_get(const cuboid_result* res, uint32_t range_idx, uint64_t* n_pairs,
                      uint64_t* counts, uint64_t* n_surv, const uint64_t** surv,
                      uint64_t* n_roots, const cuboid_root** roots);

/* Device time of the sieve kernel launches of the last CUBOID_MODE_TIME_SIEVE run, in
 * milliseconds (summed over launches), and the number of those launches (after
 * cuboid_result_wait).  EINVAL if the last run was not timed. */
int cuboid_result_sieve_ms(const cuboid_result* res, float* ms, uint32_t* launches);

/* Step counters of the last CUBOID_MODE_COUNT_STEPS run (after cuboid_result_wait). */
int cuboid_result_stats(const cuboid_result* res, cuboid_stats* out);

int cuboid_result_free(cuboid_result* res);

/* ================================================================ no-allocation sieve */

/* Largest number of ranges one cuboid_sieve_noalloc call accepts. */
#define CUBOID_NOALLOC_MAX_RANGES 4096

/* The batched sieve (all n ranges in one persistent launch, then the exact root test of
 * the survivors) for callers that may not allocate device memory when they sieve: a
 * loop with a latency budget (cudaMalloc and cudaFree synchronise the device), a host
 * that only lends the library a fixed pool, or a process at its memory limit.  This call allocates nothing and calls no
 * allocating routine.  Its working memory (tile plans and the tile-queue/counter header,
 * 4096 x 32 bytes + 256 bytes) is one static array of device memory that every GPU that
 * loads the library holds until the process exits.  No paper counterpart: the paper
 * runs one CPU thread with host memory.
 *
 *   t:              tables built beforehand (cuboid_tables_build allocates; do it at set-up).
 *   ranges_dev:     device pointer to n ranges, 1 <= n <= CUBOID_NOALLOC_MAX_RANGES.
 *   counts_dev:     device, n * n_primes uint64, written (zeroed first); counts_dev[k * n_primes + e]
 *                   is the count of the e-th prime of the EFFECTIVE order (cuboid_tables_order).
 *   npairs_dev:     device, n uint64: pairs sieved per range.
 *   surv_dev, surv_range_dev, surv_cap: device survivor records (p << 32 | q, unsorted) and
 *                   their range index; records beyond surv_cap are dropped (counts stay exact).
 *   roots_dev, root_range_dev, root_cap: device root records (unsorted) and range indices.
 *   totals_dev:     device, 3 uint64: number of survivors, number of roots (both may exceed
 *                   the capacities), and the device status bits (0 = clean; 1 survivor
 *                   overflow, 2 root overflow, 4 invalid range, 8 root test unsettled,
 *                   16 a CTA's bulk staging of the tables did not complete in time).
 *   stream:         everything is enqueued on it; the call returns without waiting.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents (each call clears what must start at zero), so calls
 * whose work overlaps on the GPU (other streams, other host threads) race: serialise them.
 * Errors: ENOTABLES, ETOOLARGE (n > CUBOID_NOALLOC_MAX_RANGES, nothing enqueued), EINVAL,
 * ECUDA. */
int cuboid_sieve_noalloc(const cuboid_tables* t, const cuboid_range* ranges_dev, uint32_t n,
                         uint64_t* counts_dev, uint64_t* npairs_dev, uint64_t* surv_dev,
                         uint32_t* surv_range_dev, uint64_t surv_cap, cuboid_root* roots_dev,
                         uint32_t* root_range_dev, uint64_t root_cap, uint64_t* totals_dev,
                         void* stream);

/* ================================================================ region search (section 5) */

/* The region of Theorem 1.2 (Eq. 1.2): min(cbrt(p/9), p/59) <= q <= 59 p; for p >= 152
 * it is the segment of Eq. 5.2, cbrt(p/9) <= q <= 59 p.  A scan walks the rows p upward,
 * each row over its segment, sieving coprime q != p, in batches aligned to hundreds of p:
 * 100 rows for the asynchronous search (the granularity of the paper's Get_current_p),
 * up to 2000 rows, two batches in flight, for the synchronous scan. */
typedef struct cuboid_search_report {
  uint32_t p, q;      /* where a resumed scan starts: the next row and its first q */
  uint32_t r_max;     /* deepest prime needed (last rejecting prime in the effective order
                         over the scanned rows; every prime if a pair survived); 0 if none */
  uint32_t depth;     /* its 1-based position in the effective order */
  uint64_t pairs;     /* coprime pairs sieved */
  uint64_t n_surv;    /* pairs that passed every prime */
  uint64_t n_roots;   /* integer roots found on them */
} cuboid_search_report;

/* Smallest q of row p in the region of Eq. 1.2 (>= 1). */
uint32_t cuboid_region_qmin(uint32_t p);

/* Synchronous scan of rows p_from..p_to (row p_from from q_from on; q_from = 0: its
 * segment start).  counts (n_primes, caller order, may be NULL) receives the per-prime
 * first-rejecter counts, surv / roots (capacities surv_cap / root_cap, may be NULL with
 * cap 0) the survivor and root records in scan order, rep the report.  Any p_from >= 1
 * is accepted (rows below 152 use the min() of Eq. 1.2).  Synchronous on stream.
 * Errors: ENOTABLES; ERANGE if p_from = 0 or p_to < p_from; EPMAX if p_to > 72796055;
 * EQLOW / EQHIGH if q_from (when nonzero) lies outside row p_from's segment; EOVERFLOW if
 * more survivors or roots arrived than a buffer holds (the per-prime counts and the pair
 * and survivor totals stay exact; records and roots past a capacity are dropped). */
int cuboid_region_scan(cuboid_tables* t, uint32_t p_from, uint32_t q_from, uint32_t p_to, void* stream,
                       uint64_t* counts, uint64_t* surv, uint64_t surv_cap, cuboid_root* roots,
                       uint64_t root_cap, cuboid_search_report* rep);

typedef struct cuboid_search cuboid_search;

/* Start an open-ended scan at row p, column q on a host thread and return at once
 * (the paper's Start_searching, section 5).  Codes as the paper's: 0 started;
 * CUBOID_EBUSY (1) a search already runs on these tables; CUBOID_ERANGE (2) p < 152;
 * CUBOID_EPMAX (3) p > 72796055; CUBOID_EQLOW (4) q below the segment of Eq. 5.2;
 * CUBOID_EQHIGH (5) q > 59 p; CUBOID_ENOTABLES (6) no tables.  The tables stay in use
 * (cuboid_tables_free returns EBUSY) until cuboid_search_stop. */
int cuboid_search_start(cuboid_tables* t, uint32_t p, uint32_t q, cuboid_search** out);

/* Progress (the paper's Get_current_p and Get_current_r_max): the first row of the
 * batch of 100 rows being scanned, and the deepest prime needed within it. */
int cuboid_search_current(const cuboid_search* s, uint32_t* p, uint32_t* r_max);

/* Stop after the batch in flight (the paper's Stop_searching), fill the report (p, q of
 * the next row: pass them to cuboid_search_start to resume), the totals and counts
 * (n_primes, caller order, may be NULL), and free the handle.  Survivor and root records
 * are not kept by a search (their numbers are in the report; cuboid_region_scan returns
 * records).  Returns the first error the scan met, else 0; EINVAL (NULL handle). */
int cuboid_search_stop(cuboid_search* s, cuboid_search_report* rep, uint64_t* counts);

/* Append the report to a text file in the paper's form (section 5): a local time stamp
 * line "Y-M-D HH:MM" and "Stop with p=<p>, q=<q>, r_max=<r_max>".  Host only.
 * Errors: EINVAL (NULL argument, file not writable). */
int cuboid_search_report_write(const cuboid_search_report* rep, const char* path);

/* ================================================================ Theorem 1.1 */

/* For each root (p, q, t), flags[i] = 1 when t satisfies the inequalities of Theorem 1.1,
 * t > p^2, t > p q, t > q^2 and (p^2 + t)(p q + t) > 2 t^2 -- for a coprime p != q such a
 * root is a perfect cuboid -- else 0 (t = 0 gives 0).  Exact in 256-bit integers.  Host
 * only; roots and flags are host arrays of n entries.  Errors: EINVAL (NULL with n > 0). */
int cuboid_theorem11_flags(const cuboid_root* roots, uint64_t n, uint8_t* flags);

/* ================================================================ sharding */

/* Shard i of k (0 <= i < k) of range r for k GPUs or processes: contiguous blocks of rows
 * holding about 1/k of the range's lattice points each (rows of p for CUBOID_Q_LT_P
 * triangles; rows of the longer side for rectangles).  The shards partition the range:
 * their sieve results add up (counts, pair totals) and concatenate (survivors, roots) to
 * the whole range's.  *out gets the shard (p_lo > p_hi or q_lo > q_hi when it is empty);
 * *points (may be NULL) its lattice-point count before coprimality.  Host only, no CUDA
 * call.  Errors: EINVAL (NULL, k = 0, i >= k), ERANGE (invalid r). */
int cuboid_shard_range(const cuboid_range* r, uint32_t k, uint32_t i, cuboid_range* out, uint64_t* points);

/* ================================================================ exact root test */

/* Run the exact integer-root test on n arbitrary (p, q) pairs (host arrays, p, q >= 1),
 * whatever the sieve says.  roots_out (capacity cap) receives the roots ascending;
 * *n_roots their number.  Synchronous on stream.  Errors: EINVAL, EOVERFLOW, EVERIFY. */
int cuboid_verify_pairs(const uint32_t* p, const uint32_t* q, uint32_t n, void* stream,
                        cuboid_root* roots_out, uint64_t cap, uint64_t* n_roots);

/* ================================================================ 64-bit ranges */

/* Section 6 puts the limit of the paper's 32-bit code at p_max = 2^32 / 59 (72796055):
 * beyond it the top of the region of Eq. 1.2, q = 59 p, leaves 32 bits.  The calls below
 * take p and q as 64-bit integers below CUBOID_WIDE_LIMIT = 2^40, which holds the region
 * of Eq. 1.2 for every p < 2^32 (59 p < 2^38).  One coordinate, the one whose values index
 * the rows of the sieve's tiles, must stay below 2^32 (coprimality with the other
 * coordinate is decided from its factorisation): rows of p when p_hi < 2^32, else rows of
 * q when q_hi < 2^32 (CUBOID_ROWS_P / CUBOID_ROWS_Q force one; with neither flag and both
 * below 2^32 the range is a 32-bit range, oriented as in cuboid_sieve).  The other
 * coordinate ("y") is cut into pieces: the values below 2^32 form one piece, sieved as a
 * 32-bit range; above 2^32 each piece holds at most 2^32 - 64 values and is sieved
 * relative to a 64-bit base (a multiple of 64), whose residues modulo the table primes and
 * the row's prime factors offset those of the relative values.  A piece above 2^32 lies
 * above every row value, so a CUBOID_Q_LT_P range keeps all of it (rows of q) or none of it
 * (rows of p), and it holds no diagonal pair.  Results are per range, as for 32-bit
 * ranges. */
#define CUBOID_WIDE_LIMIT (1ull << 40)

/* A 64-bit rectangle; flags as for cuboid_range; reserved must be 0.  40 bytes. */
typedef struct cuboid_range_wide {
  uint64_t p_lo, p_hi, q_lo, q_hi;
  uint32_t flags;
  uint32_t reserved;
} cuboid_range_wide;

/* An integer root t > 0 of Q_pq with 64-bit p, q (t = t_hi * 2^64 + t_lo). */
typedef struct cuboid_root_wide {
  uint64_t p, q;
  uint64_t t_lo, t_hi;
} cuboid_root_wide;

/* The pieces of one wide range, as sieved: pieces[i] holds the piece in coordinates
 * relative to bases[2 i] (added to p) and bases[2 i + 1] (added to q), with CUBOID_ROWS_P
 * or CUBOID_ROWS_Q set; a piece that the CUBOID_Q_LT_P restriction leaves empty is not
 * listed.  cap is the capacity of pieces (and of bases, in pairs); *n gets the number of
 * pieces even when it exceeds cap (then EOVERFLOW and nothing else is written).  Host
 * only, no CUDA call.  Errors: EINVAL (NULL, bad flags or reserved), ERANGE (a bound 0
 * or >= 2^40, lo > hi, or no coordinate below 2^32 to index the rows), EOVERFLOW. */
int cuboid_wide_pieces(const cuboid_range_wide* r, cuboid_range* pieces, uint64_t* bases, uint32_t cap,
                       uint32_t* n);

/* Sieve n wide ranges (host array): for each piece one plan and one sieve launch, then one
 * root test for all survivors, enqueued on stream with the copies back; creates *out
 * (default record capacities).  Wait with cuboid_result_wait and read with
 * cuboid_result_get_wide (cuboid_result_get refuses such a result: its internal ranges are
 * the pieces).  Errors: ENOTABLES, EINVAL, ERANGE (as cuboid_wide_pieces), ENOMEM. */
int cuboid_sieve_wide(const cuboid_tables* t, const cuboid_range_wide* ranges, uint32_t n, void* stream,
                      cuboid_result** out);

/* Results of wide range range_idx (valid after cuboid_result_wait): n_pairs and counts as
 * for cuboid_result_get; surv: 2 n_surv values p0, q0, p1, q1, ... ascending by (p, q);
 * roots ascending by (p, q, t).  Arrays are owned by res; any output may be NULL.
 * Errors: EINVAL (not waited for, not a wide result, range_idx out of range). */
int cuboid_result_get_wide(const cuboid_result* res, uint32_t range_idx, uint64_t* n_pairs,
                           uint64_t* counts, uint64_t* n_surv, const uint64_t** surv, uint64_t* n_roots,
                           const cuboid_root_wide** roots);

/* The exact integer-root test on n arbitrary 64-bit pairs (host arrays, 1 <= p, q < 2^40),
 * as cuboid_verify_pairs.  Errors: EINVAL, ERANGE, EOVERFLOW, EVERIFY. */
int cuboid_verify_pairs_wide(const uint64_t* p, const uint64_t* q, uint32_t n, void* stream,
                             cuboid_root_wide* roots_out, uint64_t cap, uint64_t* n_roots);

/* Theorem 1.1 flags for wide roots (p, q < 2^40), as cuboid_theorem11_flags.
 * Errors: EINVAL, ERANGE. */
int cuboid_theorem11_flags_wide(const cuboid_root_wide* roots, uint64_t n, uint8_t* flags);

/* Report of a region scan with 64-bit q (fields as cuboid_search_report). */
typedef struct cuboid_region_report_wide {
  uint64_t p, q;      /* where a resumed scan starts: the next row and its first q (0 past 2^32 - 1) */
  uint32_t r_max;     /* deepest prime needed; 0 if none */
  uint32_t depth;     /* its 1-based position in the effective order */
  uint64_t pairs;     /* coprime pairs sieved */
  uint64_t n_surv;    /* pairs that passed every prime */
  uint64_t n_roots;   /* integer roots found on them */
} cuboid_region_report_wide;

/* The synchronous region scan of cuboid_region_scan continued past the paper's p_max
 * (section 6): rows p_from..p_to of Eq. 1.2 for 1 <= p_from <= p_to < 2^32, row p_from from
 * q_from on (0: its segment start), every q up to 59 p (which leaves 32 bits for p >
 * 72796055), sieved as 64-bit ranges with rows of p.  counts: n_primes, caller order (may
 * be NULL); surv: 2 surv_cap values p0, q0, p1, q1, ... in scan order; roots: root_cap
 * records; rep: the report.  Synchronous on stream.  Errors: ENOTABLES; ERANGE (p_from = 0,
 * p_to < p_from, p_to >= 2^32); EQLOW / EQHIGH (q_from outside row p_from's segment);
 * EOVERFLOW (records past a capacity dropped; counts and totals exact). */
int cuboid_region_scan_wide(cuboid_tables* t, uint64_t p_from, uint64_t q_from, uint64_t p_to, void* stream,
                            uint64_t* counts, uint64_t* surv, uint64_t surv_cap, cuboid_root_wide* roots,
                            uint64_t root_cap, cuboid_region_report_wide* rep);

/* ================================================================ serving */

/* A request loop that admits range queries while others run (continuous batching):
 * queries are admitted while slots and device memory allow, grouped by an admission
 * thread into persistent-kernel batches on several streams, and polled by ticket.
 *   mem_budget: device bytes the server may hold (0 = 1 GiB); max_slots: queries in
 *   flight (0 = 4096).  The tables stay in use (cuboid_tables_free returns EBUSY) until
 *   cuboid_server_destroy. */
int cuboid_server_create(cuboid_tables* t, uint64_t mem_budget, uint32_t max_slots,
                         cuboid_server** out);

/* Submit one range.  *ticket identifies it.  EBUSY if no slot or memory is free right
 * now (admission refused; retry later); ERANGE for a bad range. */
int cuboid_server_submit(cuboid_server* s, const cuboid_range* range, uint64_t* ticket);

/* Poll a ticket.  EAGAIN while running; CUBOID_OK with *out = a result holding one
 * range (free it with cuboid_result_free); EINVAL for an unknown ticket. */
int cuboid_server_poll(cuboid_server* s, uint64_t ticket, cuboid_result** out);

/* Queue depth, queries admitted/refused/finished, batches launched, and queries run again
 * alone because their survivor or root records did not all fit in a shared batch
 * (NULL-safe).  A query that still overflows alone finishes with EOVERFLOW (exact counts);
 * the other queries of its first batch are not affected. */
int cuboid_server_stats(const cuboid_server* s, uint64_t* in_flight, uint64_t* admitted,
                        uint64_t* refused, uint64_t* finished, uint64_t* batches, uint64_t* retried);

/* Load replay (measurement of the request loop without a host language in the way):
 * submits queries[i] at arrival_s[i] seconds after the call starts (non-decreasing; a
 * refused submission is retried every 20 us and counted in *refused), then waits until all
 * have finished.  Per query: tickets[i] (its result stays available to cuboid_server_poll),
 * latency_s[i] from its admission to its result being on the host, npairs[i], status[i].
 * *wall_s: from the call's start to the last result.  All of it within timeout_ms
 * (ETIMEOUT otherwise; queries already admitted keep running).  Runs on the calling
 * thread.  Errors: EINVAL, ERANGE (a bad query: the replay stops there), ETIMEOUT. */
int cuboid_server_replay(cuboid_server* s, const cuboid_range* queries, const double* arrival_s, uint32_t n,
                         uint32_t timeout_ms, uint64_t* tickets, double* latency_s, uint64_t* npairs,
                         int32_t* status, double* wall_s, uint64_t* refused);

/* Stop the loop (waits for work in flight, at most timeout_ms; ETIMEOUT otherwise). */
int cuboid_server_destroy(cuboid_server* s, uint32_t timeout_ms);

/* ================================================================ measurement */

/* Integer-issue probe: launch `blocks` CTAs of `threads` threads, each thread running
 * `iters` iterations of 16 independent 32-bit integer ops (kind 0: add/shift/xor mix,
 * kind 1: the sieve's lookup mix with shared-memory loads; kinds 2-7 one instruction per
 * chain step: 2 lop3, 3 funnel shift, 4 popc followed by one mad.lo, 5 mad.lo, 6 mad.wide
 * (32 x 32 + 64 bits), 7 mad.hi, 8 the add-then-minimum min(a + b, c) of __viaddmin_u32,
 * which the sieve's residue steps use).  Kind > 8: EINVAL.  sink_dev: device buffer of blocks*threads uint32
 * (defeats dead-code elimination).  Asynchronous. */
int cuboid_probe_int_issue(uint32_t kind, uint32_t blocks, uint32_t threads, uint32_t iters,
                           uint32_t* sink_dev, void* stream);

/* Test probes of the arithmetic helpers (no paper counterpart; they check the library's
 * own residue and modular routines against exact references).
 *
 * cuboid_probe_mod_min: for each modulus mods[i] (2 <= mods[i], n <= 65535) the sieve's
 * residue routine (one mul.hi by floor(2^32 / r), one multiply-subtract and an unsigned
 * minimum) is compared with the % operator on the GPU for every 32-bit n; mismatches[i]
 * receives the number of n where they differ.  Host arrays; synchronous on stream.
 *
 * cuboid_probe_modarith: the root test's 62-bit arithmetic on the host (device = 0, the
 * same routines compiled for the host) or on the GPU (device = 1), over host arrays:
 * op 0: out[i] = a[i] b[i] mod m_j (Montgomery products); op 1: out[i] = a[i] mod m_j;
 * op 2: out[i] = sign of the integer X, |X| < (m_0 ... m_{j-1} - 1) / 2, with residues
 * a[i j + k] = X mod m_k (Garner), as 0, 1 or 2^64 - 1; op 3: out[k] = m_k, k < 14 (the
 * moduli: the 14 largest primes below 2^62).  Errors: EINVAL, ECUDA. */
int cuboid_probe_mod_min(const uint32_t* mods, uint32_t n, uint64_t* mismatches, void* stream);
int cuboid_probe_modarith(uint32_t op, uint32_t j, const uint64_t* a, const uint64_t* b, uint32_t n,
                          uint64_t* out, int device);

/* Number of SMs of the current device and the library version string. */
int cuboid_device_sms(uint32_t* sms);
const char* cuboid_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CUBOID_H */
