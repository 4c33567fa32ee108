/* The paper's search loop on the host CPU -- TEST INFRASTRUCTURE AND CPU BASELINE ONLY.
 *
 * Paper: Gallyamov, Kadyrov, Kashelevskiy, Kutlugallyamov, Sharipov, "A fast modulo
 * primes algorithm for searching perfect cuboids and its implementation"
 * (arXiv:1601.00636).
 *
 * What it is: the nested loop of section 5 written in plain C with OpenMP -- for every
 * pair (p, q) of a range, the primes are tried in the given order and the first prime
 * whose unsolvability bit u_r(p mod r, q mod r) is 1 rejects the pair -- over tables in
 * the byte layout of Eq. 2.6 (r x r bits, row-major index p~ r + q~, least significant bit
 * first), with 32-bit residues taken by the % operator, one row p per OpenMP work item.
 * It is the timed CPU baseline of the benchmark and is checked against the Python oracle
 * (oracle/cuboid_oracle.py) in the tests; it shares no code with the CUDA library, and
 * only the tests and the benchmark's CPU legs load it.
 *
 * Readings (the same as the oracle's): only coprime pairs p != q are sieved and counted
 * (Conjecture 1.1; the paper's loop scans every q); bounds are inclusive; flag 1 keeps
 * q < p.  The tables are built here by Definition 1.1 (section 2) at the pairs (k, 1),
 * v_r(k) = 1 iff no t in [0, r) solves Q_{k,1}(t) = 0 mod r, and expanded by the weighted
 * homogeneity of Eq. 1.1 (u_r(a, b) = v_r(a b^-1 mod r) for b != 0, u_r(a, 0) = 0); the
 * tests compare the packed bytes with the oracle's brute-force tables and with the bytes
 * printed as Eq. 2.6.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define PL_MAX_PRIMES 4096

typedef struct {
  uint32_t n;
  uint32_t r[PL_MAX_PRIMES];
  uint8_t* bits[PL_MAX_PRIMES]; /* Eq. 2.6 bytes of u_r, ceil(r^2 / 8) each */
} pl_tables;

/* Q_{k,1}(t) mod r (Eq. 1.1 with p = k, q = 1), every term reduced mod r < 2^16. */
static uint32_t q_k1_mod(uint64_t k, uint64_t t, uint64_t r) {
  const uint64_t p2 = k * k % r, p4 = p2 * p2 % r, p6 = p4 * p2 % r, p8 = p4 * p4 % r, p10 = p8 * p2 % r;
  const uint64_t t2 = t * t % r;
  /* coefficients of t^10 .. t^0 with q = 1, as non-negative residues */
  const uint64_t c8 = ((2 + p2) % r) * ((3 + 2 * r - 2 * p2) % r) % r;             /* (2+p^2)(3-2p^2) */
  const uint64_t c6 = (1 + 10 * p2 + 4 * p4 + 14 * (r - p6) + p8) % r;                  /* 1+10p^2+4p^4-14p^6+p^8 */
  const uint64_t in4 = (1 + 14 * (r - p2) + 4 * p4 + 10 * p6 + p8) % r;                 /* 1-14p^2+4p^4+10p^6+p^8 */
  const uint64_t c4 = (r - p2 * in4 % r) % r;                                           /* -p^2 (...) */
  const uint64_t c2 = (r - p6 * ((1 + 2 * p2) % r) % r * ((3 * p2 + 2 * r - 2) % r) % r) % r; /* -p^6(1+2p^2)(3p^2-2) */
  const uint64_t c0 = (r - p10) % r;                                                    /* -p^10 */
  uint64_t acc = 1;                                                                     /* Horner in t^2 */
  acc = (acc * t2 + c8) % r;
  acc = (acc * t2 + c6) % r;
  acc = (acc * t2 + c4) % r;
  acc = (acc * t2 + c2) % r;
  acc = (acc * t2 + c0) % r;
  return (uint32_t)acc;
}

static uint32_t pow_mod(uint64_t b, uint32_t e, uint64_t r) {
  uint64_t x = 1;
  b %= r;
  while (e) {
    if (e & 1) x = x * b % r;
    b = b * b % r;
    e >>= 1;
  }
  return (uint32_t)x;
}

/* Builds the packed tables of n primes (each 2 <= r < 65536).  Returns NULL on bad input
 * or when out of memory. */
pl_tables* pl_tables_build(const uint32_t* primes, uint32_t n) {
  if (!primes || n == 0 || n > PL_MAX_PRIMES) return NULL;
  pl_tables* T = (pl_tables*)calloc(1, sizeof(pl_tables));
  if (!T) return NULL;
  T->n = n;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t r = primes[i];
    T->r[i] = r;
    if (r < 2 || r >= 65536) {
      bad = 1;
      continue;
    }
    uint8_t* v = (uint8_t*)malloc(r);
    uint32_t* inv = (uint32_t*)malloc(sizeof(uint32_t) * r);
    T->bits[i] = (uint8_t*)calloc(((size_t)r * r + 7) / 8, 1);
    if (!v || !inv || !T->bits[i]) {
      bad = 1;
      free(v);
      free(inv);
      continue;
    }
    for (uint32_t k = 0; k < r; ++k) {  /* Definition 1.1 at (k, 1) */
      uint32_t solvable = 0;
      for (uint32_t t = 0; t < r && !solvable; ++t) solvable = q_k1_mod(k, t, r) == 0;
      v[k] = solvable ? 0 : 1;
    }
    inv[0] = 0;
    for (uint32_t b = 1; b < r; ++b) inv[b] = pow_mod(b, r - 2, r);
    for (uint32_t a = 0; a < r; ++a)
      for (uint32_t b = 1; b < r; ++b)
        if (v[(uint64_t)a * inv[b] % r]) {
          const uint64_t idx = (uint64_t)a * r + b;
          T->bits[i][idx >> 3] |= (uint8_t)(1u << (idx & 7));
        }
    free(v);
    free(inv);
  }
  if (bad) {
    for (uint32_t i = 0; i < n; ++i) free(T->bits[i]);
    free(T);
    return NULL;
  }
  return T;
}

void pl_tables_free(pl_tables* T) {
  if (!T) return;
  for (uint32_t i = 0; i < T->n; ++i) free(T->bits[i]);
  free(T);
}

/* The Eq. 2.6 bytes of the i-th prime's table (NULL if out of range). */
const uint8_t* pl_table_bytes(const pl_tables* T, uint32_t i) { return (T && i < T->n) ? T->bits[i] : NULL; }

/* Distinct prime factors of x (at most 9 for x < 2^32) by trial division. */
static uint32_t factors(uint32_t x, uint32_t* f) {
  uint32_t n = 0;
  for (uint32_t d = 2; (uint64_t)d * d <= x; d += (d == 2 ? 1 : 2))
    if (x % d == 0) {
      f[n++] = d;
      while (x % d == 0) x /= d;
    }
  if (x > 1) f[n++] = x;
  return n;
}

/* One range of a sieve call: inclusive bounds, flags 1 = q < p. */
typedef struct {
  uint32_t p_lo, p_hi, q_lo, q_hi, flags;
} pl_range;

/* Per-thread scratch of the row loop. */
typedef struct {
  uint32_t* pr;          /* (p mod r) r per prime, effective order */
  const uint8_t** tab;   /* tables, effective order */
  uint32_t* rr;          /* primes, effective order */
  uint8_t* shared;       /* q sharing a prime factor with p (or q = p), per row */
  size_t shared_cap;
} pl_scratch;

/* Row p of range R: every coprime q != p tries the primes in order; the first prime whose
 * bit is set takes the pair's count (cnt, effective order); survivors go to surv at slots
 * taken from *surv_pos.  Returns the pairs sieved, or -1 when out of memory. */
static int64_t sieve_row(const pl_range* R, uint32_t p, uint32_t n, pl_scratch* S, uint64_t* cnt,
                         uint64_t* n_surv, uint64_t* surv, uint32_t* surv_range, uint32_t range_idx,
                         uint64_t surv_cap, uint64_t* surv_pos) {
  uint32_t hi = R->q_hi;
  if ((R->flags & 1u) && (uint64_t)hi >= p) hi = p - 1;
  if (hi < R->q_lo) return 0;
  const uint32_t lo = R->q_lo;
  const size_t len = (size_t)hi - lo + 1;
  if (len > S->shared_cap) {
    free(S->shared);
    S->shared = (uint8_t*)malloc(len);
    S->shared_cap = S->shared ? len : 0;
    if (!S->shared) return -1;
  }
  uint8_t* shared = S->shared;
  memset(shared, 0, len);
  uint32_t f[10];
  const uint32_t nf = factors(p, f);
  for (uint32_t j = 0; j < nf; ++j) {
    const uint64_t first = ((uint64_t)lo + f[j] - 1) / f[j] * f[j];
    for (uint64_t m = first; m <= hi; m += f[j]) shared[m - lo] = 1;
  }
  if (p >= lo && p <= hi) shared[p - lo] = 1;  /* p != q */
  for (uint32_t e = 0; e < n; ++e) S->pr[e] = (p % S->rr[e]) * S->rr[e];
  int64_t pairs = 0;
  for (uint64_t q = lo; q <= hi; ++q) {
    if (shared[q - lo]) continue;
    ++pairs;
    uint32_t e = 0;
    for (; e < n; ++e) {  /* the first prime whose bit is set rejects the pair */
      const uint32_t idx = S->pr[e] + (uint32_t)q % S->rr[e];
      if ((S->tab[e][idx >> 3] >> (idx & 7)) & 1u) break;
    }
    if (e < n) {
      ++cnt[e];
    } else {
      ++*n_surv;
      if (surv) {
        uint64_t pos;
#pragma omp atomic capture
        pos = (*surv_pos)++;
        if (pos < surv_cap) {
          surv[pos] = ((uint64_t)p << 32) | q;
          if (surv_range) surv_range[pos] = range_idx;
        }
      }
    }
  }
  return pairs;
}

/* Sieves n_ranges ranges, trying the primes in the order order[0..n-1] (indices into the
 * build list); the rows of all ranges are the work items (largest row first within a
 * range).  counts[k * n + i] (build-list order) and n_pairs[k] are ADDED to; survivors
 * (p << 32 | q, unsorted) and their range index are written up to surv_cap, and *n_surv
 * is ADDED the number of them all.  threads <= 0: OpenMP's default.
 * Returns 0, or -1 on bad arguments, -2 when out of memory. */
int pl_sieve_many(const pl_tables* T, const uint32_t* order, const pl_range* ranges, uint32_t n_ranges,
                  uint64_t* counts, uint64_t* n_pairs, uint64_t* surv, uint32_t* surv_range, uint64_t surv_cap,
                  uint64_t* n_surv, int threads) {
  if (!T || !order || !ranges || !counts || !n_pairs || !n_surv) return -1;
  const uint32_t n = T->n;
  for (uint32_t i = 0; i < n; ++i)
    if (order[i] >= n) return -1;
  uint64_t* row_end = (uint64_t*)malloc(sizeof(uint64_t) * (n_ranges ? n_ranges : 1));
  if (!row_end) return -2;
  uint64_t rows = 0;
  for (uint32_t k = 0; k < n_ranges; ++k) {
    const pl_range* R = &ranges[k];
    if (R->p_lo == 0 || R->q_lo == 0 || R->p_lo > R->p_hi || R->q_lo > R->q_hi) {
      free(row_end);
      return -1;
    }
    rows += (uint64_t)R->p_hi - R->p_lo + 1;
    row_end[k] = rows;
  }
  int err = 0;
  uint64_t ns = 0, surv_pos = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
#pragma omp parallel reduction(+ : ns)
  {
    pl_scratch S = {0};
    S.pr = (uint32_t*)malloc(sizeof(uint32_t) * n);
    S.tab = (const uint8_t**)malloc(sizeof(void*) * n);
    S.rr = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t* my = (uint64_t*)calloc((size_t)n_ranges * n, sizeof(uint64_t));
    uint64_t* my_pairs = (uint64_t*)calloc(n_ranges ? n_ranges : 1, sizeof(uint64_t));
    const int ok = S.pr && S.tab && S.rr && my && my_pairs;
    if (!ok) {
#pragma omp atomic write
      err = -2;
    } else {
      for (uint32_t e = 0; e < n; ++e) {
        S.tab[e] = T->bits[order[e]];
        S.rr[e] = T->r[order[e]];
      }
    }
    /* every thread reaches the work-sharing loop (a thread without memory skips its rows) */
#pragma omp for schedule(dynamic, 1)
    for (int64_t it = 0; it < (int64_t)rows; ++it) {
      if (!ok) continue;
      uint32_t lo = 0, hi = n_ranges - 1;  /* the range holding work item it */
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (row_end[mid] > (uint64_t)it) hi = mid; else lo = mid + 1;
      }
      const pl_range* R = &ranges[lo];
      const uint64_t first = lo ? row_end[lo - 1] : 0;
      const uint32_t p = R->p_hi - (uint32_t)((uint64_t)it - first);  /* long rows first */
      const int64_t k = sieve_row(R, p, n, &S, my + (size_t)lo * n, &ns, surv, surv_range, lo, surv_cap,
                                  &surv_pos);
      if (k < 0) {
#pragma omp atomic write
        err = -2;
      } else {
        my_pairs[lo] += (uint64_t)k;
      }
    }
    if (ok) {
#pragma omp critical
      {
        for (uint32_t k = 0; k < n_ranges; ++k) {
          n_pairs[k] += my_pairs[k];
          for (uint32_t e = 0; e < n; ++e) counts[(size_t)k * n + order[e]] += my[(size_t)k * n + e];
        }
      }
    }
    free(S.pr);
    free(S.tab);
    free(S.rr);
    free(S.shared);
    free(my);
    free(my_pairs);
  }
  free(row_end);
  if (err) return err;
  *n_surv += ns;
  return 0;
}

/* One range (see pl_sieve_many): counts[n] and *n_pairs are ADDED to. */
int pl_sieve(const pl_tables* T, const uint32_t* order, uint32_t p_lo, uint32_t p_hi, uint32_t q_lo, uint32_t q_hi,
             uint32_t flags, uint64_t* counts, uint64_t* n_pairs, uint64_t* surv, uint64_t surv_cap,
             uint64_t* n_surv, int threads) {
  const pl_range R = {p_lo, p_hi, q_lo, q_hi, flags};
  return pl_sieve_many(T, order, &R, 1, counts, n_pairs, surv, NULL, surv_cap, n_surv, threads);
}

/* Threads OpenMP uses by default (the host's cores unless limited). */
int pl_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
