// K4: exact integer-root test of Q_pq(t) (Eq. 1.1) for the pairs that pass the sieve.
//
// Q is monic and even: Q(t) = R(t^2) with the monic quintic
//   R(u) = u^5 + c8 u^4 + c6 u^3 + c4 u^2 + c2 u + c0.
// An integer root t > 0 of Q is exactly a perfect square u = t^2 that is an integer root
// of R.  Every positive root of R is at most U = 45 M^4, M = max(p, q): with the bounds
// |c8| <= 9 M^4, |c6| <= 30 M^8, |c4| <= 30 M^12, |c2| <= 9 M^16, |c0| <= M^20, u > U
// makes every lower term smaller than u^5 / 5, so R(u) > 0.
//
// Exact arithmetic: R^(d)(u) for 0 <= u <= U is below 2^35 M^20 in absolute value, so
// its residues modulo K primes m_j in (2^61, 2^62) with 61 K >= 37 + 20 bitlen(M)
// determine it: all residues zero <=> the value is zero, and Garner's mixed-radix digits
// compared with those of (prod m_j - 1)/2 give its sign.  p and q are below 2^40 (64-bit
// ranges; 32-bit ones are a special case): U < 2^166 fits three 64-bit limbs and K <= 14.
//
// Isolation (exact, complete): the real roots of R^(4) (linear), R^(3), ..., R are
// bracketed level by level.  If every root of R^(d+1) in [0, U] lies in a unit cell
// [c, c+1] of a known list, R^(d) is strictly monotone between consecutive cells, so
// each gap holds at most one root, found by exact sign bisection over the integers; the
// cells of R^(d+1) are kept as cells of R^(d).  At d = 0 this finds every integer root u
// of R in [0, U] (exact zeros), and the perfect squares among them give the roots t.
// FP64 only proposes a narrow bracket around each sign change (to shorten the
// bisection); the bracket is used only if exact signs confirm it.
#include <algorithm>
#include <mutex>

#include "cuboid_internal.cuh"

namespace cuboid {

namespace {

typedef unsigned long long ull;
constexpr int kMaxMod = 14;  // 61 * 14 >= 37 + 20 * 40: M below 2^40
static_assert((37 + 20 * 40 + 60) / 61 == kMaxMod, "moduli for 40-bit pairs");
constexpr int kMaxCells = 24;
// Threads per CTA of the root test (two CTAs per SM).  The large helpers (context set-up,
// exact sign, FP64 proposal, bracket stretch) are kept out of line: inlined, the kernel's
// code outgrows the instruction cache and warps at different stages of different survivors
// stall on instruction fetch (bulk test of 318,963 survivors: 22.9 ms inlined with 64-thread
// CTAs, 13.6 ms out of line, 6.3 ms out of line with 256-thread CTAs).
constexpr int kVerifyThreads = 256;

struct ModConst {
  ull m, minv, r2, r3, r4, half;  // minv = -m^-1 mod 2^64; rk = 2^(64k) mod m; half = (m-1)/2
};
__constant__ ModConst c_mod[kMaxMod];
__constant__ ull c_ginv[kMaxMod][kMaxMod];  // Montgomery form of m_i^-1 mod m_j (i < j)

// ---------------------------------------------------------------- Montgomery arithmetic

// High 64 bits of a 64 x 64-bit product (the host build serves the host-side tests).
__host__ __device__ __forceinline__ ull mulhi64(ull a, ull b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (ull)(((unsigned __int128)a * b) >> 64);
#endif
}

// Montgomery product a b 2^-64 mod m for a, b < m < 2^62.
__host__ __device__ __forceinline__ ull mmul(ull a, ull b, const ModConst& M) {
  const ull lo = a * b, hi = mulhi64(a, b);
  const ull u = lo * M.minv;
  const ull uhi = mulhi64(u, M.m);
  const ull t = hi + uhi + (lo != 0ull);
  return t >= M.m ? t - M.m : t;
}
__host__ __device__ __forceinline__ ull madd(ull a, ull b, ull m) {
  const ull s = a + b;
  return s >= m ? s - m : s;
}
__host__ __device__ __forceinline__ ull msub(ull a, ull b, ull m) { return a >= b ? a - b : a + (m - b); }
// v mod m for any 64-bit v when 2^61 < m < 2^62 (v < 8 m).
__host__ __device__ __forceinline__ ull red64(ull v, ull m) {
  if (v >= 4 * m) v -= 4 * m;
  if (v >= 2 * m) v -= 2 * m;
  if (v >= m) v -= m;
  return v;
}
__host__ __device__ __forceinline__ ull tomont(ull x, const ModConst& M) { return mmul(red64(x, M.m), M.r2, M); }
__host__ __device__ __forceinline__ ull frommont(ull x, const ModConst& M) { return mmul(x, 1ull, M); }

// Sign of the integer X with |X| < (prod m_j - 1) / 2 whose residues modulo m_0..m_{K-1}
// are x[j] (Montgomery form; not all zero): Garner's mixed-radix digits v_j, compared
// with those of (prod m_j - 1) / 2 from the most significant digit down.  mod(j) gives
// the constants of m_j and ginv(i, j) m_i^-1 mod m_j in Montgomery form (on the device
// they read the constant bank directly, on the host the probe's arrays).
template <int KM, class ModF, class GinvF>
__host__ __device__ __forceinline__ int garner_sign(const ull* x, int K, ModF mod, GinvF ginv) {
  ull v[KM];
  v[0] = frommont(x[0], mod(0));
  for (int j = 1; j < K; ++j) {
    const ModConst M = mod(j);
    ull t = x[j];
    for (int i = 0; i < j; ++i) t = mmul(msub(t, tomont(v[i], M), M.m), ginv(i, j), M);
    v[j] = frommont(t, M);
  }
  for (int j = K - 1; j >= 0; --j) {
    const ull h = mod(j).half;
    if (v[j] != h) return v[j] > h ? -1 : 1;
  }
  return 1;
}
struct DevMod {
  __device__ const ModConst& operator()(int j) const { return c_mod[j]; }
};
struct DevGinv {
  __device__ ull operator()(int i, int j) const { return c_ginv[i][j]; }
};
struct HostMod {
  const ModConst* m;
  __host__ __device__ const ModConst& operator()(int j) const { return m[j]; }
};
struct HostGinv {
  const ull (*g)[kMaxMod];
  __host__ __device__ ull operator()(int i, int j) const { return g[i][j]; }
};

// ---------------------------------------------------------------- 192-bit unsigned

struct U192 {
  ull w[3];
};
__device__ __forceinline__ U192 u192(ull x) { return U192{{x, 0ull, 0ull}}; }
__device__ __forceinline__ int ucmp(const U192& a, const U192& b) {
  for (int i = 2; i >= 0; --i)
    if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
  return 0;
}
__device__ __forceinline__ U192 uadd(const U192& a, const U192& b) {
  U192 r;
  ull c = 0;
  for (int i = 0; i < 3; ++i) {
    const ull s = a.w[i] + b.w[i];
    const ull c1 = s < a.w[i];
    r.w[i] = s + c;
    c = c1 | (r.w[i] < s);
  }
  return r;
}
__device__ __forceinline__ U192 usub(const U192& a, const U192& b) {  // a >= b
  U192 r;
  ull br = 0;
  for (int i = 0; i < 3; ++i) {
    const ull d = a.w[i] - b.w[i];
    const ull b1 = a.w[i] < b.w[i];
    r.w[i] = d - br;
    br = b1 | (d < br);
  }
  return r;
}
__device__ __forceinline__ U192 ushr1(const U192& a) {
  return U192{{(a.w[0] >> 1) | (a.w[1] << 63), (a.w[1] >> 1) | (a.w[2] << 63), a.w[2] >> 1}};
}
__device__ __forceinline__ double utod(const U192& a) {
  return (double)a.w[2] * 0x1p128 + (double)a.w[1] * 0x1p64 + (double)a.w[0];
}
// floor(x) for 0 <= x < 2^190 as a U192.
__device__ U192 dtou(double x) {
  if (!(x > 0.0)) return u192(0);
  if (x < 0x1p64) return u192((ull)x);
  int e;
  const double f = frexp(x, &e);           // x = f 2^e, 0.5 <= f < 1, e > 64
  const ull mant = (ull)(f * 0x1p53);      // x = mant 2^(e-53), exact
  const int sh = e - 53;
  U192 r = u192(0);
  const int limb = sh / 64, bit = sh % 64;
  if (limb < 3) r.w[limb] = mant << bit;
  if (bit && limb + 1 < 3) r.w[limb + 1] = mant >> (64 - bit);
  return r;
}
// a b for a, b < 2^96 (the product fits 192 bits).
__device__ __forceinline__ U192 umul128(unsigned __int128 a, unsigned __int128 b) {
  const ull a0 = (ull)a, a1 = (ull)(a >> 64), b0 = (ull)b, b1 = (ull)(b >> 64);
  const unsigned __int128 l = (unsigned __int128)a0 * b0;
  const unsigned __int128 m1 = (unsigned __int128)a0 * b1, m2 = (unsigned __int128)a1 * b0;
  U192 r = U192{{(ull)l, (ull)(l >> 64), (ull)a1 * b1}};
  r = uadd(r, U192{{0ull, (ull)m1, (ull)(m1 >> 64)}});
  r = uadd(r, U192{{0ull, (ull)m2, (ull)(m2 >> 64)}});
  return r;
}
// u mod m in Montgomery form.
__device__ __forceinline__ ull umod_mont(const U192& u, const ModConst& M) {
  ull x = mmul(red64(u.w[0], M.m), M.r2, M);
  x = madd(x, mmul(red64(u.w[1], M.m), M.r3, M), M.m);
  x = madd(x, mmul(red64(u.w[2], M.m), M.r4, M), M.m);
  return x;
}

// ---------------------------------------------------------------- per-pair context

// Coefficient k of R^(d) (d <= k <= 5) sits at cidx(d, k) = 6 d + k (a plain row-major
// index; packing the 20 used entries tighter made the indexing cost more than it saved).
__host__ __device__ constexpr int cidx(int d, int k) { return d * 6 + k; }
constexpr int kCoef = 30;

// Moduli a survivor with max(p, q) of `bits` bits needs: 61 K >= 37 + 20 bits.
__host__ __device__ constexpr int moduli_for_bits(int bits) { return (37 + 20 * bits + 60) / 61; }

// Per-pair context for at most KM moduli (the root-test kernel is instantiated per KM, so
// its per-thread local memory is sized for the survivors of the launch, not for 2^40).
template <int KM>
struct Ctx {
  int K;
  ull co[KM][kCoef];  // Montgomery coefficient of u^(k-d) in R^(d), modulus j: co[j][cidx(d, k)]
  double dco[kCoef];  // FP64 version
};

// a_0..a_5 of R (Eq. 1.1 with u = t^2) modulo m, Montgomery form.
__device__ void r_coeffs_mod(ull p, ull q, const ModConst& M, ull a[6]) {
  const ull m = M.m;
  const ull pm = tomont(p, M), qm = tomont(q, M);  // p, q < 2^40 < 8 m
  const ull P = mmul(pm, pm, M), Q = mmul(qm, qm, M);
  auto k = [&](ull v) { return tomont(v, M); };
  const ull P2 = mmul(P, P, M), P3 = mmul(P2, P, M), P4 = mmul(P3, P, M), P5 = mmul(P4, P, M);
  const ull Q2 = mmul(Q, Q, M), Q3 = mmul(Q2, Q, M), Q4 = mmul(Q3, Q, M), Q5 = mmul(Q4, Q, M);
  // t^8: (2q^2 + p^2)(3q^2 - 2p^2)
  a[4] = mmul(madd(mmul(k(2), Q, M), P, m), msub(mmul(k(3), Q, M), mmul(k(2), P, M), m), M);
  // t^6: q^8 + 10 p^2 q^6 + 4 p^4 q^4 - 14 p^6 q^2 + p^8
  ull s = Q4;
  s = madd(s, mmul(k(10), mmul(P, Q3, M), M), m);
  s = madd(s, mmul(k(4), mmul(P2, Q2, M), M), m);
  s = msub(s, mmul(k(14), mmul(P3, Q, M), M), m);
  s = madd(s, P4, m);
  a[3] = s;
  // t^4: -p^2 q^2 (q^8 - 14 p^2 q^6 + 4 p^4 q^4 + 10 p^6 q^2 + p^8)
  s = Q4;
  s = msub(s, mmul(k(14), mmul(P, Q3, M), M), m);
  s = madd(s, mmul(k(4), mmul(P2, Q2, M), M), m);
  s = madd(s, mmul(k(10), mmul(P3, Q, M), M), m);
  s = madd(s, P4, m);
  a[2] = msub(0, mmul(mmul(P, Q, M), s, M), m);
  // t^2: -p^6 q^6 (q^2 + 2 p^2)(3 p^2 - 2 q^2)
  a[1] = msub(0, mmul(mmul(P3, Q3, M),
                      mmul(madd(Q, mmul(k(2), P, M), m), msub(mmul(k(3), P, M), mmul(k(2), Q, M), m), M), M),
              m);
  // t^0: -q^10 p^10
  a[0] = msub(0, mmul(Q5, P5, M), m);
  a[5] = k(1);
}

__device__ void r_coeffs_f64(double p, double q, double a[6]) {
  const double P = p * p, Q = q * q;
  const double P2 = P * P, P3 = P2 * P, P4 = P3 * P, Q2 = Q * Q, Q3 = Q2 * Q, Q4 = Q3 * Q;
  a[5] = 1.0;
  a[4] = (2 * Q + P) * (3 * Q - 2 * P);
  a[3] = Q4 + 10 * P * Q3 + 4 * P2 * Q2 - 14 * P3 * Q + P4;
  a[2] = -P * Q * (Q4 - 14 * P * Q3 + 4 * P2 * Q2 + 10 * P3 * Q + P4);
  a[1] = -P3 * Q3 * (Q + 2 * P) * (3 * P - 2 * Q);
  a[0] = -(Q4 * Q) * (P4 * P);
}

__device__ __forceinline__ double falling(int k, int d) {
  double f = 1;
  for (int i = 0; i < d; ++i) f *= (double)(k - i);
  return f;
}

// Returns false (and sets nothing) when the pair needs more than KM moduli.
template <int KM>
__device__ __noinline__ bool ctx_init(Ctx<KM>& C, ull p, ull q) {
  const ull M = p > q ? p : q;
  const int bits = 64 - __clzll((long long)M);
  const int K = moduli_for_bits(bits);
  if (K > KM) return false;
  C.K = K;
  for (int j = 0; j < K; ++j) {
    const ModConst Mc = c_mod[j];
    ull a[6];
    r_coeffs_mod(p, q, Mc, a);
    for (int d = 0; d < 5; ++d)
      for (int kk = d; kk <= 5; ++kk)
        C.co[j][cidx(d, kk)] = mmul(a[kk], tomont((ull)falling(kk, d), Mc), Mc);
  }
  double a[6];
  r_coeffs_f64((double)p, (double)q, a);
  for (int d = 0; d < 5; ++d)
    for (int kk = d; kk <= 5; ++kk) C.dco[cidx(d, kk)] = a[kk] * falling(kk, d);
  return true;
}

// Exact sign of R^(d)(u), 0 <= u <= U.
template <int KM>
__device__ __noinline__ int exact_sign(const Ctx<KM>& C, int d, const U192& u) {
  ull x[KM];
  bool allzero = true;
  for (int j = 0; j < C.K; ++j) {
    const ModConst M = c_mod[j];
    const ull um = umod_mont(u, M);
    ull acc = C.co[j][cidx(d, 5)];
    for (int kk = 4; kk >= d; --kk) acc = madd(mmul(acc, um, M), C.co[j][cidx(d, kk)], M.m);
    x[j] = acc;
    allzero &= (acc == 0);
  }
  if (allzero) return 0;
  return garner_sign<KM>(x, C.K, DevMod{}, DevGinv{});
}

template <int KM>
__device__ double fval(const Ctx<KM>& C, int d, double u) {
  double acc = C.dco[cidx(d, 5)];
  for (int kk = 4; kk >= d; --kk) acc = acc * u + C.dco[cidx(d, kk)];
  return acc;
}

template <int KM>
struct Isolator {
  const Ctx<KM>* C;
  U192 U;
  U192 cells[kMaxCells];
  int nc;
  U192 next[kMaxCells];
  int nn;
  U192 roots[5];
  int nroots;
  bool fail;

  __device__ void push_cell(const U192& c) {
    if (nn < kMaxCells) next[nn++] = c; else fail = true;
  }
  __device__ void zero_at(int d, const U192& z) {
    if (d > 0) {
      push_cell(z);
    } else {
      for (int i = 0; i < nroots; ++i)
        if (ucmp(roots[i], z) == 0) return;
      if (nroots < 5) roots[nroots++] = z; else fail = true;
    }
  }

  // FP64 proposal of the sign change of R^(d) inside [lo, hi] (sign sa at lo).
  // Bisection stops once the bracket is narrower than the exact step uses (the proposal
  // is widened by max(4, |g| 2^-36) before exact signs check it): width <= max(1, 2^-40 b).
  __device__ __noinline__ double guess(int d, const U192& lo, const U192& hi, int sa) {
    double a = utod(lo), b = utod(hi);
    for (int it = 0; it < 400; ++it) {
      const double m = 0.5 * (a + b);
      if (!(m > a && m < b) || b - a <= fmax(1.0, b * 0x1p-40)) break;
      const double f = fval(*C, d, m);
      if (f == 0.0) return m;
      if ((f < 0.0 ? -1 : 1) == sa) a = m; else b = m;
    }
    return 0.5 * (a + b);
  }

  __device__ __noinline__ void stretch(int d, const U192& a, const U192& b) {
    const int sa = exact_sign(*C, d, a);
    const int sb = ucmp(a, b) == 0 ? sa : exact_sign(*C, d, b);
    if (sa == 0) zero_at(d, a);
    if (sb == 0 && ucmp(a, b) != 0) zero_at(d, b);
    if (sa * sb >= 0) return;
    U192 lo = a, hi = b;
    // FP64-proposed bracket, kept only if exact signs confirm it
    const double g = guess(d, lo, hi, sa);
    const double delta = fmax(4.0, fabs(g) * 0x1p-36);
    U192 glo = dtou(fmax(g - delta, 0.0)), ghi = dtou(g + delta);
    if (ucmp(glo, lo) < 0) glo = lo;
    if (ucmp(ghi, hi) > 0) ghi = hi;
    if (ucmp(glo, ghi) < 0) {
      const int s1 = exact_sign(*C, d, glo);
      if (s1 == 0) {
        zero_at(d, glo);
        return;
      }
      const int s2 = exact_sign(*C, d, ghi);
      if (s2 == 0) {
        zero_at(d, ghi);
        return;
      }
      if (s1 == sa && s2 == sb) {
        lo = glo;
        hi = ghi;
      } else if (s1 == sb) {
        hi = glo;
      } else if (s2 == sa) {
        lo = ghi;
      }
    }
    const U192 one = u192(1);
    while (ucmp(usub(hi, lo), one) > 0) {
      const U192 mid = ushr1(uadd(lo, hi));
      const int sm = exact_sign(*C, d, mid);
      if (sm == 0) {
        zero_at(d, mid);
        return;
      }
      if (sm == sa) lo = mid; else hi = mid;
    }
    if (d > 0) push_cell(lo);  // the root lies in (lo, lo + 1)
  }

  __device__ void run() {
    nc = 0;
    nroots = 0;
    fail = false;
    const U192 one = u192(1);
    for (int d = 4; d >= 0 && !fail; --d) {
      nn = 0;
      for (int i = 0; i < nc; ++i) push_cell(cells[i]);
      U192 a = u192(0);
      bool done = false;
      for (int ci = 0; ci <= nc && !done; ++ci) {
        U192 b = ci < nc ? cells[ci] : U;
        if (ucmp(b, U) > 0) b = U;
        if (ucmp(a, b) <= 0) stretch(d, a, b);
        if (ci < nc) {
          a = uadd(cells[ci], one);
          if (ucmp(a, U) > 0) done = true;
        }
      }
      // sort + dedupe the cells of R^(d)
      for (int i = 1; i < nn; ++i) {
        U192 v = next[i];
        int j = i - 1;
        while (j >= 0 && ucmp(next[j], v) > 0) {
          next[j + 1] = next[j];
          --j;
        }
        next[j + 1] = v;
      }
      nc = 0;
      for (int i = 0; i < nn; ++i)
        if (nc == 0 || ucmp(cells[nc - 1], next[i]) != 0) cells[nc++] = next[i];
    }
  }
};

// floor(sqrt(u)) for u < 2^168, as a 128-bit integer.
__device__ unsigned __int128 isqrt192(const U192& u) {
  unsigned __int128 r = 0;
  for (int bit = 83; bit >= 0; --bit) {
    const unsigned __int128 c = r | ((unsigned __int128)1 << bit);
    // c^2 as U192
    const ull c0 = (ull)c, c1 = (ull)(c >> 64);
    const unsigned __int128 l = (unsigned __int128)c0 * c0;
    const unsigned __int128 mid = (unsigned __int128)c0 * c1;  // times 2^64, twice
    const unsigned __int128 h = (unsigned __int128)c1 * c1;
    U192 sq = U192{{(ull)l, (ull)(l >> 64), 0ull}};
    const U192 m1 = U192{{0ull, (ull)mid, (ull)(mid >> 64)}};
    sq = uadd(sq, m1);
    sq = uadd(sq, m1);
    sq = uadd(sq, U192{{0ull, 0ull, (ull)h}});
    if (ucmp(sq, u) <= 0) r = c;
  }
  return r;
}

template <int KM>
__global__ void __launch_bounds__(kVerifyThreads) k_verify(VerifyArgs a) {
  pdl_wait();  // the sieve grid's survivors and header are complete from here on
  if (a.zero_block && blockIdx.x == 0) {  // the other result block, for the next single-range run
    for (uint32_t i = threadIdx.x; i < a.zero_words; i += blockDim.x) a.zero_block[i] = 0ull;
    for (uint32_t i = threadIdx.x; i < a.zero_words2; i += blockDim.x) a.zero_block2[i] = 0ull;
  }
  ull n = a.hdr->n_surv;
  if (n > a.surv_cap) n = a.surv_cap;
  Ctx<KM> C;
  Isolator<KM> iso;
  iso.C = &C;
  for (ull idx = blockIdx.x * (ull)blockDim.x + threadIdx.x; idx < n;
       idx += (ull)gridDim.x * blockDim.x) {
    const ull rec = a.surv[idx];
    const uint32_t p32 = (uint32_t)(rec >> 32), q32 = (uint32_t)rec;  // relative to the range's base
    const uint32_t k = a.surv_range ? a.surv_range[idx] : 0u;
    const ull p = p32 + (a.base ? a.base[2 * (ull)k] : 0ull), q = q32 + (a.base ? a.base[2 * (ull)k + 1] : 0ull);
    if (!ctx_init(C, p, q)) {  // more moduli than this instantiation holds: never guess
      atomicOr(&a.hdr->status, kStatusVerifyFail);
      continue;
    }
    const ull M = p > q ? p : q;
    const unsigned __int128 M2 = (unsigned __int128)M * M;  // < 2^80
    iso.U = umul128(M2 * 45u, M2);                           // 45 M^4 < 2^166
    iso.run();
    if (iso.fail) atomicOr(&a.hdr->status, kStatusVerifyFail);
    for (int i = 0; i < iso.nroots; ++i) {
      const unsigned __int128 t = isqrt192(iso.roots[i]);
      const ull t0 = (ull)t, t1 = (ull)(t >> 64);
      // t^2 == u ?
      const unsigned __int128 l = (unsigned __int128)t0 * t0;
      const unsigned __int128 mid = (unsigned __int128)t0 * t1;
      U192 sq = U192{{(ull)l, (ull)(l >> 64), 0ull}};
      const U192 m1 = U192{{0ull, (ull)mid, (ull)(mid >> 64)}};
      sq = uadd(uadd(sq, m1), m1);
      sq = uadd(sq, U192{{0ull, 0ull, (ull)((unsigned __int128)t1 * t1)}});
      if (ucmp(sq, iso.roots[i]) != 0 || t == 0) continue;
      const ull slot = atomicAdd(&a.hdr->n_roots, 1ull);
      if (slot < a.root_cap) {
        a.roots[slot] = cuboid_root{p32, q32, t0, t1};
        a.root_range[slot] = a.surv_range ? a.surv_range[idx] : 0u;
      } else {
        atomicOr(&a.hdr->status, kStatusRootOverflow);
      }
    }
  }
}

// ---------------------------------------------------------------- host: moduli

typedef unsigned __int128 u128;

ull powmod_h(ull b, ull e, ull m) {
  ull r = 1 % m;
  b %= m;
  while (e) {
    if (e & 1) r = (ull)((u128)r * b % m);
    b = (ull)((u128)b * b % m);
    e >>= 1;
  }
  return r;
}

bool is_prime64(ull n) {
  if (n < 2) return false;
  static const ull small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  for (ull p : small) {
    if (n % p == 0) return n == p;
  }
  ull d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  for (ull a : small) {  // deterministic for n < 3.3e24
    ull x = powmod_h(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int i = 1; i < s; ++i) {
      x = (ull)((u128)x * x % n);
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}

std::mutex g_init_mu;
bool g_inited[64];

// The moduli: the kMaxMod largest primes below 2^62 (all above 2^61), with their
// Montgomery constants, and the Garner inverses m_i^-1 mod m_j in Montgomery form.
void host_moduli(ModConst mods[kMaxMod], ull ginv[kMaxMod][kMaxMod]) {
  ull cand = (1ull << 62) - 1;
  for (int j = 0; j < kMaxMod; ++j) {
    while (!is_prime64(cand)) cand -= 2;
    const ull m = cand;
    cand -= 2;
    ull inv = m;  // m^-1 mod 2^64 by Newton
    for (int it = 0; it < 6; ++it) inv *= 2 - m * inv;
    ModConst M;
    M.m = m;
    M.minv = (ull)0 - inv;
    const ull r1 = (ull)(((u128)1 << 64) % m);
    M.r2 = (ull)((u128)r1 * r1 % m);
    M.r3 = (ull)((u128)M.r2 * r1 % m);
    M.r4 = (ull)((u128)M.r2 * M.r2 % m);
    M.half = (m - 1) / 2;
    mods[j] = M;
  }
  for (int i = 0; i < kMaxMod; ++i)
    for (int j = i + 1; j < kMaxMod; ++j) {
      const ull mj = mods[j].m;
      const ull inv = powmod_h(mods[i].m % mj, mj - 2, mj);
      ginv[i][j] = (ull)(((u128)inv << 64) % mj);  // Montgomery form
    }
}

}  // namespace

cudaError_t verify_init_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_init_mu);
  if (dev >= 0 && dev < 64 && g_inited[dev]) return cudaSuccess;
  ModConst mods[kMaxMod];
  ull ginv[kMaxMod][kMaxMod] = {};
  host_moduli(mods, ginv);
  cudaError_t e = cudaMemcpyToSymbol(c_mod, mods, sizeof(mods));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_ginv, ginv, sizeof(ginv));
  if (e == cudaSuccess && dev >= 0 && dev < 64) g_inited[dev] = true;
  return e;
}

// The instantiation holding the moduli of the launch's largest p, q (max_bits; 0: any
// 32-bit pair, or any pair below 2^40 when records carry bases).
namespace {

// Test probe of the modular arithmetic (op 0: a b mod m_j; op 1: a mod m_j; op 2: the
// sign of the integer whose residues modulo m_0..m_{j-1} are a[i j .. i j + j - 1]).
__global__ void k_probe_modarith(uint32_t op, uint32_t j, const ull* a, const ull* b, uint32_t n, ull* out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = 0;
  if (op == 0) {
    const ModConst M = c_mod[j];
    out[i] = frommont(mmul(tomont(a[i], M), tomont(b[i], M), M), M);
  } else if (op == 1) {
    out[i] = red64(a[i], c_mod[j].m);
  } else {
    ull x[kMaxMod];
    bool zero = true;
    for (uint32_t k = 0; k < j; ++k) {
      x[k] = tomont(a[(size_t)i * j + k], c_mod[k]);
      zero &= x[k] == 0;
    }
    out[i] = zero ? 0ull : (ull)(long long)garner_sign<kMaxMod>(x, (int)j, DevMod{}, DevGinv{});
  }
}

}  // namespace

cudaError_t launch_verify(const VerifyArgs& a, uint32_t blocks, cudaStream_t s, bool pdl) {
  const int bits = a.max_bits ? (int)a.max_bits : (a.base ? 40 : 32);
  const int K = moduli_for_bits(bits);
  cudaError_t e;
  if (K <= 4) e = launch_ex(k_verify<4>, blocks, kVerifyThreads, 0, s, pdl, a);
  else if (K <= 6) e = launch_ex(k_verify<6>, blocks, kVerifyThreads, 0, s, pdl, a);
  else if (K <= 8) e = launch_ex(k_verify<8>, blocks, kVerifyThreads, 0, s, pdl, a);
  else if (K <= 10) e = launch_ex(k_verify<10>, blocks, kVerifyThreads, 0, s, pdl, a);
  else if (K <= 12) e = launch_ex(k_verify<12>, blocks, kVerifyThreads, 0, s, pdl, a);
  else e = launch_ex(k_verify<kMaxMod>, blocks, kVerifyThreads, 0, s, pdl, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace cuboid

// Probe of the root test's modular arithmetic for the tests: on the host (device = 0, the
// same functions compiled for the host) or on the GPU (device = 1).  op 0: out[i] =
// a[i] b[i] mod m_j by Montgomery products; op 1: out[i] = a[i] mod m_j; op 2: out[i] =
// sign (0, 1 or 2^64 - 1 for -1) of the integer X with |X| < (prod m_k - 1) / 2 whose
// residues modulo m_0 .. m_{j-1} are a[i j .. i j + j - 1] (Garner); op 3: out[k] = m_k for
// k < 14 (n ignored).  Host buffers; synchronous.
extern "C" int cuboid_probe_modarith(uint32_t op, uint32_t j, const uint64_t* a, const uint64_t* b, uint32_t n,
                                     uint64_t* out, int device) {
  using namespace cuboid;
  if (!out || op > 3 || (op < 2 && j >= (uint32_t)kMaxMod) || (op == 2 && (j < 1 || j > (uint32_t)kMaxMod)) ||
      (op < 3 && n && !a) || (op == 0 && n && !b))
    return CUBOID_EINVAL;
  ModConst mods[kMaxMod];
  ull ginv[kMaxMod][kMaxMod] = {};
  host_moduli(mods, ginv);
  if (op == 3) {
    for (int k = 0; k < kMaxMod; ++k) out[k] = mods[k].m;
    return CUBOID_OK;
  }
  if (n == 0) return CUBOID_OK;
  if (!device) {
    for (uint32_t i = 0; i < n; ++i) {
      if (op == 0) {
        const ModConst& M = mods[j];
        out[i] = frommont(mmul(tomont(a[i], M), tomont(b[i], M), M), M);
      } else if (op == 1) {
        out[i] = red64(a[i], mods[j].m);
      } else {
        ull x[kMaxMod];
        bool zero = true;
        for (uint32_t k = 0; k < j; ++k) {
          x[k] = tomont(a[(size_t)i * j + k], mods[k]);
          zero &= x[k] == 0;
        }
        out[i] = zero ? 0ull : (ull)(long long)garner_sign<kMaxMod>(x, (int)j, HostMod{mods}, HostGinv{ginv});
      }
    }
    return CUBOID_OK;
  }
  cudaError_t e = verify_init_device();
  const size_t na = op == 2 ? (size_t)n * j : n;
  ull *d_a = nullptr, *d_b = nullptr, *d_out = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&d_a, na * sizeof(ull));
  if (e == cudaSuccess) e = cudaMalloc(&d_b, n * sizeof(ull));
  if (e == cudaSuccess) e = cudaMalloc(&d_out, n * sizeof(ull));
  if (e == cudaSuccess) e = cudaMemcpy(d_a, a, na * sizeof(ull), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && op == 0) e = cudaMemcpy(d_b, b, n * sizeof(ull), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_probe_modarith<<<(n + 255) / 256, 256>>>(op, j, d_a, d_b, n, d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d_out, n * sizeof(ull), cudaMemcpyDeviceToHost);
  cudaFree(d_a);
  cudaFree(d_b);
  cudaFree(d_out);
  return status_from_cuda(e);
}
