// Theorem 1.1 on reported roots: a positive root t of Q_pq (coprime p != q) gives a perfect
// cuboid exactly when t > p^2, t > p q, t > q^2 and (p^2 + t)(p q + t) > 2 t^2.  The last
// inequality is p^3 q + (p^2 + p q) t > t^2; with p, q below 2^40 and t below 2^128 both
// sides stay below 2^256 and are compared exactly in four 64-bit limbs.  Host code: roots
// are rare and already on the host when this runs.
#include <cstdint>

#include "cuboid_internal.cuh"

namespace {

typedef unsigned __int128 u128;

struct U256 {
  uint64_t w[4] = {0, 0, 0, 0};  // little-endian limbs
};

void add_at(U256& x, int k, u128 v) {
  for (; k < 4 && v; ++k) {
    const u128 s = (u128)x.w[k] + (uint64_t)v;
    x.w[k] = (uint64_t)s;
    v = (v >> 64) + (s >> 64);
  }
}

U256 mul(u128 a, u128 b) {
  U256 r;
  const uint64_t a0 = (uint64_t)a, a1 = (uint64_t)(a >> 64), b0 = (uint64_t)b, b1 = (uint64_t)(b >> 64);
  add_at(r, 0, (u128)a0 * b0);
  add_at(r, 1, (u128)a0 * b1);
  add_at(r, 1, (u128)a1 * b0);
  add_at(r, 2, (u128)a1 * b1);
  return r;
}

int cmp(const U256& x, const U256& y) {
  for (int k = 3; k >= 0; --k)
    if (x.w[k] != y.w[k]) return x.w[k] < y.w[k] ? -1 : 1;
  return 0;
}

void add(U256& x, const U256& y) {
  uint64_t c = 0;
  for (int k = 0; k < 4; ++k) {
    const u128 s = (u128)x.w[k] + y.w[k] + c;
    x.w[k] = (uint64_t)s;
    c = (uint64_t)(s >> 64);
  }
}

// p, q < 2^40: p^2, pq, q^2 < 2^80; (p^2 + pq) t < 2^209, p^3 q < 2^160, t^2 < 2^256.
bool holds(uint64_t p, uint64_t q, u128 t) {
  const u128 p2 = (u128)p * p, pq = (u128)p * q, q2 = (u128)q * q;
  if (t == 0 || !(t > p2) || !(t > pq) || !(t > q2)) return false;
  U256 lhs = mul(p2 + pq, t);
  add(lhs, mul(p2, pq));
  return cmp(lhs, mul(t, t)) > 0;
}

}  // namespace

extern "C" int cuboid_theorem11_flags(const cuboid_root* roots, uint64_t n, uint8_t* flags) {
  if (n && (!roots || !flags)) return CUBOID_EINVAL;
  for (uint64_t i = 0; i < n; ++i)
    flags[i] = holds(roots[i].p, roots[i].q, ((u128)roots[i].t_hi << 64) | roots[i].t_lo) ? 1 : 0;
  return CUBOID_OK;
}

extern "C" int cuboid_theorem11_flags_wide(const cuboid_root_wide* roots, uint64_t n, uint8_t* flags) {
  if (n && (!roots || !flags)) return CUBOID_EINVAL;
  for (uint64_t i = 0; i < n; ++i) {
    if (roots[i].p >= CUBOID_WIDE_LIMIT || roots[i].q >= CUBOID_WIDE_LIMIT) return CUBOID_ERANGE;
  }
  for (uint64_t i = 0; i < n; ++i)
    flags[i] = holds(roots[i].p, roots[i].q, ((u128)roots[i].t_hi << 64) | roots[i].t_lo) ? 1 : 0;
  return CUBOID_OK;
}
