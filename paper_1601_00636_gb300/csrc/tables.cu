// K1: device builder of the unsolvability tables u_r (Eq. 2.3, Definition 1.1, section 2).
//
// For each prime r of the caller's list:
//   * v_r(k) = u_r(k, 1) for k in [0, r): (k, 1) is unsolvable iff no t in [0, r) makes
//     Q_{k,1}(t) = 0 mod r (every t is tried, Definition 1.1);
//   * the full table u_r(a, b), either from v_r by the weighted homogeneity of Eq. 1.1
//     (Q_{la,lb}(l^2 t) = l^20 Q_ab(t), so u_r(a, b) = v_r(a b^-1) for b != 0 and
//     u_r(a, 0) = 0 because t = 0 is then a root), or -- CUBOID_BUILD_FULL -- by trying
//     every t for every (a, b);
//   * the effective order (caller order or decreasing unsolvable fraction).
// The tables are stored as "window rows" (see cuboid_internal.cuh) in the effective
// order, and can be exported in the byte layout of Eq. 2.6.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "cuboid_internal.cuh"

namespace cuboid {

namespace {

// Residues below r < 2^14: products stay below 2^28.
__device__ __forceinline__ uint32_t mulm(uint32_t a, uint32_t b, uint32_t r) { return a * b % r; }
__device__ __forceinline__ uint32_t addm(uint32_t a, uint32_t b, uint32_t r) {
  uint32_t s = a + b;
  return s >= r ? s - r : s;
}
__device__ __forceinline__ uint32_t negm(uint32_t a, uint32_t r) { return a ? r - a : 0; }
__device__ __forceinline__ uint32_t scal(uint32_t k, uint32_t a, uint32_t r) { return (k % r) * a % r; }

// Coefficients of Q_ab(t) (Eq. 1.1) modulo r: c[0..4] = t^8, t^6, t^4, t^2, t^0 terms
// (the t^10 coefficient is 1).  a, b < r.
__device__ void q_coeffs_mod(uint32_t a, uint32_t b, uint32_t r, uint32_t c[5]) {
  const uint32_t P = mulm(a, a, r), Q = mulm(b, b, r);
  const uint32_t P2 = mulm(P, P, r), P3 = mulm(P2, P, r), P4 = mulm(P3, P, r), P5 = mulm(P4, P, r);
  const uint32_t Q2 = mulm(Q, Q, r), Q3 = mulm(Q2, Q, r), Q4 = mulm(Q3, Q, r), Q5 = mulm(Q4, Q, r);
  // t^8: (2 q^2 + p^2)(3 q^2 - 2 p^2)
  c[0] = mulm(addm(scal(2, Q, r), P, r), addm(scal(3, Q, r), negm(scal(2, P, r), r), r), r);
  // t^6: q^8 + 10 p^2 q^6 + 4 p^4 q^4 - 14 p^6 q^2 + p^8
  uint32_t s = Q4;
  s = addm(s, scal(10, mulm(P, Q3, r), r), r);
  s = addm(s, scal(4, mulm(P2, Q2, r), r), r);
  s = addm(s, negm(scal(14, mulm(P3, Q, r), r), r), r);
  s = addm(s, P4, r);
  c[1] = s;
  // t^4: -p^2 q^2 (q^8 - 14 p^2 q^6 + 4 p^4 q^4 + 10 p^6 q^2 + p^8)
  s = Q4;
  s = addm(s, negm(scal(14, mulm(P, Q3, r), r), r), r);
  s = addm(s, scal(4, mulm(P2, Q2, r), r), r);
  s = addm(s, scal(10, mulm(P3, Q, r), r), r);
  s = addm(s, P4, r);
  c[2] = negm(mulm(mulm(P, Q, r), s, r), r);
  // t^2: -p^6 q^6 (q^2 + 2 p^2)(3 p^2 - 2 q^2)
  c[3] = negm(mulm(mulm(P3, Q3, r),
                   mulm(addm(Q, scal(2, P, r), r), addm(scal(3, P, r), negm(scal(2, Q, r), r), r), r),
                   r), r);
  // t^0: -q^10 p^10
  c[4] = negm(mulm(Q5, P5, r), r);
}

// Q(t) mod r with the coefficients above; Q depends on t through s = t^2 only.
__device__ __forceinline__ uint32_t q_at(const uint32_t c[5], uint32_t t, uint32_t r) {
  const uint32_t s = mulm(t, t, r);
  uint32_t v = 1 % r;
  for (int j = 0; j < 5; ++j) v = addm(mulm(v, s, r), c[j], r);
  return v;
}

__device__ bool solvable(uint32_t a, uint32_t b, uint32_t r) {
  uint32_t c[5];
  q_coeffs_mod(a, b, r, c);
  for (uint32_t t = 0; t < r; ++t)   // Definition 1.1: every t in [0, r)
    if (q_at(c, t, r) == 0) return true;
  return false;
}

// v_r(k) = u_r(k, 1) for every prime (caller order) and the unsolvable counts.
__global__ void k_reduced(const uint32_t* primes, const unsigned long long* voff, uint8_t* vbytes,
                          uint32_t* unsolvable) {
  const uint32_t i = blockIdx.x;
  const uint32_t r = primes[i];
  uint32_t cnt = 0;
  for (uint32_t k = threadIdx.x; k < r; k += blockDim.x) {
    const uint8_t u = solvable(k, 1 % r, r) ? 0 : 1;
    vbytes[voff[i] + k] = u;
    cnt += u;
  }
  if (cnt) atomicAdd(&unsolvable[i], cnt);
}

// v_r(k) = u_r(k, 1) read from full tables (imported files): bit k r + 1 of prime i.
__global__ void k_reduced_from_bits(const uint32_t* primes, const unsigned long long* voff,
                                    const unsigned long long* foff, const uint32_t* fbits, uint8_t* vbytes,
                                    uint32_t* unsolvable) {
  const uint32_t i = blockIdx.x;
  const uint32_t r = primes[i];
  uint32_t cnt = 0;
  for (uint32_t k = threadIdx.x; k < r; k += blockDim.x) {
    const uint64_t b = (uint64_t)k * r + 1 % r;
    const uint8_t u = (uint8_t)((fbits[foff[i] + b / 32] >> (b % 32)) & 1u);
    vbytes[voff[i] + k] = u;
    cnt += u;
  }
  if (cnt) atomicAdd(&unsolvable[i], cnt);
}

// Brute-force full tables, bit (a r + b) of prime i at fbits + foff[i] (words).
__global__ void k_full(const uint32_t* primes, const unsigned long long* foff, uint32_t* fbits) {
  const uint32_t i = blockIdx.y;
  const uint32_t r = primes[i];
  for (uint32_t a = blockIdx.x; a < r; a += gridDim.x) {
    for (uint32_t b = threadIdx.x; b < r; b += blockDim.x) {
      if (!solvable(a, b, r)) {
        const uint64_t bit = (uint64_t)a * r + b;
        atomicOr(&fbits[foff[i] + bit / 32], 1u << (bit % 32));
      }
    }
  }
}

// Effective order: order[rank] = caller index.  mode 0: caller order; 1: decreasing
// count/r; 2: decreasing count/(r + 1), the rejection rate of a random coprime pair.
__global__ void k_order(const uint32_t* primes, const uint32_t* unsolvable, uint32_t n, int mode,
                        uint32_t* order) {
  const uint64_t d = mode == 2 ? 1 : 0;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    if (mode == 0) {
      order[i] = i;
      continue;
    }
    const uint64_t ci = unsolvable[i], ri = primes[i];
    uint32_t rank = 0;
    for (uint32_t j = 0; j < n; ++j) {
      const uint64_t cj = unsolvable[j], rj = primes[j];
      const uint64_t lhs = cj * (ri + d), rhs = ci * (rj + d);  // fraction_j vs fraction_i
      if (lhs > rhs || (lhs == rhs && rj < ri)) ++rank;
    }
    order[rank] = i;
  }
}

// Window rows of effective prime e.  Dynamic smem: uint16 inverses [r].
__global__ void k_expand(const uint32_t* order, const PrimeInfo* info, const unsigned long long* voff,
                         const uint8_t* vbytes, const unsigned long long* foff, const uint32_t* fbits,
                         int full, uint32_t* words) {
  extern __shared__ uint16_t s_inv[];
  const uint32_t e = blockIdx.x;
  const PrimeInfo pi = info[e];
  const uint32_t r = pi.r, W = pi.W, i = order[e];
  const uint8_t* v = vbytes + voff[i];
  if (!full) {
    for (uint32_t y = threadIdx.x; y < r; y += blockDim.x) {
      uint32_t inv = 0;
      if (y) {  // y^(r-2) mod r
        uint32_t base = y, ex = r - 2, acc = 1;
        while (ex) {
          if (ex & 1) acc = acc * base % r;
          base = base * base % r;
          ex >>= 1;
        }
        inv = acc;
      }
      s_inv[y] = (uint16_t)inv;
    }
    __syncthreads();
  }
  const uint64_t total = (uint64_t)r * W;
  for (uint64_t idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const uint32_t a = (uint32_t)(idx / W), w = (uint32_t)(idx % W);
    uint32_t word = 0;
    for (uint32_t j = 0; j < 32; ++j) {
      const uint32_t y = (32u * w + j) % r;
      uint32_t bit;
      if (full) {
        const uint64_t b = (uint64_t)a * r + y;
        bit = (fbits[foff[i] + b / 32] >> (b % 32)) & 1u;
      } else {
        bit = y ? v[a * (uint32_t)s_inv[y] % r] : 0u;
      }
      word |= bit << j;
    }
    words[pi.off + idx] = word;
  }
}

// Eq. 2.6 export: byte k holds bits 8k..8k+7 of the row-major r x r table, lsb first.
__global__ void k_pack(const uint32_t* words, PrimeInfo pi, uint8_t* out, uint64_t nbytes) {
  const uint64_t rr = (uint64_t)pi.r * pi.r;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < nbytes;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t byte = 0;
    for (uint32_t j = 0; j < 8; ++j) {
      const uint64_t bi = 8 * k + j;
      if (bi >= rr) break;
      const uint32_t a = (uint32_t)(bi / pi.r), b = (uint32_t)(bi % pi.r);
      byte |= ((words[pi.off + (uint64_t)a * pi.W + b / 32] >> (b % 32)) & 1u) << j;
    }
    out[k] = (uint8_t)byte;
  }
}

bool is_prime_host(uint32_t x) {
  if (x < 2) return false;
  for (uint32_t f = 2; f * f <= x; ++f)
    if (x % f == 0) return false;
  return true;
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

}  // namespace

int status_from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CUBOID_OK;
  if (e == cudaErrorMemoryAllocation) return CUBOID_ENOMEM;
  return CUBOID_ECUDA;
}

int build_tables(const uint32_t* primes, uint32_t n, uint32_t flags, cudaStream_t s, cuboid_tables** out,
                 const uint8_t* const* packed) {
  if (!primes || !out || n == 0 || n > kMaxPrimes) return CUBOID_EINVAL;
  if (flags & ~(CUBOID_ORDER_BY_DENSITY | CUBOID_ORDER_BY_RATE | CUBOID_BUILD_FULL)) return CUBOID_EINVAL;
  if ((flags & CUBOID_ORDER_BY_DENSITY) && (flags & CUBOID_ORDER_BY_RATE)) return CUBOID_EINVAL;
  std::vector<uint32_t> pr(primes, primes + n);
  {
    std::vector<uint32_t> sorted = pr;
    std::sort(sorted.begin(), sorted.end());
    for (uint32_t i = 0; i < n; ++i) {
      if (sorted[i] >= kPrimeLimit || !is_prime_host(sorted[i])) return CUBOID_EINVAL;
      if (i && sorted[i] == sorted[i - 1]) return CUBOID_EINVAL;
    }
  }
  cuboid_tables* t = new (std::nothrow) cuboid_tables();
  if (!t) return CUBOID_ENOMEM;
  t->n = n;
  t->flags = flags | (packed ? CUBOID_TABLES_IMPORTED : 0u);
  t->primes = pr;
  cudaGetDevice(&t->device);
  cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, t->device);
  cudaDeviceGetAttribute(&t->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, t->device);
  cudaDeviceGetAttribute(&t->smem_per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, t->device);

  uint32_t* d_primes = nullptr;
  unsigned long long* d_voff = nullptr;
  unsigned long long* d_foff = nullptr;
  uint32_t* d_cnt = nullptr;
  uint32_t* d_order = nullptr;
  uint32_t* d_fbits = nullptr;
  int st = CUBOID_OK;
  cudaError_t e = cudaSuccess;
  const bool full = (flags & CUBOID_BUILD_FULL) || packed;
  std::vector<unsigned long long> foff(n);
  uint64_t ftot = 0;
  for (uint32_t i = 0; i < n; ++i) {
    foff[i] = ftot;  // words; the Eq. 2.6 bytes of prime i read as little-endian words
    ftot += ((uint64_t)pr[i] * pr[i] + 31) / 32;
  }

  // reduced-table offsets (caller order)
  t->vbyte_off.resize(n);
  uint64_t vtot = 0;
  uint32_t rmax = 0;
  for (uint32_t i = 0; i < n; ++i) {
    t->vbyte_off[i] = vtot;
    vtot += pr[i];
    rmax = std::max(rmax, pr[i]);
  }

#define CK(x)                     \
  do {                            \
    e = (x);                      \
    if (e != cudaSuccess) {       \
      st = status_from_cuda(e);   \
      goto fail;                  \
    }                             \
  } while (0)

  CK(cudaMalloc(&d_primes, n * sizeof(uint32_t)));
  CK(cudaMalloc(&d_voff, n * sizeof(unsigned long long)));
  CK(cudaMalloc(&d_cnt, n * sizeof(uint32_t)));
  CK(cudaMalloc(&d_order, n * sizeof(uint32_t)));
  CK(cudaMalloc(&t->d_vbytes, vtot));
  CK(cudaMemcpyAsync(d_primes, pr.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_voff, t->vbyte_off.data(), n * sizeof(unsigned long long),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(d_cnt, 0, n * sizeof(uint32_t), s));
  if (full) {
    CK(cudaMalloc(&d_foff, n * sizeof(unsigned long long)));
    CK(cudaMalloc(&d_fbits, ftot * sizeof(uint32_t)));
    CK(cudaMemcpyAsync(d_foff, foff.data(), n * sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(d_fbits, 0, ftot * sizeof(uint32_t), s));
  }
  if (packed) {
    for (uint32_t i = 0; i < n; ++i)
      CK(cudaMemcpyAsync(d_fbits + foff[i], packed[i], ((uint64_t)pr[i] * pr[i] + 7) / 8, cudaMemcpyHostToDevice,
                         s));
    k_reduced_from_bits<<<n, 256, 0, s>>>(d_primes, d_voff, d_foff, d_fbits, t->d_vbytes, d_cnt);
  } else {
    k_reduced<<<n, 256, 0, s>>>(d_primes, d_voff, t->d_vbytes, d_cnt);
  }
  CK(cudaGetLastError());
  k_order<<<1, 1024, 0, s>>>(d_primes, d_cnt, n,
                             (flags & CUBOID_ORDER_BY_RATE) ? 2 : ((flags & CUBOID_ORDER_BY_DENSITY) ? 1 : 0), d_order);
  CK(cudaGetLastError());
  t->order.resize(n);
  t->unsolvable.resize(n);
  CK(cudaMemcpyAsync(t->order.data(), d_order, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(t->unsolvable.data(), d_cnt, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));

  {
    // window-row layout in the effective order
    t->info.resize(n);
    uint64_t off = 0;
    for (uint32_t k = 0; k < n; ++k) {
      const uint32_t r = pr[t->order[k]];
      PrimeInfo pi;
      pi.r = r;
      pi.magic = (uint32_t)((1ull << 32) / r);
      pi.off = (uint32_t)off;
      pi.W = row_words(r);
      t->info[k] = pi;
      off += (uint64_t)r * pi.W;
    }
    t->total_words = off;
    if (off >= (1ull << 32)) {
      st = CUBOID_EINVAL;
      goto fail;
    }
  }
  if (full && !packed) {
    dim3 grid(std::min<uint32_t>(rmax, 1024), n);
    k_full<<<grid, 256, 0, s>>>(d_primes, d_foff, d_fbits);
    CK(cudaGetLastError());
  }
  CK(cudaMalloc(&t->d_info, n * sizeof(PrimeInfo)));
  CK(cudaMalloc(&t->d_words, (t->total_words + 4) * sizeof(uint32_t)));
  CK(cudaMemsetAsync(t->d_words, 0, (t->total_words + 4) * sizeof(uint32_t), s));
  CK(cudaMemcpyAsync(t->d_info, t->info.data(), n * sizeof(PrimeInfo), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_order, t->order.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  k_expand<<<n, 256, full ? 0 : rmax * sizeof(uint16_t), s>>>(d_order, t->d_info, d_voff, t->d_vbytes,
                                                               d_foff, d_fbits, full ? 1 : 0, t->d_words);
  CK(cudaGetLastError());

  {
    // odd trial-division primes below 2^16 for the coprimality mask
    std::vector<uint8_t> comp(1u << 16, 0);
    std::vector<TrialPrime> tp;
    for (uint32_t f = 3; f < (1u << 16); f += 2) {
      if (comp[f]) continue;
      for (uint32_t m = f * f; m < (1u << 16); m += 2 * f) comp[m] = 1;
      uint32_t inv = f;  // Newton iteration for f^-1 mod 2^32 (f odd)
      for (int it = 0; it < 5; ++it) inv *= 2u - f * inv;
      tp.push_back(TrialPrime{f, inv, 0xFFFFFFFFu / f, 0});
    }
    t->n_trial = (uint32_t)tp.size();
    CK(cudaMalloc(&t->d_trial, tp.size() * sizeof(TrialPrime)));
    CK(cudaMemcpyAsync(t->d_trial, tp.data(), tp.size() * sizeof(TrialPrime), cudaMemcpyHostToDevice, s));
  }
  {
    // coprimality mask image (layout in cuboid_internal.cuh)
    static std::vector<uint32_t> img;  // the same for every table set; filled once
    static std::mutex img_mu;
    std::lock_guard<std::mutex> lk(img_mu);
    if (img.empty()) {
      img.assign(kMaskImageWords, 0);
      uint32_t base = 0;
      for (uint32_t f = 3; f < kPeriodicBelow; f += 2) {
        if (!is_prime_host(f)) continue;
        for (uint32_t t = 0; t < f; ++t)
          for (uint32_t b = t; b < 128; b += f) img[4 * (base + t) + b / 32] |= 1u << (b % 32);
        img[4 * kMaskTab + f] = base;
        base += f;
      }
      for (uint32_t b = 0; b < 128; ++b) img[4 * (kBitTab + b) + b / 32] = 1u << (b % 32);
      for (uint32_t n2 = 0; n2 < kPeriodicBelow; ++n2)
        if (n2 < 3 || n2 % 2 == 0 || !is_prime_host(n2)) img[4 * kMaskTab + n2] = kBitTab;
    }
    CK(cudaMalloc(&t->d_mimg, kMaskImageWords * sizeof(uint32_t)));
    CK(cudaMemcpyAsync(t->d_mimg, img.data(), kMaskImageWords * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  }
  CK(cudaStreamSynchronize(s));
  CK(verify_init_device());

  dfree(d_primes);
  dfree(d_voff);
  dfree(d_foff);
  dfree(d_cnt);
  dfree(d_order);
  dfree(d_fbits);
  *out = t;
  return CUBOID_OK;

fail:
  cudaStreamSynchronize(s);
  dfree(d_primes);
  dfree(d_voff);
  dfree(d_foff);
  dfree(d_cnt);
  dfree(d_order);
  dfree(d_fbits);
  dfree(t->d_info);
  dfree(t->d_words);
  dfree(t->d_vbytes);
  dfree(t->d_trial);
  dfree(t->d_mimg);
  delete t;
  return st == CUBOID_OK ? CUBOID_ECUDA : st;
#undef CK
}

}  // namespace cuboid

using namespace cuboid;

extern "C" int cuboid_tables_build(const uint32_t* primes, uint32_t n, uint32_t flags, void* stream,
                                   cuboid_tables** out) {
  return build_tables(primes, n, flags, (cudaStream_t)stream, out, nullptr);
}

extern "C" int cuboid_tables_info(const cuboid_tables* t, uint32_t* n_primes, uint64_t* device_bytes,
                                  uint32_t* flags) {
  if (!t) return CUBOID_ENOTABLES;
  if (n_primes) *n_primes = t->n;
  if (device_bytes) {
    uint64_t vt = 0;
    for (uint32_t r : t->primes) vt += r;
    *device_bytes = (t->total_words + 4) * 4 + t->n * sizeof(PrimeInfo) + vt +
                    (uint64_t)t->n_trial * sizeof(TrialPrime) + kMaskImageWords * sizeof(uint32_t);
  }
  if (flags) *flags = t->flags;
  return CUBOID_OK;
}

extern "C" int cuboid_tables_order(const cuboid_tables* t, uint32_t* order_out) {
  if (!t) return CUBOID_ENOTABLES;
  if (!order_out) return CUBOID_EINVAL;
  std::memcpy(order_out, t->order.data(), t->n * sizeof(uint32_t));
  return CUBOID_OK;
}

extern "C" int cuboid_tables_copy_bits(const cuboid_tables* t, uint32_t prime_idx, uint8_t* dst,
                                       size_t cap, size_t* written) {
  if (!t) return CUBOID_ENOTABLES;
  if (prime_idx >= t->n) return CUBOID_EINVAL;
  uint32_t e = 0;
  while (t->order[e] != prime_idx) ++e;
  const PrimeInfo pi = t->info[e];
  const uint64_t nbytes = ((uint64_t)pi.r * pi.r + 7) / 8;
  if (written) *written = nbytes;
  if (!dst || cap < nbytes) return CUBOID_EOVERFLOW;
  uint8_t* d_out = nullptr;
  cudaError_t err = cudaMalloc(&d_out, nbytes);
  if (err != cudaSuccess) return status_from_cuda(err);
  k_pack<<<(unsigned)std::min<uint64_t>((nbytes + 255) / 256, 4096), 256>>>(t->d_words, pi, d_out, nbytes);
  err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaMemcpy(dst, d_out, nbytes, cudaMemcpyDeviceToHost);
  cudaFree(d_out);
  return status_from_cuda(err);
}

extern "C" int cuboid_tables_copy_reduced(const cuboid_tables* t, uint32_t prime_idx, uint8_t* dst,
                                          size_t cap) {
  if (!t) return CUBOID_ENOTABLES;
  if (prime_idx >= t->n || !dst) return CUBOID_EINVAL;
  const uint32_t r = t->primes[prime_idx];
  if (cap < r) return CUBOID_EOVERFLOW;
  return status_from_cuda(cudaMemcpy(dst, t->d_vbytes + t->vbyte_off[prime_idx], r, cudaMemcpyDeviceToHost));
}

extern "C" int cuboid_tables_set_tuning(cuboid_tables* t, const cuboid_tuning* tune) {
  if (!t) return CUBOID_ENOTABLES;
  if (!tune) return CUBOID_EINVAL;
  const uint32_t rl = tune->row_lanes;
  if (tune->block_threads % 32 || tune->block_threads > 1024 || tune->ctas_per_sm > 32 ||
      (rl != 0 && rl != 8 && rl != 16 && rl != 32) ||
      tune->hot_primes > kMaxHot)
    return CUBOID_EINVAL;
  t->tuning = *tune;
  return CUBOID_OK;
}

extern "C" int cuboid_tables_get_tuning(const cuboid_tables* t, cuboid_tuning* tune) {
  if (!t) return CUBOID_ENOTABLES;
  if (!tune) return CUBOID_EINVAL;
  *tune = t->tuning;
  return CUBOID_OK;
}

extern "C" int cuboid_tables_free(cuboid_tables* t) {
  if (!t) return CUBOID_ENOTABLES;
  if (t->users.load() > 0) return CUBOID_EBUSY;
  cudaDeviceSynchronize();
  cudaFree(t->d_info);
  cudaFree(t->d_words);
  cudaFree(t->d_vbytes);
  cudaFree(t->d_trial);
  cudaFree(t->d_mimg);
  delete t;
  return CUBOID_OK;
}
