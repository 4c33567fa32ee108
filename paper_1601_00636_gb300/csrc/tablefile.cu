// The paper's table files (section 2, section 3): the bit tables file holds, one after
// another, the r x r tables u_r packed as in Eq. 2.6 (ceil(r^2 / 8) bytes each, row-major
// index p~ r + q~, least significant bit first, last byte zero-padded); the primes file
// holds one record per prime, the C struct {short prime; unsigned int offset;} with the
// offset of the prime's table in the bit tables file.  Both are little-endian and the
// record is 8 bytes, the two bytes after `prime` being the struct's alignment padding
// (written as zero, ignored on reading).  Host code only: the device work is the table
// builder's.
#include <cstdio>
#include <cstring>
#include <vector>

#include "cuboid_internal.cuh"

using namespace cuboid;

namespace {

constexpr size_t kRecordBytes = 8;

// A prime the table builder accepts: r in [2, 9697) (the bound below Eq. 2.7).
bool is_table_prime(uint32_t r) {
  if (r < 2 || r >= kPrimeLimit) return false;
  for (uint32_t f = 2; f * f <= r; ++f)
    if (r % f == 0) return false;
  return true;
}

uint64_t packed_bytes(uint32_t r) { return ((uint64_t)r * r + 7) / 8; }

bool read_file(const char* path, std::vector<uint8_t>& out) {
  FILE* f = std::fopen(path, "rb");
  if (!f) return false;
  out.clear();
  uint8_t buf[1 << 16];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) out.insert(out.end(), buf, buf + k);
  const bool ok = !std::ferror(f);
  std::fclose(f);
  return ok;
}

bool write_file(const char* path, const uint8_t* data, size_t n) {
  FILE* f = std::fopen(path, "wb");
  if (!f) return false;
  const bool ok = std::fwrite(data, 1, n, f) == n;
  return (std::fclose(f) == 0) && ok;
}

void put_le(uint8_t* p, uint64_t v, int bytes) {
  for (int i = 0; i < bytes; ++i) p[i] = (uint8_t)(v >> (8 * i));
}

uint64_t get_le(const uint8_t* p, int bytes) {
  uint64_t v = 0;
  for (int i = 0; i < bytes; ++i) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

}  // namespace

extern "C" int cuboid_tables_export(const cuboid_tables* t, const char* bit_tables_path, const char* primes_path,
                                    uint64_t* bytes_written) {
  if (!t) return CUBOID_ENOTABLES;
  if (!bit_tables_path || !primes_path) return CUBOID_EINVAL;
  std::vector<uint8_t> blob, recs(t->n * kRecordBytes, 0);
  for (uint32_t i = 0; i < t->n; ++i) {
    const uint32_t r = t->primes[i];
    if (r > 32767) return CUBOID_ERANGE;                          // `short prime`
    if (blob.size() + packed_bytes(r) > 0xFFFFFFFFull) return CUBOID_ERANGE;  // Eq. 2.7
    put_le(&recs[i * kRecordBytes], r, 2);
    put_le(&recs[i * kRecordBytes + 4], blob.size(), 4);
    const size_t at = blob.size();
    blob.resize(at + packed_bytes(r));
    size_t got = 0;
    const int st = cuboid_tables_copy_bits(t, i, blob.data() + at, packed_bytes(r), &got);
    if (st != CUBOID_OK) return st;
  }
  if (!write_file(bit_tables_path, blob.data(), blob.size())) return CUBOID_EINVAL;
  if (!write_file(primes_path, recs.data(), recs.size())) return CUBOID_EINVAL;
  if (bytes_written) *bytes_written = blob.size();
  return CUBOID_OK;
}

extern "C" int cuboid_tables_import(const char* bit_tables_path, const char* primes_path, uint32_t flags,
                                    void* stream, cuboid_tables** out, uint64_t* bytes_loaded) {
  if (!bit_tables_path || !primes_path || !out) return CUBOID_EINVAL;
  if (flags & ~(CUBOID_ORDER_BY_DENSITY | CUBOID_ORDER_BY_RATE | CUBOID_IMPORT_CHECK)) return CUBOID_EINVAL;
  std::vector<uint8_t> blob, recs;
  if (!read_file(bit_tables_path, blob) || !read_file(primes_path, recs)) return CUBOID_EINVAL;
  if (recs.empty() || recs.size() % kRecordBytes) return CUBOID_EINVAL;
  const uint32_t n = (uint32_t)(recs.size() / kRecordBytes);
  if (n > kMaxPrimes) return CUBOID_EINVAL;
  std::vector<uint32_t> primes(n);
  std::vector<const uint8_t*> packed(n);
  for (uint32_t i = 0; i < n; ++i) {
    const uint8_t* rec = &recs[i * kRecordBytes];
    const uint32_t r = (uint32_t)get_le(rec, 2);
    const uint64_t off = get_le(rec + 4, 4);
    if (!is_table_prime(r)) return CUBOID_EINVAL;
    const uint64_t nb = packed_bytes(r);
    if (off + nb > blob.size()) return CUBOID_ERANGE;
    const uint32_t pad = (uint32_t)(nb * 8 - (uint64_t)r * r);  // Eq. 2.6: zero bits after r^2
    if (pad && (blob[off + nb - 1] >> (8 - pad)) != 0) return CUBOID_EINVAL;
    primes[i] = r;
    packed[i] = blob.data() + off;
  }
  const uint32_t order_flags = flags & (CUBOID_ORDER_BY_DENSITY | CUBOID_ORDER_BY_RATE);
  cudaStream_t s = (cudaStream_t)stream;
  cuboid_tables* t = nullptr;
  int st = build_tables(primes.data(), n, order_flags, s, &t, packed.data());
  if (st != CUBOID_OK) return st;
  if (flags & CUBOID_IMPORT_CHECK) {
    cuboid_tables* ref = nullptr;
    st = build_tables(primes.data(), n, order_flags, s, &ref, nullptr);
    std::vector<uint8_t> a, b;
    for (uint32_t i = 0; i < n && st == CUBOID_OK; ++i) {
      const uint64_t nb = packed_bytes(primes[i]);
      a.resize(nb);
      b.resize(nb);
      size_t got = 0;
      st = cuboid_tables_copy_bits(t, i, a.data(), nb, &got);
      if (st == CUBOID_OK) st = cuboid_tables_copy_bits(ref, i, b.data(), nb, &got);
      if (st == CUBOID_OK && std::memcmp(a.data(), b.data(), nb) != 0) st = CUBOID_EVERIFY;
    }
    if (ref) cuboid_tables_free(ref);
    if (st != CUBOID_OK) {
      cuboid_tables_free(t);
      return st;
    }
  }
  *out = t;
  if (bytes_loaded) *bytes_loaded = recs.size();
  return CUBOID_OK;
}
