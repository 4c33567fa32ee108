// K5 front: the reset and plan kernels of a sieve run.
//
// The plan turns each range (an inclusive rectangle of (p, q), optionally the triangle
// q < p) into row-oriented work: the row orientation (rows of p, or of q when the range
// is narrow in q), the chunk of 64-value words a subtile covers, and the inclusive prefix
// sum of tiles over the ranges that the sieve kernel's tile queue walks.
#include "cuboid_internal.cuh"

namespace cuboid {

namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t kNoRange = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
  for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  return v;
}

__global__ void k_reset(DevHeader* hdr, uint32_t n_ranges) {
  DevHeader h = {};
  h.n_ranges = n_ranges;
  *hdr = h;
}

// Plans ranges [first, first + count): row orientation, tile size and the inclusive
// prefix sum of tiles; zeroes their counts and pair totals; resets the queue cursor.
// count_arg == kNoRange: read the count from the header (batched launches).  reset:
// also clear the header's counters (the first launch of a plain run).
__global__ void __launch_bounds__(1024) k_plan(const cuboid_range* ranges, uint32_t first,
                                               uint32_t count_arg, DevHeader* hdr, TilePlan* plan,
                                               unsigned long long* counts, unsigned long long* npairs,
                                               uint32_t n_primes, uint32_t target_tiles, uint32_t reset,
                                               uint32_t subtiles_per_tile, cuboid_range inl, uint32_t use_inl) {
  __shared__ unsigned long long s_words;
  __shared__ unsigned long long s_carry;
  __shared__ unsigned long long s_warp[32];
  const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  pdl_trigger();  // a dependent sieve grid may start its prologue now
  const uint32_t count = count_arg == kNoRange ? hdr->n_ranges : count_arg;
  __syncthreads();
  if (tid == 0) {
    s_words = 0;
    s_carry = 0;
    if (reset) {
      DevHeader h = {};
      h.n_ranges = count;
      *hdr = h;
    }
  }
  __syncthreads();
  unsigned long long my_words = 0;
  TilePlan P_first{};  // this thread's first range, kept for the scan below
  for (uint32_t k = tid; k < count; k += blockDim.x) {
    const cuboid_range R = use_inl ? inl : ranges[first + k];  // inl: one range passed by value
    TilePlan P;
    unsigned long long words;
    if (!plan_orient(R, P, words)) atomicOr(&hdr->status, kStatusBadRange);
    my_words += words;
    if (k == tid) P_first = P;
    else plan[first + k] = P;
  }
  my_words = warp_sum_u64(my_words);
  if (lane == 0 && my_words) atomicAdd(&s_words, my_words);
  __syncthreads();
  // chunk size from the target number of subtiles (a tile is subtiles_per_tile of them)
  const unsigned long long cw = plan_chunk(s_words, target_tiles, subtiles_per_tile);

  for (uint32_t base = 0; base < count; base += blockDim.x) {
    const uint32_t k = base + tid;
    unsigned long long tiles = 0;
    TilePlan P;
    if (k < count) {
      P = base == 0 ? P_first : plan[first + k];
      tiles = plan_tiles(P, cw, subtiles_per_tile);
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

}  // namespace

cudaError_t launch_reset(DevHeader* hdr, uint32_t n_ranges, cudaStream_t s) {
  k_reset<<<1, 1, 0, s>>>(hdr, n_ranges);
  return cudaGetLastError();
}

cudaError_t launch_plan(const cuboid_range* ranges, uint32_t first, uint32_t count, DevHeader* hdr,
                        TilePlan* plan, unsigned long long* counts, unsigned long long* npairs,
                        uint32_t n_primes, uint32_t target_tiles, cudaStream_t s, bool reset,
                        uint32_t row_lanes, const cuboid_range* inline_range) {
  const cuboid_range inl = inline_range ? *inline_range : cuboid_range{};
  // one warp plans up to 32 ranges (a plain launch plans one): no block-wide barriers
  const uint32_t threads = count <= 32 ? 32u : 1024u;
  k_plan<<<1, threads, 0, s>>>(ranges, first, count, hdr, plan, counts, npairs, n_primes, target_tiles,
                            reset ? 1u : 0u, 32u / (row_lanes ? row_lanes : 32u), inl, inline_range ? 1u : 0u);
  return cudaGetLastError();
}

}  // namespace cuboid
