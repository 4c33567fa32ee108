// An entry point of the sieve that allocates nothing.
//
// Who needs it: code that must not call cudaMalloc / cudaFree at the moment it sieves.
// A serving loop with a latency budget cannot afford them (both synchronise the device
// and can stall for milliseconds); a host that embeds the library may hand it a fixed
// memory pool and forbid any other device allocation; and a process at its memory limit
// has nothing left to allocate.  For them the working memory the sieve needs besides its
// inputs and outputs -- the tile plan of every range and the device header that holds
// the tile-queue cursor and the survivor/root counters -- lives in one fixed array of
// device memory that the library owns for as long as it is loaded.
#include <mutex>

#include "cuboid_internal.cuh"

namespace cuboid {

namespace {

constexpr size_t kHeaderBytes = (sizeof(DevHeader) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kHeaderBytes + (size_t)CUBOID_NOALLOC_MAX_RANGES * sizeof(TilePlan);

// The working memory of cuboid_sieve_noalloc: [DevHeader | pad to 256 | TilePlan x max].
// Every GPU that loads the library holds one copy until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_scratch_mu;
void* g_scratch_ptr[64];   // device address of g_noalloc_scratch, per device
bool g_scratch_ready[64];

// Host code cannot use g_noalloc_scratch's name as a device address (on the host it names
// a stand-in); ask the runtime for the real address once per device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ready[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
    g_scratch_ready[dev] = true;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void k_totals(const DevHeader* hdr, unsigned long long* totals) {
  totals[0] = hdr->n_surv;
  totals[1] = hdr->n_roots;
  totals[2] = hdr->status;
}

}  // namespace

}  // namespace cuboid

using namespace cuboid;

extern "C" int cuboid_sieve_noalloc(const cuboid_tables* t, const cuboid_range* ranges_dev, uint32_t n,
                                    uint64_t* counts_dev, uint64_t* npairs_dev, uint64_t* surv_dev,
                                    uint32_t* surv_range_dev, uint64_t surv_cap, cuboid_root* roots_dev,
                                    uint32_t* root_range_dev, uint64_t root_cap, uint64_t* totals_dev,
                                    void* stream) {
  if (!t) return CUBOID_ENOTABLES;
  if (n > CUBOID_NOALLOC_MAX_RANGES) return CUBOID_ETOOLARGE;
  if (!ranges_dev || n == 0 || !counts_dev || !npairs_dev || !totals_dev) return CUBOID_EINVAL;
  if ((surv_cap && (!surv_dev || !surv_range_dev)) || (root_cap && (!roots_dev || !root_range_dev)))
    return CUBOID_EINVAL;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != t->device) return CUBOID_EINVAL;
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return status_from_cuda(e);
  DevHeader* hdr = reinterpret_cast<DevHeader*>(base);
  TilePlan* plan = reinterpret_cast<TilePlan*>(static_cast<unsigned char*>(base) + kHeaderBytes);
  cudaStream_t s = (cudaStream_t)stream;

  const LaunchShape L = launch_shape(t);
  e = sieve_set_smem_limit(false, L.smem);
  if (e != cudaSuccess) return status_from_cuda(e);
  // the header keeps the previous call's counters: start from zero (n_ranges = n)
  e = launch_reset(hdr, n, s);
  if (e == cudaSuccess)
    e = launch_plan(ranges_dev, 0, 0xFFFFFFFFu, hdr, plan, reinterpret_cast<unsigned long long*>(counts_dev),
                    reinterpret_cast<unsigned long long*>(npairs_dev), t->n, L.target_tiles, s, false,
                    L.row_lanes);
  if (e == cudaSuccess) {
    SieveArgs a;
    a.info = t->d_info;
    a.words = t->d_words;
    a.trial = t->d_trial;
    a.mimg = t->d_mimg;
    a.plan = plan;
    a.hdr = hdr;
    a.counts = reinterpret_cast<unsigned long long*>(counts_dev);
    a.npairs = reinterpret_cast<unsigned long long*>(npairs_dev);
    a.surv = reinterpret_cast<unsigned long long*>(surv_dev);
    a.surv_range = surv_range_dev;
    a.surv_cap = surv_cap;
    a.n_primes = t->n;
    a.n_smem_primes = L.n_smem;
    a.smem_words = L.smem_words;
    a.n_trial = t->n_trial;
    a.range_first = 0;
    a.range_count = 0xFFFFFFFFu;
    fill_hot(a, t, L);
    e = launch_sieve(a, false, L.blocks, L.threads, L.smem, s);
  }
  if (e == cudaSuccess) {
    VerifyArgs v;
    v.surv = reinterpret_cast<const unsigned long long*>(surv_dev);
    v.surv_range = surv_range_dev;
    v.surv_cap = surv_cap;
    v.hdr = hdr;
    v.roots = roots_dev;
    v.root_range = root_range_dev;
    v.root_cap = root_cap;
    e = launch_verify(v, (uint32_t)t->sms * 2, s);
  }
  if (e == cudaSuccess) {
    k_totals<<<1, 1, 0, s>>>(hdr, reinterpret_cast<unsigned long long*>(totals_dev));
    e = cudaGetLastError();
  }
  return status_from_cuda(e);
}
