// noalloc.cu -- mrr_masks_static: the mask stage (edge image -> per-level masks, work
// lists, counts, labels) for callers that cannot allocate device memory.
//
// Some host programs may not call cudaMalloc: a plug-in inside an engine that owns
// every device allocation, a process whose allocator is already fully reserved, code
// run inside a pre-planned memory budget.  They can still hand in buffers they were
// given (the edge image and the mrr_levels outputs), but cannot create a context,
// because mrr_create allocates the context's pools.  This entry point needs no
// context: the one piece of scratch memory the stage uses -- the per-chunk counts of
// the work-list compaction -- lives in a file-scope __device__ array of fixed size.
//
// That array exists once per device that loads the library and stays allocated until
// the process exits.  Host code cannot use its name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with that device
// current) and keeps it; make that first call before any stream capture.  Every call
// shares the array: calls whose work overlaps on the GPU (two streams, or two host
// threads) race on it and must be ordered by the caller.  Nothing in it needs to start
// at zero: the count pass writes every entry the scatter pass then reads.
#include <cmath>
#include <cstring>
#include <mutex>

#include "mrr_internal.cuh"

namespace {

// Capacity: enough chunks for every level of a 4096 x 4096 frame (four levels of
// 4096^2, 2048^2, 1024^2 and 512^2 texels at 4096 texels per chunk = 4096 + 1024 + 256
// + 64 = 5440 chunks); 8192 entries = 32 KiB.
constexpr int STATIC_CHUNKS = 8192;
constexpr int STATIC_MAX_DIM = 4096;

__device__ __align__(256) uint32_t g_static_chunk_counts[STATIC_CHUNKS];

constexpr int MAX_DEVICES = 64;
uint32_t* g_static_ptr[MAX_DEVICES] = {};
std::mutex g_static_mu;

// Device address of the scratch array on the current device (looked up once).
cudaError_t static_scratch(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_chunk_counts);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

inline int level_dim(int n, int i) { return (n + (1 << i) - 1) >> i; }

}  // namespace

extern "C" mrr_status mrr_masks_static(const mrr_config* cfg, const uint8_t* edges_dev, const mrr_levels* lv,
                                       void* stream) {
  using namespace mrr;
  if (!cfg || !edges_dev || !lv || !lv->counts) return MRR_EINVAL;
  const mrr_config& c = *cfg;
  if (c.num_levels < 1 || c.num_levels > MRR_MAX_LEVELS || !c.enabled[c.num_levels - 1]) return MRR_EINVAL;
  if (lv->num_levels != c.num_levels) return MRR_EINVAL;
  const int W = lv->width[0], H = lv->height[0];
  if (W < 1 || H < 1 || W > STATIC_MAX_DIM || H > STATIC_MAX_DIM) return MRR_EINVAL;  // beyond the scratch
  MaskParams m;
  if (!mask_level_params(c, lv, m)) return MRR_EINVAL;  // a blurred level with sigma2 <= 0 or R > 6
  CompactParams cp;
  std::memset(&cp, 0, sizeof cp);
  int nchunks = 0;
  for (int i = 0; i < c.num_levels; ++i) {
    if (lv->width[i] != level_dim(W, i) || lv->height[i] != level_dim(H, i)) return MRR_EINVAL;
    if (c.enabled[i] && (!lv->alpha[i] || !lv->stencil[i] || !lv->worklist[i])) return MRR_EINVAL;
    if (!c.enabled[i]) {
      cp.zero_mask |= 1 << i;
      continue;
    }
    const int l = cp.nlev++;
    cp.level_of[l] = i;
    cp.chunk_begin[l] = nchunks;
    cp.Wi[l] = lv->width[i];
    cp.Hi[l] = lv->height[i];
    cp.stencil[l] = lv->stencil[i];
    cp.list[l] = lv->worklist[i];
    nchunks += (int)(((size_t)lv->width[i] * lv->height[i] + COMPACT_CHUNK - 1) / COMPACT_CHUNK);
  }
  for (int i = c.num_levels; i < MRR_MAX_LEVELS; ++i) cp.zero_mask |= 1 << i;
  cp.chunk_begin[cp.nlev] = nchunks;
  if (nchunks > STATIC_CHUNKS) return MRR_EINVAL;
  uint32_t* scratch = nullptr;
  if (static_scratch(&scratch) != cudaSuccess) return MRR_ECUDA;
  cp.chunk_counts = scratch;
  cp.counts = lv->counts;
  cudaStream_t s = (cudaStream_t)stream;
  if (launch_masks(m, edges_dev, s) != cudaSuccess) return MRR_ECUDA;
  if (launch_compact(cp, s) != cudaSuccess) return MRR_ECUDA;
  return MRR_OK;
}
