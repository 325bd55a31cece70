// noalloc.cu -- rabitq_search_noalloc: the search entry point that allocates
// no memory at call time.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocating
// routine) when they search -- e.g. a serving process whose own allocator has
// already reserved the GPU's free memory up front, so a library allocation
// would fail or fragment it; a caller on a latency-critical path where an
// allocation's implicit synchronization or page mapping is not acceptable; or
// a host that forbids allocation after start-up for predictability. They pass
// their own inputs and outputs; the scratch comes from one fixed array that is
// part of the library's device image.
//
// The scratch: g_noalloc_scratch below, kScratchBytes = 64 MiB, 256-byte
// aligned. Every GPU that loads this library holds it until the process exits.
// Host code cannot use the array's name as a device address (on the host it
// is only a stand-in symbol), so the first call on each device, with that
// device current, looks its address up with cudaGetSymbolAddress and keeps it;
// make that first call before any stream capture. All calls share the one
// array and it keeps the last call's contents; the only state that must start
// at zero (the overflow flag and the non-finite-query flag) is cleared by
// every call. Calls whose work
// overlaps on the GPU (two streams, two host threads) race on the array.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

bool device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int rabitq_search_noalloc(const rabitq_index* X, const float* queries, int64_t nq,
                                     int32_t k, int32_t nprobe, int32_t bq, float eps0,
                                     int64_t* out_ids, float* out_dist,
                                     const rabitq_search_opts* opts_in) {
  using namespace rbq;
  set_error("");
  if (!X) return fail(RABITQ_EINVAL, "rabitq_search_noalloc: index is null");
  rabitq_search_opts opts;
  rabitq_search_opts_default(&opts);
  if (opts_in) opts = *opts_in;
  if (opts.max_candidates == 0) opts.max_candidates = 65536;
  if (nq < 0) return fail(RABITQ_EINVAL, "rabitq_search_noalloc: nq < 0");
  if (nq == 0) return RABITQ_OK;
  if (!queries || !out_ids || !out_dist)
    return fail(RABITQ_EINVAL, "rabitq_search_noalloc: null pointer");
  if (k < 1 || k > 1024) return fail(RABITQ_EINVAL, "rabitq_search_noalloc: need 1 <= k <= 1024");
  if (nprobe < 1 || nprobe > X->K || nprobe > 16384)
    return fail(RABITQ_EINVAL, "rabitq_search_noalloc: need 1 <= nprobe <= min(K, 16384)");
  if (bq < 1 || bq > 8) return fail(RABITQ_EINVAL, "rabitq_search_noalloc: need 1 <= bq <= 8");
  if (!(eps0 >= 0.0f) || !(eps0 < __builtin_inff()))
    return fail(RABITQ_EINVAL, "rabitq_search_noalloc: eps0 must be finite and >= 0");
  if (opts.max_candidates < 4096 || opts.max_candidates > (1 << 26))
    return fail(RABITQ_EINVAL, "rabitq_search_noalloc: max_candidates must be in [4096, 2^26]");
  if (opts.rot_precision != RABITQ_ROT_FP32 ||
      (opts.scan_path != RABITQ_SCAN_AUTO && opts.scan_path != RABITQ_SCAN_POPC))
    return fail(RABITQ_EUNSUPPORTED, "rabitq_search_noalloc: FP32 rotation, popcount scan only");
  if (!device_pointer(queries) || !device_pointer(out_ids) || !device_pointer(out_dist) ||
      (opts.per_query_nprobe && !device_pointer(opts.per_query_nprobe)))
    return fail(RABITQ_EINVAL,
                "rabitq_search_noalloc: queries, outputs and per_query_nprobe must be device "
                "memory (host buffers would need staging memory)");
  // the scratch address below belongs to the current device, and the index's
  // arrays to the device it was built or loaded on: they must be the same
  RBQ_CHECK(check_device(X->device, "rabitq_search_noalloc"));
  int dev = 0;
  RBQ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(RABITQ_EUNSUPPORTED, "rabitq_search_noalloc: device ordinal out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(RABITQ_ECUDA, std::string("rabitq_search_noalloc: scratch address lookup "
                                              "failed: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  SearchArgs a;
  a.X = X;
  a.queries = queries;
  a.nq = nq;
  a.k = k;
  a.nprobe = nprobe;
  a.bq = bq;
  a.eps0 = eps0;
  a.seed = opts.quant_seed;
  a.per_query_nprobe = opts.per_query_nprobe;
  a.cand_cap = opts.max_candidates;
  a.out_ids = out_ids;
  a.out_dist = out_dist;
  a.trace = nullptr;
  a.rot_precision = opts.rot_precision;
  a.scan_path = opts.scan_path;
  a.stage_ms = nullptr;
  a.allow_warp = 0;  // the warp layout's candidate regions do not fit the fixed scratch
  return search_dev_prealloc(a, static_cast<unsigned char*>(scratch), kScratchBytes,
                             static_cast<cudaStream_t>(opts.stream));
}
