// nnmg_restrict_noalloc: the restriction r_c = P^T r_f of nnmg_restrict, for
// callers that must not allocate device memory while they run.
//
// Who needs this: code that runs where cudaMalloc is not allowed or not wanted,
// for example inside a host callback or a signal-safe path, a process whose
// device memory is handed out by an external pool or budget, or a real-time
// loop that must never hit the allocator's latency or its out-of-memory
// failure.  nnmg_restrict itself allocates its work buffers on first use; this
// variant takes its scratch (the per-coarse-cell buffer of the first phase)
// from a fixed array that is part of the library's device image, so it never
// calls cudaMalloc, cudaFree or any allocating routine.
//
// Costs and limits: every GPU that loads the library holds the array
// (kNoAllocScratchBytes) until the process exits.  The array is shared by all
// calls: two calls that overlap on the GPU (different streams, or different
// host threads without ordering) race on it and give wrong results; serialize
// them on one stream.  The array keeps whatever the last call left; nothing
// needs clearing, because the first phase writes every entry that the second
// phase reads.
#include <mutex>

#include "nnmg_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_restrict_scratch[kNoAllocScratchBytes];

// Device address of g_restrict_scratch per device.  Host code cannot use the
// symbol itself (on the host it names a stand-in, not device memory), so the
// address is looked up once per device with that device current.
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

int scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    nnmg::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return NNMG_CUDA_ERROR;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    nnmg::set_error("device ordinal too large for the scratch address table");
    return NNMG_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_restrict_scratch);
    if (e != cudaSuccess || !p) {
      nnmg::set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return NNMG_CUDA_ERROR;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return NNMG_OK;
}

}  // namespace

// Defined with the other entry points: the handle's level data.
namespace nnmg {
const DevLevel* handle_level(const nnmg_handle* h, int level);
int handle_max_nrhs(const nnmg_handle* h);
}  // namespace nnmg

extern "C" int nnmg_restrict_noalloc(nnmg_handle* h, int fine_level, int precision,
                                     const void* fine, void* coarse, int nrhs, void* stream) {
  using namespace nnmg;
  const DevLevel* F = handle_level(h, fine_level);
  const DevLevel* C = handle_level(h, fine_level - 1);
  if (!F || !C || fine_level < 1) {
    set_error("nnmg_restrict_noalloc: bad handle or fine_level (must be >= 1)");
    return NNMG_INVALID_ARG;
  }
  if ((precision != NNMG_F32 && precision != NNMG_F64) || nrhs < 1 || nrhs > handle_max_nrhs(h) ||
      !fine || !coarse) {
    set_error("nnmg_restrict_noalloc: bad precision, nrhs or null vector");
    return NNMG_INVALID_ARG;
  }
  const size_t tsize = precision == NNMG_F64 ? sizeof(double) : sizeof(float);
  const size_t need = (size_t)C->n_cells * C->nloc * F->ncomp * nrhs * tsize;
  if (need > kNoAllocScratchBytes) {
    set_error("nnmg_restrict_noalloc: needs " + std::to_string(need) +
              " bytes of scratch (coarse cells x (k+1)^d x components x nrhs x value size), "
              "more than the fixed " + std::to_string(kNoAllocScratchBytes) +
              " bytes; use nnmg_restrict");
    return NNMG_INVALID_ARG;
  }
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != NNMG_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (precision == NNMG_F64)
    e = launch_restrict<double>(*F, *C, (const double*)fine, (double*)coarse, (double*)scratch, nrhs, s);
  else
    e = launch_restrict<float>(*F, *C, (const float*)fine, (float*)coarse, (float*)scratch, nrhs, s);
  if (e != cudaSuccess) {
    set_error(std::string("nnmg_restrict_noalloc: ") + cudaGetErrorString(e));
    return NNMG_CUDA_ERROR;
  }
  return NNMG_OK;
}
