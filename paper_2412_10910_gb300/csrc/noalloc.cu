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
// (kNoAllocScratchBytes) until the process exits.  The array's device address
// is looked up when a hierarchy is set up (with its device current) and kept
// with the handle, so the call must be made with that device current; a
// device reset frees the hierarchy's memory and the array together, and the
// handle must not be used after it (set up a new one).  The array is shared by all
// calls: two calls that overlap on the GPU (different streams, or different
// host threads without ordering) race on it and give wrong results; serialize
// them on one stream.  The array keeps whatever the last call left; nothing
// needs clearing, because the first phase writes every entry that the second
// phase reads.
#include "nnmg_internal.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_restrict_scratch[kNoAllocScratchBytes];

}  // namespace

namespace nnmg {
// Device address of g_restrict_scratch on the current device.  Host code cannot
// use the symbol itself (on the host it names a stand-in, not device memory).
// nnmg_setup_hierarchy calls this once per hierarchy, with the hierarchy's
// device current, and keeps the address with the handle; the lookup also makes
// the runtime load the array onto that device then, so a later
// nnmg_restrict_noalloc allocates nothing, not even on its first call.
int noalloc_scratch_lookup(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_restrict_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    return NNMG_CUDA_ERROR;
  }
  *out = p;
  return NNMG_OK;
}

// Defined with the other entry points: the handle's level data, its device
// and the scratch address looked up at its setup.
const DevLevel* handle_level(const nnmg_handle* h, int level);
int handle_max_nrhs(const nnmg_handle* h);
int handle_device(const nnmg_handle* h, void** noalloc_scratch);
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
  const int hdev = handle_device(h, &scratch);
  int dev = -1;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess || dev != hdev || !scratch) {
    set_error("nnmg_restrict_noalloc: call with the hierarchy's device current (device " +
              std::to_string(hdev) + ", current " + std::to_string(dev) + ")");
    return NNMG_INVALID_ARG;
  }
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
