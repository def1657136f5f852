// tt_inner_noalloc: the TT inner product with its scratch in a fixed device array.
//
// Some callers cannot hand the library a workspace: plain C programs that embed
// libtt without a device allocator of their own, and latency-critical loops that run
// under a fixed device-memory budget, where a cudaMalloc / cudaFree would both
// synchronise the device and fragment the budget.  For them this entry point needs
// no workspace and allocates nothing: the environment matrices of the sweep live in
// the file-scope array below, which every GPU that loads the library holds
// (kInnerScratchBytes of device memory) until the process exits.
#include <mutex>
#include <vector>

#include "tt_inner_eval.cuh"

namespace tt {

namespace {

constexpr size_t kInnerScratchDoubles = size_t(1) << 19;  // 4 MiB
constexpr size_t kInnerScratchBytes = kInnerScratchDoubles * sizeof(double);

// Device scratch shared by every call on a device.  In host code this name is only a
// host-side stand-in for the symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_inner_scratch[kInnerScratchDoubles];

std::mutex g_mu;
std::vector<void*> g_scratch_by_device;  // index = device ordinal; nullptr until set up

// Once per device, with that device current: look up the device address of the array.
int scratch_address(void** out) {
  int dev = 0;
  TT_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_mu);
  if ((int)g_scratch_by_device.size() <= dev) g_scratch_by_device.resize(dev + 1, nullptr);
  if (!g_scratch_by_device[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_inner_scratch);
    if (e != cudaSuccess || !p)
      return fail(TT_ERR_CUDA, std::string("tt_inner_noalloc: cudaGetSymbolAddress failed: ") +
                                   cudaGetErrorString(e));
    g_scratch_by_device[dev] = p;
  }
  *out = g_scratch_by_device[dev];
  return TT_OK;
}

}  // namespace

int inner_noalloc(const tt_train* x, const tt_train* y, double* out, cudaStream_t s) {
  const size_t need = inner_workspace_bytes(x, y);
  if (need > kInnerScratchBytes)
    return fail(TT_ERR_UNSUPPORTED,
                "tt_inner_noalloc: the trains need " + std::to_string(need) +
                    " bytes of environment scratch, more than the fixed " +
                    std::to_string(kInnerScratchBytes) + " bytes; use tt_inner with a workspace");
  void* scratch = nullptr;
  TT_TRY(scratch_address(&scratch));
  // Nothing in the scratch has to start at zero: the sweep sets E_0 = 1 itself and
  // writes every other entry before reading it.
  return x->dtype == TT_F64 ? inner_impl<double, double>(x, y, out, scratch, kInnerScratchBytes, s)
                            : inner_impl<float, float>(x, y, out, scratch, kInnerScratchBytes, s);
}

}  // namespace tt
