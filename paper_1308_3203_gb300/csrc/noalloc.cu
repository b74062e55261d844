// rc_sort_accesses_noalloc: the access-record sort for callers that cannot
// allocate device memory.
//
// Some callers must not call cudaMalloc: a serving process that reserved its
// whole device-memory budget at start-up and runs under that fixed budget,
// a real-time pipeline that cannot accept the implicit device-wide
// synchronisation an allocation may cause, or a library embedded in a host
// application whose allocator it must not touch.  For them this entry point
// takes its scratch memory (the ping-pong record buffer and the digit
// histograms of the radix sort) from one file-scope device array of fixed
// size instead of the library workspace.  The array exists on every GPU that
// loads this module and stays allocated until the process exits.  Under lazy
// module loading (CUDA's default) the driver loads the module, and so creates
// the array, on a device's first call of this entry point: that set-up call
// must come before the caller reserves the rest of its device budget.
#include <mutex>
#include <string>

#include "device.cuh"
#include "racecheck.h"

namespace rc {

// Largest input of the allocation-free sort (4 MiB of records).
constexpr uint64_t kNoAllocMaxRecords = 1ull << 18;
// Digit histograms and scan partials for kNoAllocMaxRecords records.
constexpr size_t kNoAllocTmpWords = 65536 + 1024;
constexpr size_t kNoAllocScratchBytes = kNoAllocMaxRecords * sizeof(LogRec) + kNoAllocTmpWords * 4;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void *g_noalloc_addr[kMaxDevices] = {};  // device address of the array, per device
}  // namespace

}  // namespace rc

using namespace rc;

namespace {
int noalloc_fail(int code, const char *msg) {
  set_last_error(std::string("rc_sort_accesses_noalloc: ") + msg);
  return code;
}
}  // namespace

extern "C" int rc_sort_accesses_noalloc(const rc_access *in, rc_access *out, uint64_t n, uint32_t cell_bits,
                                        uint32_t item_bits, void *cuda_stream) {
  if (n == 0) return RC_OK;
  if (!in || !out || item_bits > 31 || cell_bits + item_bits > 58)
    return noalloc_fail(RC_E_INVALID, "bad pointers or sizes");
  if (n > kNoAllocMaxRecords || sort_tmp_words(n) > kNoAllocTmpWords)
    return noalloc_fail(RC_E_CAPACITY, "more than 2^18 records (the size of the fixed scratch array)");
  // an error left by some earlier, unrelated launch is not this call's: report it as such
  // instead of taking it for a failure of the sort below
  if (cudaPeekAtLastError() != cudaSuccess)
    return noalloc_fail(RC_E_CUDA, "a CUDA error was pending before the call");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(RC_E_CUDA, "no usable current device");
  void *base = nullptr;
  {
    // set-up, once per device, with that device current: the array's name is
    // only a host-side stand-in, the kernels need its device address.  With
    // lazy module loading this is also where the driver loads the module that
    // holds the array and creates the array on this device.
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
        return noalloc_fail(RC_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
      g_noalloc_addr[dev] = p;
    }
    base = g_noalloc_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  LogRec *scratch = static_cast<LogRec *>(base);
  uint32_t *tmp = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(base) + kNoAllocMaxRecords * sizeof(LogRec));
  const uint32_t ib = item_bits ? item_bits : 1;
  // every histogram entry and scan partial is written before it is read, so
  // nothing left in the array by an earlier call needs clearing
  sort_log_into(reinterpret_cast<const LogRec *>(in), reinterpret_cast<LogRec *>(out), scratch, n, ib,
                cell_bits + ib, tmp, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(RC_E_CUDA, cudaGetErrorString(e));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(RC_E_CUDA, cudaGetErrorString(e));
  return RC_OK;
}
