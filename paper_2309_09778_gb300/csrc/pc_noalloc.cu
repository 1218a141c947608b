// Decompression for callers that cannot allocate device memory.
//
// Some callers of this library have no way to obtain device memory when
// they need to decompress: hosts whose device-memory budget is fixed up
// front (every byte is handed out before the first call), or plugins given
// only an input and an output buffer by a framework that owns every
// allocation.  pc_decompress_noalloc serves them: it runs the same kernels as
// pc_decompress, with the scratch space taken from a fixed array compiled
// into this library.  Like pc_decompress it reads the container header back
// to the host and synchronizes the stream.
//
// The array is a file-scope __device__ array of kNoAllocScratchBytes.  Every
// GPU that loads this library's code for it holds the array until the
// process exits.  Host code cannot use the array's name as a device address,
// so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; later calls
// reuse it.
//
// Every call shares the one array and it keeps the contents of the last
// call; the decompression kernels overwrite every scratch word they read and
// pc_decompress clears the error word before launching.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array and must be serialized by the caller.
#include <mutex>

#include "pc_kernels.cuh"

namespace {
constexpr size_t kNoAllocScratchBytes = 32ull << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_pc_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

int scratch_of_current_device(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PC_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pc_noalloc_scratch) != cudaSuccess || p == nullptr) return PC_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PC_OK;
}
}  // namespace

extern "C" int pc_decompress_noalloc(const void* d_in, size_t in_size, void* d_field, size_t field_cap,
                                     size_t dims_out[3], int* dtype_out, void* stream) {
  if (!d_in || !d_field) return PC_ERR_ARG;
  if (in_size < (size_t)pc::kHdr) return PC_ERR_CORRUPT;
  void* scratch = nullptr;
  const int st = scratch_of_current_device(&scratch);
  if (st) return st;
  // pc_decompress refuses, before any launch, a container that needs more
  // scratch than the array holds (PC_ERR_CAPACITY)
  return pc_decompress(d_in, in_size, d_field, field_cap, dims_out, dtype_out, scratch, kNoAllocScratchBytes, stream);
}
