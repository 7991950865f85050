// apax_noalloc.cu -- an encode entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc or any allocating routine: code that
// runs inside another runtime's memory pool or allocator hook (where a
// nested allocation would re-enter that allocator or break its accounting),
// signal-safe or real-time paths that must not block on the CUDA driver's
// allocator, and plug-ins whose host application owns all device memory and
// forbids allocations behind its back.  apax_encode already takes its
// workspace from the caller; this variant needs no workspace at all: its
// scratch (the offset-scan tile words, a ticket and completion counter, and
// the status word) lives in one fixed array of device memory that every GPU
// loading this library keeps until the process exits.
#include <mutex>

#include "apax_kernels.h"

namespace {

// Fixed scratch: enough for a fixed-quality encode of up to 32,760 tiles.
constexpr size_t kScratchBytes = APAX_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices];        // device address of g_scratch, per device
cudaError_t g_err[kMaxDevices];   // result of the one-time lookup
bool g_ready[kMaxDevices];

// Once per device, with that device current: the device address of the
// array (the host-side symbol is only a stand-in and must never reach a
// kernel).
int scratch_address(void **addr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return APAX_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
        void *p = nullptr;
        g_err[dev] = cudaGetSymbolAddress(&p, g_scratch);
        g_addr[dev] = p;
        g_ready[dev] = true;
    }
    if (g_err[dev] != cudaSuccess || !g_addr[dev]) return APAX_ERR_CUDA;
    *addr = g_addr[dev];
    return APAX_OK;
}

}  // namespace

extern "C" int apax_encode_noalloc(const void *x, int dtype, uint64_t n, const apax_params *p,
                                   void *out, uint64_t out_capacity, apax_result *res,
                                   void *stream)
{
    uint64_t need = 0;
    int st = apax_workspace_size(dtype, n, p, &need);
    if (st) return st;
    if (need > kScratchBytes) return APAX_ERR_CAPACITY;  // array too small for this many tiles
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st) return st;
    // the encode clears the scratch words it uses on the stream before launching
    return apax::encode_with_workspace(x, dtype, n, p, out, out_capacity, scratch, kScratchBytes,
                                       res, stream);
}
