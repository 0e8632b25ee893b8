// static_scratch.cu -- pcf_pairwise_noalloc: pairwise matrices without a
// caller-provided workspace and without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need the
// matrices: code running inside a host framework whose operator interface
// hands over only input and output buffers (no allocator), real-time or
// embedded services that must not touch the driver's allocator after start-up,
// and code paths where a cudaMalloc would synchronize the device or fail
// because the memory budget is fully reserved.  For them this entry point
// uses a fixed scratch array that lives in the library's own device memory.
//
// The scratch is a file-scope __device__ array of PCF_NOALLOC_SCRATCH_BYTES.
// Every GPU on which the library is loaded holds it until the process exits.
// Host code cannot use the array's name as a device address (it names a
// host-side shadow), so the device address is fetched with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device; the result is cached.  That first call
// should therefore come before any stream capture.
//
// All calls on a device share the one array.  Each call re-initializes what
// it needs (error word, counters) at its start, so nothing is carried over;
// calls whose GPU work overlaps in time (different streams, different host
// threads without ordering) race on the array and produce garbage.
#include <mutex>

#include "internal.cuh"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[PCF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

// Device address of the scratch array on the current device (cached).
int scratch_address(void** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PCF_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PCF_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PCF_OK;
}

}  // namespace

extern "C" int pcf_pairwise_noalloc(const pcf_csr* x, const pcf_integral* F, int nF,
                                    int precision, int layout, int out_dtype,
                                    cudaStream_t stream)
{
    if (!x) return PCF_EINVAL;
    size_t need = 0;
    int rc = pcf_workspace_size(x, nullptr, precision, PCF_WS_FORWARD, &need);
    if (rc != PCF_OK) return rc;
    if (need > (size_t)PCF_NOALLOC_SCRATCH_BYTES) return PCF_ENOWS;
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != PCF_OK) return rc;
    return pcf_pairwise(x, F, nF, precision, layout, out_dtype, 0, scratch,
                        (size_t)PCF_NOALLOC_SCRATCH_BYTES, stream);
}
