// zc_noalloc.cu -- compression without a caller-supplied workspace.
//
// Some callers may not allocate device memory: code on a collective's
// progress path, where cudaMalloc would synchronise the whole device and stall
// the communication it serves, or a plugin inside a framework that owns every
// device byte through its own allocator and offers the plugin no way to get
// more.  zc_compress_noalloc gives them compression with no allocation at
// all: the scratch that zc_compress keeps in the caller's workspace (look-back
// records, range partials, the control block, the encoder CTAs' tile rings)
// lives instead in one fixed file-scope device array of this library; the
// rings it has room for bound the encoder grid of these calls.
#include <mutex>

#include "zc_launch.h"

namespace {

constexpr uint64_t NOALLOC_MAX_N = ZC_NOALLOC_MAX_N;
constexpr size_t NOALLOC_BYTES = 32u << 20;  // 32 MiB on every GPU that loads the library
constexpr int MAX_DEVICES = 64;

std::mutex g_mutex;
void* g_scratch[MAX_DEVICES];  // device address of the array, per device
bool g_ready[MAX_DEVICES];

}  // namespace

// The shared scratch.  In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

extern "C" int zc_compress_noalloc(const void* d_in, uint64_t n, int dtype, int eb_mode,
                                   double eb_value, int block, void* d_out, size_t out_cap,
                                   uint64_t* d_out_bytes, int* d_status, zc_stream_t s)
{
    if (n > NOALLOC_MAX_N || d_status == nullptr) return ZC_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZC_ERR_CUDA;
    if (dev < 0 || dev >= MAX_DEVICES) return ZC_ERR_ARG;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_ready[dev]) {
            // Once per device, with that device current: find the array's
            // device address and stamp it as an initialised workspace.
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
                return ZC_ERR_CUDA;
            const int st = zc_workspace_init(p, NOALLOC_BYTES, s);
            if (st != ZC_OK) return st;
            g_scratch[dev] = p;
            g_ready[dev] = true;
        }
        scratch = g_scratch[dev];
    }
    // The array keeps the previous call's contents; only the status word has
    // to start at zero (the look-back records are tagged per launch).
    int st = zc_clear_device_status(scratch, s);
    if (st != ZC_OK) return st;
    st = zc_compress(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap, d_out_bytes,
                     scratch, NOALLOC_BYTES, s);
    if (st != ZC_OK) return st;
    // This call's device status (a zc_status) goes to the caller's int.
    if (cudaMemcpyAsync(d_status, scratch, sizeof(int), cudaMemcpyDeviceToDevice,
                        (cudaStream_t)s) != cudaSuccess)
        return ZC_ERR_CUDA;
    return ZC_OK;
}
