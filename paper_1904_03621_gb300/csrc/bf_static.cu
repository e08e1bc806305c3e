// bf_low_spectrum_noalloc: the single-instance search with a workspace that
// lives in a fixed device array of this library instead of caller memory.
//
// Who needs it: callers that are not allowed to allocate device memory at
// the point where they search -- for example code running under a host
// framework whose caching allocator already owns the free device memory,
// callbacks and real-time loops where cudaMalloc's implicit device
// synchronisation is not acceptable, or embedded hosts whose memory budget
// is fixed at start-up.  They pass inputs and outputs only.
//
// The array below is a file-scope device symbol: every GPU that loads this
// library holds its 4 MiB until the process exits.  Host code cannot use
// the symbol's name as a device address, so the first call on each device
// (with that device current) asks the runtime for the address once and
// caches it for the life of the process (a cudaDeviceReset() destroys the
// array with its context, after which this entry point must not be called).  Calls share the array: two calls whose work overlaps on the
// GPU (different streams, or the same device from several host threads
// without ordering) race on it and give undefined results.
#include <cstring>
#include <mutex>

#include "bf.h"
#include "bf_internal.cuh"

namespace {

constexpr size_t kStaticWorkspaceBytes = (size_t)4 << 20;   // 4 MiB per device
constexpr int kStaticSpillLog2 = 16;                          // 65536 spill records
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices];   // device address of g_static_workspace, per device

}  // namespace

extern "C" bf_status bf_low_spectrum_noalloc(const void* J, const void* h, int n, int S, bf_dtype dtype,
                                             void* energies, uint64_t* states, const bf_options* opt,
                                             void* stream)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bf::report(BF_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return bf::report(BF_EUNSUPPORTED, "device ordinal beyond 63");
    void* ws = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_workspace);
            if (e != cudaSuccess || !p) return bf::report(BF_ECUDA, "cudaGetSymbolAddress of the static workspace failed");
            g_static_ptr[dev] = p;
        }
        ws = g_static_ptr[dev];
    }
    bf_options o{};
    if (opt) o = *opt;
    if (o.spill_log2 == 0) o.spill_log2 = kStaticSpillLog2;
    const size_t need = bf_workspace_size(n, S, dtype, &o);
    if (need > kStaticWorkspaceBytes)
        return bf::report(BF_EUNSUPPORTED, "this search needs a larger workspace than the 4 MiB static one "
                                           "(reduce S or spill_log2, or call bf_low_spectrum)");
    // need == 0: invalid arguments; bf_low_spectrum reports them before any launch
    bf_status st = bf_low_spectrum(J, h, n, S, dtype, energies, states, ws, kStaticWorkspaceBytes, &o, stream);
    if (st != BF_OK) return st;
    return bf_workspace_status(ws, stream);
}
