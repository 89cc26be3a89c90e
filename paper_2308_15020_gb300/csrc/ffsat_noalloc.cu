// Statically reserved gradient scratch for ffsat_step_noalloc.
//
// The array below is part of the library's device image: every GPU on which
// the library is loaded holds it until the process exits.  Host code may not
// use its name as an address (on the host it names a stand-in object), so the
// device address is looked up once per device with cudaGetSymbolAddress, with
// that device current, and cached.
#include <mutex>

#include "ffsat.h"
#include "ffsat_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[FFSAT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

}  // namespace

namespace ffsat {

cudaError_t static_scratch(int device, void **ptr) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = p;
    }
    *ptr = g_addr[device];
    return cudaSuccess;
}

}  // namespace ffsat
