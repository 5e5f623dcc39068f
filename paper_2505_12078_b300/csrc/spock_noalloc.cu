// spock_noalloc.cu -- spock_op_T_noalloc: one evaluation of T that allocates
// no device memory. Its scratch (control block, barrier flags, reduction
// partials, sweep vectors) lives in the file-scope device array below, which
// every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include "../../include/spock.h"
#include "spock_internal.h"

// every call on a device shares this array; calls that overlap on the GPU race
static __device__ __align__(256) unsigned char g_spock_scratch[SPOCK_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
// device address of g_spock_scratch per device (the host-side name of the
// array is only a stand-in, never a device address)
void* g_scratch_addr[kMaxDevices] = {};
}  // namespace

extern "C" int spock_op_T_noalloc(spock_problem* p, int precision, const void* v_in, void* v_out,
                                  double* stats, void* stream) {
  if (!p || !v_in || !v_out || (precision != 32 && precision != 64)) return SPOCK_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPOCK_EDEVICE;
  if (!g_scratch_addr[dev]) {
    // first call on this device, with the device current: look the address up once
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_spock_scratch) != cudaSuccess || !ptr) return SPOCK_EDEVICE;
    g_scratch_addr[dev] = ptr;
  }
  return spock::op_T_with_scratch(p, precision, v_in, v_out, stats, (cudaStream_t)stream,
                                  static_cast<unsigned char*>(g_scratch_addr[dev]),
                                  (size_t)SPOCK_NOALLOC_SCRATCH_BYTES);
}
