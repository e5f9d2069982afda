// mera_ascend_noalloc: the ascending superoperator with its scratch held in a
// library-owned device array instead of a caller-provided workspace.
//
// Some callers cannot give this library a scratch buffer: an application
// whose pool allocator owns every byte of device memory and may not be
// bypassed, or a latency-bound loop where a cudaMalloc (which can
// synchronise the device) is not acceptable.  This entry point lets them
// run the map with only their inputs and output.  The scratch is a
// file-scope device array of MERA_NOALLOC_SCRATCH_BYTES that every device
// loading the library keeps until the process exits.
#include <cstdio>
#include <map>
#include <mutex>

#include "../../include/mera.h"

namespace mera {
mera_status set_last_error(mera_status st, const char* msg);
void* current_cu_context();
}

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MERA_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
// (device ordinal, driver context) -> device address of the array.  The
// context is part of the key: after a device reset the device's new primary
// context loads the module again, possibly at another address.
std::map<std::pair<int, void*>, void*> g_noalloc_addr;

// Device address of the array on the current device, looked up once per
// device and context.  In host code `g_noalloc_scratch` only names a
// host-side shadow, so it must never be handed to a kernel directly.
mera_status scratch_address(void** out, const char** why) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    *why = "cudaGetDevice failed";
    return MERA_ECUDA;
  }
  const std::pair<int, void*> key{dev, mera::current_cu_context()};
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_addr.find(key);
  if (it != g_noalloc_addr.end()) {
    *out = it->second;
    return MERA_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    *why = "cudaGetSymbolAddress of the static scratch array failed";
    return MERA_ECUDA;
  }
  // the lookup made the device's context current if none was: file the
  // address under that context
  g_noalloc_addr[{dev, mera::current_cu_context()}] = p;
  *out = p;
  return MERA_OK;
}

}  // namespace

extern "C" mera_status mera_ascend_noalloc(const double* h, const double* u, const double* w, int chi_b, int chi_t,
                                           double* h_out, int prec, void* stream) {
  size_t need = 0;
  mera_status st = mera_workspace_size(MERA_OP_ASCEND, chi_b, chi_t, prec, &need);
  if (st != MERA_OK) return st;  // message already recorded
  if (need > size_t(MERA_NOALLOC_SCRATCH_BYTES)) {
    char msg[160];
    snprintf(msg, sizeof msg, "mera_ascend_noalloc: chi_b=%d chi_t=%d needs %zu scratch bytes, the static array holds %zu",
             chi_b, chi_t, need, size_t(MERA_NOALLOC_SCRATCH_BYTES));
    return mera::set_last_error(MERA_EINVAL, msg);
  }
  void* scratch = nullptr;
  const char* why = "";
  st = scratch_address(&scratch, &why);
  if (st != MERA_OK) return mera::set_last_error(st, why);
  return mera_ascend(h, u, w, chi_b, chi_t, h_out, prec, scratch, size_t(MERA_NOALLOC_SCRATCH_BYTES), stream);
}
