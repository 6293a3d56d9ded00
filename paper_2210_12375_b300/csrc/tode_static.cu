// tode_static.cu -- tode_adjoint_static: the discrete adjoint for callers
// that cannot allocate device memory.
//
// Some callers only receive their input and output buffers from a host
// framework (a plugin interface, say) and hold no device allocator of their
// own; others must not call cudaMalloc inside a latency-critical loop,
// because it can synchronise the whole device.  For them the adjoint's
// scratch (the work counter and one segment of recomputed step-start states
// per instance) lives in the file-scope array below instead of a caller
// buffer.  Every GPU that loads this library holds the array until the
// process exits.
//
// Host code sees g_adjoint_scratch only as a host-side stand-in; its device
// address comes from cudaGetSymbolAddress, taken once per device (with that
// device current) by the first call on the device and cached.
#include <mutex>

#include "tode_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_adjoint_scratch[TODE_STATIC_ADJOINT_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the static scratch on the current device.
tode_err static_scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    (void)cudaGetLastError();
    return TODE_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return TODE_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_adjoint_scratch) != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return TODE_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TODE_OK;
}

}  // namespace

extern "C" tode_err tode_adjoint_static(const tode_field_desc* f, const tode_options* o,
                                        const double* t0, const double* t1,
                                        const double* t_eval, int K, const int32_t* n_acc,
                                        const int32_t* status, const tode_tape* tape,
                                        const void* gy_eval, const void* gy_final, void* gy0,
                                        void* gparam, float* const* gW, float* const* gb,
                                        int32_t* overflow, void* stream) {
  // Arguments and tape first: tode_adjoint without scratch validates
  // everything and launches nothing, returning TODE_EWORKSPACE only when all
  // else is valid (TODE_OK when the batch is empty, an argument error
  // otherwise).  Then the size against the array, before any device work.
  const tode_err v = tode_adjoint(f, o, t0, t1, t_eval, K, n_acc, status, tape, gy_eval,
                                  gy_final, gy0, gparam, gW, gb, overflow, nullptr, 0, stream);
  if (v != TODE_EWORKSPACE) return v;
  const size_t need = tode_adjoint_scratch_size(f, o, tape);
  if (need > (size_t)TODE_STATIC_ADJOINT_SCRATCH_BYTES) return TODE_EWORKSPACE;
  void* scratch = nullptr;
  const tode_err e = static_scratch_address(&scratch);
  if (e != TODE_OK) return e;
  // the adjoint launcher clears the work counter at the start of the scratch
  // on `stream` before its kernel runs; nothing else needs to start at zero
  return tode_adjoint(f, o, t0, t1, t_eval, K, n_acc, status, tape, gy_eval, gy_final, gy0,
                      gparam, gW, gb, overflow, scratch, (size_t)TODE_STATIC_ADJOINT_SCRATCH_BYTES,
                      stream);
}
