// Block inner product entry point that allocates nothing.
//
// lsba_gram needs a scratch buffer for the per-CTA partial sums of its
// two-stage reduction, and takes it from the handle's workspace, which is
// allocated with cudaMalloc the first time it is needed.  Some callers cannot
// allow that: latency-critical serving loops in which an allocation (and the
// device-wide synchronisation cudaFree implies) is not acceptable, and hosts
// that must keep the device's memory footprint fixed after start-up (a memory
// budget shared with other processes, or an allocator that owns all device
// memory).  lsba_gram_noalloc gives them the same result with no handle and no
// allocation: its scratch is a fixed array in the library's own device memory.
#include <mutex>

#include "../../include/lsba.h"
#include "lsba_internal.cuh"

using namespace lsba;

#define LSBA_NOALLOC_MAX_DEVICES 64

// Partial-sum scratch shared by every call on a device.  Every GPU that loads
// the library holds these LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES * 8 bytes (512 KiB)
// until the process exits.
static __device__ __align__(256) double g_gram_scratch[LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES];

// Device address of g_gram_scratch per device.  In host code the symbol's name
// is only a host-side stand-in: the address a kernel may use comes from
// cudaGetSymbolAddress, taken once per device with that device current.
static double* g_scratch_addr[LSBA_NOALLOC_MAX_DEVICES];
static int g_sms[LSBA_NOALLOC_MAX_DEVICES];
static std::mutex g_setup_mutex;

static int setup_device(int dev, double** addr, int* sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_gram_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LSBA_CUDA_ERROR;
    }
    int n_sms = 0;
    if (cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n_sms < 1) {
      cudaGetLastError();
      return LSBA_CUDA_ERROR;
    }
    g_sms[dev] = n_sms;
    g_scratch_addr[dev] = (double*)p;
  }
  *addr = g_scratch_addr[dev];
  *sms = g_sms[dev];
  return LSBA_OK;
}

extern "C" int lsba_gram_noalloc(const double* d_L, int a, const double* d_R, int b, int64_t n, int s,
                                 double* d_G, void* cuda_stream) {
  if (!d_L || !d_R || !d_G || a < 1 || b < 1 || b > 2 || s < 1 || s > LSBA_MAX_S || n < 1 ||
      a + b > LSBA_MAXB || (int64_t)a * s > LSBA_MAX_MS)
    return LSBA_INVALID_ARG;
  // The output alone must fit the scratch (one partial per CTA and entry).
  if ((int64_t)a * s * b * s > LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES) return LSBA_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= LSBA_NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return LSBA_CUDA_ERROR;
  }
  double* scratch = nullptr;
  int sms = 0;
  int rc = setup_device(dev, &scratch, &sms);
  if (rc != LSBA_OK) return rc;
  GramPlan p = plan_gram(n, s, a, b, sms);
  // Fewer row partitions when the planned partials would not fit the scratch.
  if ((int64_t)p.grid_x * p.q > LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES) {
    int gx = LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES / p.q;
    if (gx < 1) gx = 1;
    int64_t rpc = (n + gx - 1) / gx;
    rpc = ((rpc + p.rows_per_chunk - 1) / p.rows_per_chunk) * p.rows_per_chunk;
    p.rows_per_cta = rpc;
    p.grid_x = (int)((n + rpc - 1) / rpc);
  }
  if ((int64_t)p.grid_x * p.q > LSBA_GRAM_NOALLOC_SCRATCH_DOUBLES) return LSBA_INVALID_ARG;
  BlockPtrs L, R;
  for (int i = 0; i < LSBA_MAXB; ++i) L.p[i] = R.p[i] = nullptr;
  for (int i = 0; i < a; ++i) L.p[i] = d_L + (size_t)i * n * s;
  for (int i = 0; i < b; ++i) R.p[i] = d_R + (size_t)i * n * s;
  // An error left pending by earlier, unrelated work is the caller's: report
  // it without launching and without clearing it.  After the launch, an error
  // is this launch's own, so it is read and cleared.
  if (cudaPeekAtLastError() != cudaSuccess) return LSBA_CUDA_ERROR;
  launch_gram((cudaStream_t)cuda_stream, p, L, a, R, b, n, s, scratch, d_G, nullptr, 0);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return LSBA_CUDA_ERROR;
  }
  return LSBA_OK;
}
