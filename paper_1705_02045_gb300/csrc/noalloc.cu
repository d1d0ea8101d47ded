// ecc_compute_device_noalloc: the integer single-image computation for
// callers that cannot allocate device memory (see include/ecc.h).
//
// The only scratch the path needs beyond the caller's image and curve is the
// int64 VCEC accumulator and an error word. Here they live in file-scope
// device arrays of a fixed size, present on every GPU that loads the library
// for as long as the process runs. Host code cannot use the array names as
// device addresses, so the address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
#include "engine.h"

#include <mutex>

namespace ecc {

namespace {

constexpr int64_t kNoAllocMaxBins = 65536;  // 512 KiB of int64 counters
constexpr int kMaxDevices = 64;

static __device__ __align__(256) long long g_noalloc_vcec[kNoAllocMaxBins];
static __device__ __align__(256) int g_noalloc_err[64];

struct DeviceScratch {
  long long* vcec = nullptr;
  int* err = nullptr;
  int num_sms = 0;
  bool ready = false;
};

std::mutex g_setup_mu;
DeviceScratch g_scratch[kMaxDevices];

// Per-device set-up on the first call made with that device current.
int scratch_for(int dev, DeviceScratch* out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceScratch& s = g_scratch[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_vcec) != cudaSuccess) return ECC_ERR_CUDA;
    s.vcec = static_cast<long long*>(p);
    if (cudaGetSymbolAddress(&p, g_noalloc_err) != cudaSuccess) return ECC_ERR_CUDA;
    s.err = static_cast<int*>(p);
    if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return ECC_ERR_CUDA;
    s.ready = true;
  }
  *out = s;
  return ECC_OK;
}

// Device or managed memory of device dev.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
         at.device == dev;
}

}  // namespace

}  // namespace ecc

using namespace ecc;

extern "C" int ecc_compute_device_noalloc(const void* d_image, const int64_t* dims, int ndim,
                                          ecc_dtype dtype, int64_t bins, int convention,
                                          int64_t* d_curve, void* stream) {
  try {
    Shape s;
    int rc = validate_shape(nullptr, dims, ndim, &s);
    if (rc) return rc;
    if (dtype != ECC_U8 && dtype != ECC_U16) return ECC_ERR_DTYPE;
    if (bins < 1 || bins > kNoAllocMaxBins) return ECC_ERR_ARG;  // scratch holds 65536 counters
    if (convention != ECC_CONV_V && convention != ECC_CONV_T) return ECC_ERR_ARG;
    if (!d_curve || (s.voxels > 0 && !d_image)) return ECC_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ECC_ERR_CUDA;
    // both buffers must be device (or managed) memory of the current device,
    // and the image aligned to its element size (the kernels read whole
    // elements)
    if (!on_device(d_curve, dev) || (s.voxels > 0 && !on_device(d_image, dev)))
      return ECC_ERR_ARG;
    if (s.voxels > 0 && !elem_aligned(d_image, dtype)) return ECC_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(d_curve) & 7u) != 0) return ECC_ERR_ARG;
    DeviceScratch sc;
    if ((rc = scratch_for(dev, &sc))) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Once anything is queued, an error return first waits for the stream, so
    // that no kernel of a failed call is still writing the shared arrays when
    // the next call starts.
    auto fail = [&](int code) {
      cudaStreamSynchronize(st);
      cudaGetLastError();
      return code;
    };
    // the arrays keep the previous call's contents: clear what starts at zero
    if (cudaMemsetAsync(sc.vcec, 0, sizeof(long long) * bins, st) != cudaSuccess ||
        cudaMemsetAsync(sc.err, 0, sizeof(int), st) != cudaSuccess)
      return fail(ECC_ERR_CUDA);
    int64_t launches = 0;
    if (s.voxels > 0) {
      LocalArgs a;
      a.img = d_image;
      a.dtype = dtype;
      a.conv = convention;
      a.view = s.view;
      for (int i = 0; i < 4; ++i) a.n[i] = s.n[i];
      a.bins = bins;
      a.vcec = sc.vcec;
      a.err = sc.err;
      a.stream = st;
      a.w_mem_lo = 0;
      a.w_mem_hi = a.n[0];
      const int64_t step = max_planes_per_launch(s, sc.num_sms);
      for (int64_t w = 0; w < a.n[0]; w += step) {
        a.w_lo = w;
        a.w_hi = std::min(a.n[0], w + step);
        if (launch_local(a, sc.num_sms, &launches) != cudaSuccess) return fail(ECC_ERR_CUDA);
      }
    }
    if (launch_scan(sc.vcec, reinterpret_cast<long long*>(d_curve), bins, st, &launches) !=
        cudaSuccess)
      return fail(ECC_ERR_CUDA);
    int word = 0;
    if (cudaMemcpyAsync(&word, sc.err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return fail(ECC_ERR_CUDA);
    if (cudaStreamSynchronize(st) != cudaSuccess) return ECC_ERR_CUDA;
    if (word & kErrValue) return ECC_ERR_VALUE;
    if (word & kErrOverflow) return ECC_ERR_CUDA;
    return ECC_OK;
  } catch (...) {
    return ECC_ERR_CUDA;
  }
}
