// Host engine shared by the C-ABI translation units (not a public header).
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstdarg>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/ecc.h"
#include "ecc_internal.h"

namespace ecc {

// A growable device allocation owned by the handle.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    const size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&p, want);
    if (e == cudaSuccess) cap = want;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

// A shape validated and viewed as 3D/4D for the kernels.
struct Shape {
  int ndim = 0;
  int64_t dims[4] = {0, 0, 0, 0};
  int64_t voxels = 0;
  int view = 3;
  int64_t n[4] = {1, 1, 1, 1};
};

// Pinned host memory holding the curves of one batched computation, which
// the results of ecc_compute_batch point into (ecc_result.owned = 2) instead
// of owning a copy. Each curve is preceded by a 16-byte header: the block's
// address and kResultMagic. refs counts the results still alive plus one
// while the handle keeps the block for reuse; the last release frees it.
struct ResultBlock {
  unsigned char* p = nullptr;
  size_t cap = 0;
  std::atomic<int64_t> refs{1};
};
constexpr uint64_t kResultMagic = 0x45434342524c4b31ull;  // "ECCBRLK1"
constexpr size_t kResultHeader = 16;
// Drops one reference; frees the block's memory with the last one.
void result_block_release(ResultBlock* b);

struct BatchEngine;  // batch.cu
struct Server;       // batch.cu

// Tuned launch shape of the bit-sliced kernel for one shape class (tuner.cu).
struct TuneChoice {
  int warps = 0;
  int zc = 0;
  float ms = 0.f;
  int hist = 0;    // LocalArgs::hist
  int layout = 0;  // LocalArgs::layout (0: the default for the value bits)
};

struct Tuner {
  std::string path;  // JSON-lines cache file ("" = in memory only)
  std::map<std::string, TuneChoice> table;
  std::mutex mu;
  static std::string key(const LocalArgs& a);
  void load(const std::string& file);
  bool lookup(const std::string& k, TuneChoice* c);
  void store(const std::string& k, const TuneChoice& c);
};

}  // namespace ecc

struct ecc_handle {
  ecc_config cfg{};
  int device = 0;
  int num_sms = 0;
  int variant = 0;                     // contribution kernel: 0 auto, 1 generic, 2 bit-sliced
  int bits_warps = 0;                  // bit-sliced kernel warps per block (0 = auto)
  int bits_zc = 0;                     // bit-sliced kernel planes per tile (0 = auto)
  int bits_layout = 0;                 // bit-sliced kernel: 0 auto, 1 row groups, 2 warp columns
  ecc::Tuner* tuner = nullptr;         // launch-shape tuner (tuner_cache set or ECC_TUNE)
  cudaStream_t stream = nullptr;       // compute
  cudaStream_t copy_stream = nullptr;  // host <-> device
  std::mutex api_mu;                    // serialises the blocking entry points
  std::atomic<int64_t> launches{0};
  int64_t launch_tmp = 0;

  ecc::DevBuf img, vcec, curve, errw, pairs, pair_count, tmp, out_vals, out_chi, out_count;
  ecc::DevBuf codes;                    // value-transform codes (ecc_compute_quantized)
  ecc::DevBuf done;                     // block counter of the fused curve scan (kept at 0)
  const void* clean_vcec = nullptr;     // vcec buffer known to be zero on its first
  int64_t clean_bins = 0;               // clean_bins entries (fused launches keep it so)
  ecc::DevBuf batch_desc, batch_items, batch_vcec, batch_curve;
  int* h_err = nullptr;                 // pinned scalar for error readback
  unsigned long long* h_cnt = nullptr;  // pinned counts of the float path (pairs, survivors)
  std::vector<cudaEvent_t> up_ev;       // chunked host-image upload (ecc_compute)
  cudaEvent_t up_free = nullptr;        // the image buffer's previous readers are done
  cudaEvent_t sync_ev = nullptr;        // bounded waits of the blocking calls
  int64_t* h_curve = nullptr;           // pinned staging of integer curves
  size_t h_curve_cap = 0;               // entries of h_curve
  // pinned blocks the (threshold, chi) pairs of float images are copied into
  // (results owned = 2); the handle holds one reference to each, and a block
  // only it still references is reused by the next float image
  std::vector<ecc::ResultBlock*> pair_blocks;

  // instrumentation: event pairs around contribution kernels
  bool prof_on = false;
  double prof_span_ms = 0.0;           // span of the record read last (ecc_profile_span)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  std::vector<cudaEvent_t> prof_pool;  // events of earlier records, for reuse

  // batched launches and serving (batch.cu)
  ecc::BatchEngine* batch = nullptr;   // used by ecc_compute_batch
  ecc::Server* server = nullptr;       // request loop of ecc_submit / ecc_poll
};

namespace ecc {

// Error messages are kept per thread (the request loop's scheduler thread
// reports errors while the caller's threads use the handle): set_err records
// the message for (this thread, h), clear_err forgets it, last_err reads it.
int set_err(ecc_handle* h, int code, const char* fmt, ...);
void clear_err(const ecc_handle* h);
const char* last_err(const ecc_handle* h);
int cuda_err(ecc_handle* h, cudaError_t e, const char* what);
int validate_shape(ecc_handle* h, const int64_t* dims, int ndim, Shape* s);
int64_t default_bins(const ecc_handle* h, int dtype);
size_t dtype_bytes(int dtype);
bool is_device_ptr(const ecc_handle* h, const void* p);
// A device image is read with loads of its element type: its address must be
// a multiple of the element size (host images are copied, so any address).
inline bool elem_aligned(const void* p, int dtype) {
  return (reinterpret_cast<uintptr_t>(p) % dtype_bytes(dtype)) == 0;
}
// Enqueues VCEC accumulation (zeroed first) + contribution kernel + scan of
// an integer image already on the device.
// With n_chunks > 0 the image is still arriving in plane chunks: planes
// [chunk_end[k-1], chunk_end[k]) are on the device once chunk_ev[k] completed,
// and the contribution launches of a chunk wait for the next chunk's event
// (its first plane is their upper collar).
int enqueue_int(ecc_handle* h, const void* d_img, int64_t row_pitch, const Shape& s, int dtype,
                int64_t bins, long long* d_vcec, long long* d_curve, cudaStream_t stream,
                const int64_t* chunk_end = nullptr, const cudaEvent_t* chunk_ev = nullptr,
                int n_chunks = 0);
// True when the bit-sliced kernel applies to this shape / dtype / bin count.
bool bits_eligible(const ecc_handle* h, const Shape& s, int dtype, int64_t bins);
// Device copy of an image for the contribution kernels: a device image is used
// in place, a host image is copied (dense) into the handle's image buffer.
// *row_pitch = 0 means dense rows.
int stage_image(ecc_handle* h, const void* image, bool on_device, const Shape& s, int dtype,
                int64_t bins, cudaStream_t st, const void** d_img, int64_t* row_pitch);
// Bounded wait on an event (host side); ECC_ERR_TIMEOUT after timeout_us.
int wait_event(ecc_handle* h, cudaEvent_t ev, int64_t timeout_us);
cudaError_t launch_local(const LocalArgs& a, int num_sms, int64_t* launches);
// Planes of n[0] per contribution launch that keep every block's int32
// shared-memory histogram from overflowing.
int64_t max_planes_per_launch(const Shape& s, int num_sms);
void serve_shutdown(ecc_handle* h);
// Profiling events from the handle's pool (creating events costs host time
// on every call): take one, or give one back (caller holds api_mu).
cudaError_t prof_event_take(ecc_handle* h, cudaEvent_t* ev);
void prof_event_give(ecc_handle* h, cudaEvent_t ev);
// Times candidate launch shapes of the bit-sliced kernel on this launch.
int tune_bits(ecc_handle* h, const LocalArgs& base, TuneChoice* best);
int bits_nb(int dtype, int64_t bins);

}  // namespace ecc
