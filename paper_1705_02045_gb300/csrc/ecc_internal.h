// Internal interface between the host engine and the kernel translation units.
// Not part of the public ABI (include/ecc.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ecc {

enum Dtype : int { kU8 = 1, kU16 = 2, kF32 = 3 };
enum Conv : int { kConvV = 0, kConvT = 1 };

// Largest bin count whose int32 block histogram lives in shared memory.
constexpr int64_t kSmemBinsMax = 16384;

// Error bits the kernels OR into the device error word.
enum ErrBits : int { kErrValue = 1, kErrOverflow = 2 };

// One launch of the per-voxel contribution kernel over an image.
// The image is viewed as 3D (view = 3: n = {z, y, x}) or 4D (view = 4:
// n = {w, z, y, x}), slowest first; 1D/2D images are 3D views with leading
// extents 1 (embedding an image in a thicker box whose outside is +inf keeps
// its complex, so its curve). The kernels march along n[0].
// Streamed slabs: only planes [w_lo, w_hi) of n[0] are processed, and only
// planes [w_mem_lo, w_mem_hi) are readable; `img` points at plane w_mem_lo.
// Planes outside the image are +inf; planes inside the image but outside
// [w_mem_lo, w_mem_hi) must not be needed (w_mem_lo <= w_lo - 1 or 0, etc.).
struct LocalArgs {
  const void* img = nullptr;
  int dtype = kU8;
  int conv = kConvV;
  int view = 3;
  int64_t n[4] = {1, 1, 1, 1};
  int64_t w_lo = 0, w_hi = 0;   // voxel planes to process along n[0]
  int64_t w_mem_lo = 0, w_mem_hi = 0;  // planes present in memory
  int64_t bins = 256;
  int64_t row_pitch = 0;        // bytes between rows; 0 = dense (n_x * element size).
                                // Only the bit-sliced kernel takes a pitch.
  long long* vcec = nullptr;    // int64[bins] accumulator (integer images)
  int* err = nullptr;           // device error word
  unsigned long long* pairs = nullptr;       // float images: (key<<32 | contrib)
  unsigned long long* pair_count = nullptr;  // device counter
  int64_t pair_cap = 0;
  int grid = 0;                 // 0 = occupancy-sized persistent grid
  int variant = 0;              // kernel variant (0 = generic key kernel)
  int zc = 0;                   // planes per tile along the marching axis (0 = auto)
  int warps = 0;                // bit-sliced kernel: warps per block (0 = auto)
  int layout = 0;               // bit-sliced kernel: 0 auto, 1 row groups, 2 warp columns
  int hist = 0;                 // bit-sliced kernel histogram: 0 auto (shared memory when
                                // bins <= kSmemBinsMax), 1 shared memory, 2 global atomics
  long long* fused_curve = nullptr;  // bit-sliced kernel: the last block to finish writes
                                     // the curve (prefix sum of vcec), then zeroes vcec and
                                     // *done (which must start at 0)
  unsigned int* done = nullptr;
  cudaStream_t stream = nullptr;
};

// Launches the contribution+histogram (integer) or contribution+pairs
// (float) kernel. Returns the CUDA error of the launch. `launches` counts
// kernel launches.
cudaError_t launch_local(const LocalArgs& a, int num_sms, int64_t* launches);

// Codes of the value transform (k_quant.cu): out[i] = clamp(floor((in[i] - lo)
// * scale), 0, bins - 1) as uint8 (code_bytes 1) or uint16 (2), float32
// round-to-nearest steps; NaN / inf set kErrValue in *err.
cudaError_t launch_quantize(const float* in, void* out, int code_bytes, int64_t n, float lo,
                            float scale, int64_t bins, int* err, int num_sms, cudaStream_t stream,
                            int64_t* launches);

// curve[t] = sum_{s <= t} vcec[s], t < bins (one block).
cudaError_t launch_scan(const long long* vcec, long long* curve, int64_t bins,
                        cudaStream_t stream, int64_t* launches);

// Float path: sorts `n` packed pairs by key (radix sort on the high 32 bits),
// reduces equal keys, drops zero sums and prefix-sums: writes out_vals[k]
// (the thresholds as float32 bit patterns), out_chi[k] and *out_count.
// Temporary buffers come from `tmp` (bytes).
size_t float_tail_tmp_bytes(int64_t n);
cudaError_t launch_float_tail(unsigned long long* pairs, int64_t n, void* tmp,
                              size_t tmp_bytes, uint32_t* out_vals, long long* out_chi,
                              unsigned long long* out_count, cudaStream_t stream,
                              int64_t* launches);

}  // namespace ecc
