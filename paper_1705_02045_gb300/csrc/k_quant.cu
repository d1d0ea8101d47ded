// The value transform of Sec. 3 ("Other Ranges of Gray Values"): float values
// are shifted, scaled and rounded down into codes 0..bins-1, after which the
// integer algorithm runs unchanged on the codes; by the paper's remark the
// resulting curve is the float curve with its domain transformed.
//
// Reading taken: code(v) = clamp(floor((v - lo) * scale), 0, bins - 1) with
// scale = bins / (hi - lo); each step is one float32 operation rounded to
// nearest (explicit _rn intrinsics: no contraction into a fused multiply-add),
// so the codes are those of any IEEE float32 evaluation in the same order.
// NaN and +-inf set the value-error flag.
#include "ecc_internal.h"

#include <algorithm>

namespace ecc {

namespace {

template <typename Code>
__device__ __forceinline__ Code encode(float v, float lo, float scale, float top, int* err) {
  if (!isfinite(v)) {
    atomicOr(err, kErrValue);
    return 0;
  }
  const float p = __fmul_rn(__fsub_rn(v, lo), scale);
  if (!(p >= 0.f)) return 0;                 // below lo
  if (p >= top) return (Code)((int)top - 1);  // at or above hi
  return (Code)(int)p;                       // truncation = floor for p >= 0
}

// Grid-stride over groups of four values (16-byte loads when the input is
// 16-byte aligned), then the ragged tail one value at a time.
template <typename Code>
__global__ void __launch_bounds__(256)
k_quantize(const float* __restrict__ in, Code* __restrict__ out, int64_t n, float lo,
           float scale, float top, int* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t done = 0;
  if ((reinterpret_cast<uintptr_t>(in) & 15u) == 0) {
    const int64_t groups = n / 4;
    const float4* in4 = reinterpret_cast<const float4*>(in);
    for (int64_t g = t0; g < groups; g += stride) {
      const float4 v = __ldg(in4 + g);
      Code c[4] = {encode<Code>(v.x, lo, scale, top, err), encode<Code>(v.y, lo, scale, top, err),
                   encode<Code>(v.z, lo, scale, top, err), encode<Code>(v.w, lo, scale, top, err)};
      if (sizeof(Code) == 1) {
        const uint32_t w = (uint32_t)c[0] | ((uint32_t)c[1] << 8) | ((uint32_t)c[2] << 16) |
                           ((uint32_t)c[3] << 24);
        if ((reinterpret_cast<uintptr_t>(out) & 3u) == 0) {
          reinterpret_cast<uint32_t*>(out)[g] = w;
        } else {
          for (int k = 0; k < 4; ++k) out[4 * g + k] = c[k];
        }
      } else {
        if ((reinterpret_cast<uintptr_t>(out) & 7u) == 0) {
          const uint2 w = make_uint2((uint32_t)c[0] | ((uint32_t)c[1] << 16),
                                     (uint32_t)c[2] | ((uint32_t)c[3] << 16));
          reinterpret_cast<uint2*>(out)[g] = w;
        } else {
          for (int k = 0; k < 4; ++k) out[4 * g + k] = c[k];
        }
      }
    }
    done = groups * 4;
  }
  for (int64_t i = done + t0; i < n; i += stride) out[i] = encode<Code>(__ldg(in + i), lo, scale, top, err);
}

}  // namespace

cudaError_t launch_quantize(const float* in, void* out, int code_bytes, int64_t n, float lo,
                            float scale, int64_t bins, int* err, int num_sms, cudaStream_t stream,
                            int64_t* launches) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t want = (n / 4 + threads - 1) / threads;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms * 8));
  const float top = (float)bins;
  if (code_bytes == 1)
    k_quantize<uint8_t><<<grid, threads, 0, stream>>>(in, static_cast<uint8_t*>(out), n, lo,
                                                      scale, top, err);
  else
    k_quantize<uint16_t><<<grid, threads, 0, stream>>>(in, static_cast<uint16_t*>(out), n, lo,
                                                       scale, top, err);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace ecc
