// Batched and served computation.
//
// The paper processes independent chunks with a pool of worker threads, each
// keeping its own VCEC (Sec. 3, "Parallel Computations"). On the GPU the same
// independence lets many images share one persistent launch: a work list of
// (image, tile range) items, balanced by voxel work on the host, is walked by
// a fixed grid; each block keeps a private shared-memory histogram per image
// (flushed when the image changes) and every image has its own int64 VCEC.
// Images the bit-sliced kernel takes (1-3D, uint8 with 256 bins or uint16 with
// 16384 / 65536 bins) go to the batched bit-sliced kernel, the others to the
// batched generic kernel. The launch sequence (zero VCECs, the two batched
// contribution kernels, batched scan) is captured once per slot in a CUDA
// graph whose kernels read the batch from a fixed device descriptor buffer; a
// new batch only re-uploads the descriptors and replays the graph.
//
// Serving (ecc_submit / ecc_poll): a scheduler thread admits requests while
// their device memory fits under the cap, launches the admitted ones as a
// batch on one of two slots (two streams), and keeps launching new batches
// while earlier ones run (continuous batching). Completion is detected by
// events; a request's curve stays in place in the pinned slab its batch's
// records were copied to (ecc_poll hands it out), device memory returns to
// the cap. A
// request larger than the ring is streamed through it in z-slabs on two
// streams of its own, alongside the batches.
#include "ecc_bits.cuh"
#include "ecc_scan.cuh"
#include "ecc_tile.cuh"
#include "engine.h"

#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>
#include <system_error>

namespace ecc {

int bits_nb(int dtype, int64_t bins);  // k_bits.cu

struct BImage {
  const void* img;
  long long* vcec;
  long long* curve;
  int* err;
  int64_t n[3];  // z, y, x
  int64_t bins;
  int64_t row_pitch;  // bytes (bit-sliced images)
  int64_t tiles_x, tiles_y, zc;  // generic tiling
  BitsGeo geo;        // bit-sliced tiling
  int dtype;
  int nb;             // 0: generic kernel; 8 / 14 / 16: bit-sliced kernel
};

struct BItem {
  int image;
  int pad;
  int64_t tile_lo, tile_hi;
};

struct BHeader {
  int n_images;
  int n_items_bits, n_items_gen;
  int n_chunks_b;  // chunks of the bit-sliced work list (runs of items of about equal cost)
  int next_b;      // next chunk to claim; 0 in every uploaded descriptor
};

constexpr int kMaxBatch = 1024;
constexpr int64_t kSmallBins = 256;
constexpr int kBatchBitsWarps = 8;
constexpr int kBatchPlRec = 17;  // odd and >= 16 + 1 planes
constexpr int kBatchMinDepth = 4;  // planes per tile of the thinnest batched tiles
constexpr int kZeroThreads = 1024;  // threads clearing one image's VCEC
constexpr int kGrabPerBlock = 4;  // bit-sliced work-list chunks per persistent block

namespace {

struct DescLayout {
  size_t hdr = 0, imgs = 0, items_b = 0, starts_b = 0, items_g = 0, starts_g = 0, total = 0;
  int item_cap_b = 0, item_cap_g = 0, grid_b = 0, grid_g = 0;
};

DescLayout desc_layout(int grid_b, int grid_g) {
  auto up = [](size_t x) { return (x + 255) & ~size_t(255); };
  DescLayout L;
  L.grid_b = grid_b;
  L.grid_g = grid_g;
  L.item_cap_b = kMaxBatch + grid_b * kGrabPerBlock + 1;
  L.item_cap_g = kMaxBatch + grid_g + 1;
  size_t o = 0;
  L.hdr = o; o += up(sizeof(BHeader));
  L.imgs = o; o += up(sizeof(BImage) * kMaxBatch);
  L.items_b = o; o += up(sizeof(BItem) * L.item_cap_b);
  L.starts_b = o; o += up(sizeof(int) * (grid_b * kGrabPerBlock + 1));
  L.items_g = o; o += up(sizeof(BItem) * L.item_cap_g);
  L.starts_g = o; o += up(sizeof(int) * (grid_g + 1));
  L.total = o;
  return L;
}

// ---- batched generic kernel (images the bit-sliced kernel does not take) ----
template <int CONV, int SMEM_BINS>
__global__ void __launch_bounds__(kTileThreads)
k_batch3(const unsigned char* __restrict__ desc, DescLayout L) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* ring = reinterpret_cast<uint32_t*>(smem);
  int8_t* g2 = reinterpret_cast<int8_t*>(ring + 4 * kT3PL);
  int* hist = reinterpret_cast<int*>(g2 + 256);
  const BImage* imgs = reinterpret_cast<const BImage*>(desc + L.imgs);
  const BItem* items = reinterpret_cast<const BItem*>(desc + L.items_g);
  const int* starts = reinterpret_cast<const int*>(desc + L.starts_g);
  const int i0 = starts[blockIdx.x], i1 = starts[blockIdx.x + 1];
  if (i0 >= i1) return;
  g2[threadIdx.x] = (int8_t)g2_entry(threadIdx.x);
  for (int b = threadIdx.x; b < SMEM_BINS; b += kTileThreads) hist[b] = 0;
  __syncthreads();
  for (int it = i0; it < i1; ++it) {
    const BItem item = items[it];
    const BImage& im = imgs[item.image];
    Sink s;
    s.bins = im.bins;
    s.vcec = im.vcec;
    s.hist = hist;
    s.err = im.err;
    const bool smem_hist = im.bins <= SMEM_BINS;
    const int64_t txy = im.tiles_x * im.tiles_y;
    for (int64_t t = item.tile_lo; t < item.tile_hi; ++t) {
      const int64_t tz = t / txy, rem = t - tz * txy;
      const int64_t y0 = (rem / im.tiles_x) * kT3Y, x0 = (rem % im.tiles_x) * kT3X;
      const int64_t z0 = tz * im.zc, z1 = min(z0 + im.zc, im.n[0]);
      if (im.dtype == kU8) {
        const uint8_t* p = static_cast<const uint8_t*>(im.img);
        if (smem_hist)
          run_tile3<uint8_t, CONV, kSmemHist>(p, im.n[0], im.n[1], im.n[2], 0, im.n[0], x0, y0,
                                              z0, z1, ring, g2, s);
        else
          run_tile3<uint8_t, CONV, kGlobalHist>(p, im.n[0], im.n[1], im.n[2], 0, im.n[0], x0,
                                                y0, z0, z1, ring, g2, s);
      } else {
        const uint16_t* p = static_cast<const uint16_t*>(im.img);
        if (smem_hist)
          run_tile3<uint16_t, CONV, kSmemHist>(p, im.n[0], im.n[1], im.n[2], 0, im.n[0], x0, y0,
                                               z0, z1, ring, g2, s);
        else
          run_tile3<uint16_t, CONV, kGlobalHist>(p, im.n[0], im.n[1], im.n[2], 0, im.n[0], x0,
                                                 y0, z0, z1, ring, g2, s);
      }
    }
    if (smem_hist) flush_smem_hist(s);
  }
}

// ---- batched bit-sliced kernel ----------------------------------------------
template <int CONV, int NB, int HM>
__device__ void bits_item(const BImage& im, const BItem& item, uint32_t* pl, uint32_t* g0,
                          uint32_t* g1, int* hist) {
  BitsImg bi;
  bi.img = static_cast<const unsigned char*>(im.img);
  bi.n[0] = im.n[0];
  bi.n[1] = im.n[1];
  bi.n[2] = im.n[2];
  bi.row_pitch = im.row_pitch;
  bi.w_lo = 0;
  bi.w_hi = im.n[0];
  bi.w_mem_lo = 0;
  bi.w_mem_hi = im.n[0];
  bi.bins = im.bins;
  bi.vcec = im.vcec;
  bi.err = im.err;
  bi.curve = nullptr;
  bi.done = nullptr;
  for (int64_t t = item.tile_lo; t < item.tile_hi; ++t)
    bits_tile<NB, CONV, HM>(bi, im.geo, t, pl, g0, g1, kBatchPlRec, hist);
}

// Adds the block's shared histogram into the image's VCEC and clears it.
__device__ __forceinline__ void flush_bits_hist(const BImage& im, int* hist) {
  __syncthreads();
  for (int64_t b = threadIdx.x; b < im.bins; b += blockDim.x) {
    const int v = hist[b];
    if (v) {
      atomicAdd(reinterpret_cast<unsigned long long*>(im.vcec) + b,
                (unsigned long long)(long long)v);
      hist[b] = 0;
    }
  }
  __syncthreads();
}

// Persistent blocks claim chunks of the work list in order through the
// header's counter, so that a block whose chunks ran fast takes more of them.
// A block's shared histogram is flushed when its next item belongs to
// another image and after its last chunk.
template <int CONV, int SMEM_BINS>
__global__ void __launch_bounds__(32 * kBatchBitsWarps, 2)
k_batch_bits(unsigned char* __restrict__ desc, DescLayout L) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int s_chunk;
  const int recs = 32 * kBatchBitsWarps;
  uint32_t* pl = sm;
  uint32_t* g0 = pl + recs * kBatchPlRec;
  uint32_t* g1 = g0 + recs * kBitsG0Rec;
  int* hist = reinterpret_cast<int*>(g1 + 2 * recs * kBitsG1Rec);
  BHeader* hdr = reinterpret_cast<BHeader*>(desc + L.hdr);
  const BImage* imgs = reinterpret_cast<const BImage*>(desc + L.imgs);
  const BItem* items = reinterpret_cast<const BItem*>(desc + L.items_b);
  const int* starts = reinterpret_cast<const int*>(desc + L.starts_b);
  const int n_chunks = hdr->n_chunks_b;
  if (n_chunks <= 0) return;
  for (int b = threadIdx.x; b < SMEM_BINS; b += blockDim.x) hist[b] = 0;
  int cur = -1;  // image whose counts sit in the shared histogram
  for (;;) {
    if (threadIdx.x == 0) s_chunk = atomicAdd(&hdr->next_b, 1);
    __syncthreads();
    const int c = s_chunk;
    __syncthreads();
    if (c >= n_chunks) break;
    for (int it = starts[c]; it < starts[c + 1]; ++it) {
      const BItem item = items[it];
      const BImage& im = imgs[item.image];
      const bool smem_hist = im.bins <= SMEM_BINS;
      if (cur >= 0 && cur != item.image) {
        flush_bits_hist(imgs[cur], hist);
        cur = -1;
      }
      if (smem_hist) {
        cur = item.image;
        if (im.nb == 8) bits_item<CONV, 8, kBitsSmem>(im, item, pl, g0, g1, hist);
        else if (im.nb == 14) bits_item<CONV, 14, kBitsSmem>(im, item, pl, g0, g1, hist);
        else bits_item<CONV, 16, kBitsSmem>(im, item, pl, g0, g1, hist);
      } else {
        if (im.nb == 8) bits_item<CONV, 8, kBitsGlobal>(im, item, pl, g0, g1, hist);
        else if (im.nb == 14) bits_item<CONV, 14, kBitsGlobal>(im, item, pl, g0, g1, hist);
        else bits_item<CONV, 16, kBitsGlobal>(im, item, pl, g0, g1, hist);
      }
    }
  }
  if (cur >= 0) flush_bits_hist(imgs[cur], hist);
}

// Copies a batch's work list from the slot's pinned host buffer (mapped into
// the device's address space) into device memory with the SMs, so that it
// does not queue on the copy engine behind request images being uploaded.
__global__ void __launch_bounds__(256)
k_desc_pull(uint4* __restrict__ dst, const uint4* __restrict__ src, int64_t n16) {
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n16; i += (int64_t)gridDim.x * 256)
    dst[i] = src[i];
}

// Clears image blockIdx.x's VCEC (16-byte stores where it is 16-byte
// aligned) and error word.
__global__ void __launch_bounds__(kZeroThreads)
k_batch_zero(const unsigned char* __restrict__ desc, DescLayout L) {
  const BHeader* hdr = reinterpret_cast<const BHeader*>(desc + L.hdr);
  if ((int)blockIdx.x >= hdr->n_images) return;
  const BImage& im = reinterpret_cast<const BImage*>(desc + L.imgs)[blockIdx.x];
  long long* v = im.vcec;
  int64_t b0 = 0;
  if ((reinterpret_cast<uintptr_t>(v) & 15u) == 0) {
    longlong2* v2 = reinterpret_cast<longlong2*>(v);
    const int64_t n2 = im.bins / 2;
    for (int64_t i = threadIdx.x; i < n2; i += blockDim.x) v2[i] = make_longlong2(0, 0);
    b0 = 2 * n2;
  }
  for (int64_t b = b0 + threadIdx.x; b < im.bins; b += blockDim.x) v[b] = 0;
  if (threadIdx.x == 0) *im.err = 0;
}

__global__ void __launch_bounds__(kScanThreads)
k_batch_scan(const unsigned char* __restrict__ desc, DescLayout L) {
  const BHeader* hdr = reinterpret_cast<const BHeader*>(desc + L.hdr);
  if ((int)blockIdx.x >= hdr->n_images) return;
  const BImage& im = reinterpret_cast<const BImage*>(desc + L.imgs)[blockIdx.x];
  block_scan_curve(im.vcec, im.curve, im.bins);
}

template <int SMEM_BINS>
size_t gen_smem() { return 4 * kT3PL * 4 + 256 + sizeof(int) * SMEM_BINS; }

template <int SMEM_BINS>
size_t bits_smem() {
  const size_t recs = 32 * kBatchBitsWarps;
  return recs * (kBatchPlRec + kBitsG0Rec + 2 * kBitsG1Rec) * 4 + sizeof(int) * SMEM_BINS;
}

}  // namespace

// One launch slot: stream, descriptor buffers, per-image arena and the two
// captured graphs (small histograms <= 256 bins, large <= 16384 bins).
struct Slot {
  cudaStream_t stream = nullptr;
  DescLayout L;
  DevBuf desc;
  unsigned char* h_desc = nullptr;
  void* h_desc_dev = nullptr;  // h_desc as the device sees it (mapped pinned memory)
  DevBuf arena;
  unsigned char* h_arena = nullptr;
  size_t h_arena_cap = 0;
  std::vector<unsigned char*> h_retired;  // outgrown pinned arenas, freed with the slot
  DevBuf staging;  // device copies of the batch's host images (dense rows)
  cudaGraphExec_t exec_small = nullptr, exec_large = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;  // around the graph, for the online tuner
  std::vector<size_t> res_off;             // byte offset of each image's curve in h_arena
  std::vector<ResultBlock*> blocks;        // result blocks of ecc_compute_batch (one
                                           // reference each held by the slot)
  int tune_cand = -1;                      // candidate timed by the last run, or -1
  double tune_vox = 0;                     // its bit-sliced voxels
};

// Online tuner of the batched bit-sliced kernel's planes per tile (its
// z-march depth): while undecided, successive batches take the candidates in
// turn, each run timed by events around the graph; once every candidate has
// kTrials runs, the one with the highest voxel rate is kept for the engine's
// later batches. ECC_BATCH_ZC fixes the depth instead.
struct BatchTune {
  static constexpr int kCands = 3;
  static constexpr int kTrials = 2;
  static constexpr int kDepth[kCands] = {16, 32, 64};
  double vox[kCands] = {}, ms[kCands] = {};
  int runs[kCands] = {};
  int chosen = -1;
  int next = 0;
  int fixed = 0;  // planes per tile from ECC_BATCH_ZC, 0 = tune
};

struct BatchEngine {
  std::vector<Slot> slots;
  BatchTune tune;
  cudaEvent_t staged = nullptr;  // ecc_compute_batch: host images staged on slot 0's stream
  BatchEngine() {
    if (const char* z = std::getenv("ECC_BATCH_ZC")) tune.fixed = std::max(0, std::atoi(z));
  }
};

namespace {

struct ImgSpec {
  const void* d_img;
  int64_t n[3];
  int dtype;
  int64_t bins;
  int64_t row_pitch;  // bytes between rows of d_img (0 = dense)
};

template <int CONV>
cudaError_t capture_graph(Slot& sl, bool large, cudaGraphExec_t* out) {
  cudaError_t e;
  cudaGraph_t g = nullptr;
  unsigned char* d = sl.desc.as<unsigned char>();
  if ((e = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal))) return e;
  k_batch_zero<<<kMaxBatch, kZeroThreads, 0, sl.stream>>>(d, sl.L);
  if (large) {
    k_batch_bits<CONV, kSmemBinsMax><<<sl.L.grid_b, 32 * kBatchBitsWarps,
                                       bits_smem<kSmemBinsMax>(), sl.stream>>>(d, sl.L);
    k_batch3<CONV, kSmemBinsMax><<<sl.L.grid_g, kTileThreads, gen_smem<kSmemBinsMax>(),
                                   sl.stream>>>(d, sl.L);
  } else {
    k_batch_bits<CONV, kSmallBins><<<sl.L.grid_b, 32 * kBatchBitsWarps, bits_smem<kSmallBins>(),
                                     sl.stream>>>(d, sl.L);
    k_batch3<CONV, kSmallBins><<<sl.L.grid_g, kTileThreads, gen_smem<kSmallBins>(),
                                 sl.stream>>>(d, sl.L);
  }
  k_batch_scan<<<kMaxBatch, kScanThreads, 0, sl.stream>>>(d, sl.L);
  e = cudaStreamEndCapture(sl.stream, &g);
  if (e) return e;
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  return e;
}

// Resident blocks of each batched contribution kernel (the large-histogram
// variants, which fit the fewest blocks, fix the persistent grid sizes).
template <int CONV>
cudaError_t grids_for(int num_sms, int* grid_b, int* grid_g) {
  cudaError_t e;
  auto kbs = k_batch_bits<CONV, kSmallBins>;
  auto kbl = k_batch_bits<CONV, kSmemBinsMax>;
  auto kgs = k_batch3<CONV, kSmallBins>;
  auto kgl = k_batch3<CONV, kSmemBinsMax>;
  if ((e = cudaFuncSetAttribute(kbs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bits_smem<kSmallBins>())) ||
      (e = cudaFuncSetAttribute(kbl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bits_smem<kSmemBinsMax>())) ||
      (e = cudaFuncSetAttribute(kgs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gen_smem<kSmallBins>())) ||
      (e = cudaFuncSetAttribute(kgl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)gen_smem<kSmemBinsMax>())))
    return e;
  int pb = 0, pg = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pb, kbl, 32 * kBatchBitsWarps,
                                                         bits_smem<kSmemBinsMax>())) ||
      (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pg, kgl, kTileThreads,
                                                         gen_smem<kSmemBinsMax>())))
    return e;
  *grid_b = std::max(pb, 1) * num_sms;
  *grid_g = std::max(pg, 1) * num_sms;
  return cudaSuccess;
}

// blocking: the slot's stream synchronises with the legacy default stream
// (ecc_compute_batch, whose device images may come from there); the serving
// slots take host images only and stay non-blocking.
int slot_init(ecc_handle* h, Slot& sl, bool blocking) {
  cudaError_t e;
  int gb = 0, gg = 0;
  e = h->cfg.convention == kConvT ? grids_for<kConvT>(h->num_sms, &gb, &gg)
                                  : grids_for<kConvV>(h->num_sms, &gb, &gg);
  if (e) return cuda_err(h, e, "batch occupancy");
  sl.L = desc_layout(gb, gg);
  if ((e = cudaStreamCreateWithFlags(&sl.stream,
                                     blocking ? cudaStreamDefault : cudaStreamNonBlocking)) ||
      (e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) ||
      (e = cudaEventCreate(&sl.t0)) || (e = cudaEventCreate(&sl.t1)) ||
      (e = sl.desc.ensure(sl.L.total)) || (e = cudaMallocHost(&sl.h_desc, sl.L.total)) ||
      (e = cudaHostGetDevicePointer(&sl.h_desc_dev, sl.h_desc, 0)))
    return cuda_err(h, e, "batch slot");
  std::memset(sl.h_desc, 0, sl.L.total);
  return ECC_OK;
}

void slot_free(Slot& sl) {
  if (sl.stream) cudaStreamSynchronize(sl.stream);
  if (sl.exec_small) cudaGraphExecDestroy(sl.exec_small);
  if (sl.exec_large) cudaGraphExecDestroy(sl.exec_large);
  if (sl.h_desc) cudaFreeHost(sl.h_desc);
  if (sl.h_arena) cudaFreeHost(sl.h_arena);
  for (unsigned char* p : sl.h_retired) cudaFreeHost(p);
  for (ResultBlock* b : sl.blocks) result_block_release(b);
  sl.blocks.clear();
  sl.desc.release();
  sl.arena.release();
  sl.staging.release();
  if (sl.done) cudaEventDestroy(sl.done);
  if (sl.t0) cudaEventDestroy(sl.t0);
  if (sl.t1) cudaEventDestroy(sl.t1);
  if (sl.stream) cudaStreamDestroy(sl.stream);
  sl = Slot();
}

// Per-image arena record: vcec[bins], curve[bins], err word.
size_t arena_bytes(int64_t bins) { return sizeof(long long) * (2 * bins + 1); }

// Bit-sliced kernel for this image? (any row alignment)
int image_nb(const ecc_handle* h, const ImgSpec& sp) {
  if (h->variant == 1) return 0;
  const int nb = bits_nb(sp.dtype, sp.bins);
  if (!nb) return 0;
  const uintptr_t eb = sp.dtype == kU8 ? 1 : 2;
  if ((reinterpret_cast<uintptr_t>(sp.d_img) & (eb - 1)) != 0) return 0;
  return nb;
}

// Splits tiles[i] tiles of cost cost[i] (images in order) into per-block
// contiguous item ranges of about equal work.
int partition(const std::vector<int>& img_of, const std::vector<int64_t>& tiles,
              const std::vector<int64_t>& cost, int grid, BItem* items, int item_cap,
              int* starts) {
  double total = 0;
  for (size_t j = 0; j < tiles.size(); ++j) total += (double)tiles[j] * cost[j];
  const double per_block = total / grid;
  int n_items = 0, b = 0;
  double acc = 0;
  starts[0] = 0;
  for (size_t j = 0; j < tiles.size(); ++j) {
    int64_t t = 0;
    while (t < tiles[j]) {
      const double room = per_block * (b + 1) - acc;
      int64_t k = std::max<int64_t>(1, (int64_t)(room / cost[j] + 0.999));
      k = std::min(k, tiles[j] - t);
      if (n_items >= item_cap) return -1;
      items[n_items++] = BItem{img_of[j], 0, t, t + k};
      t += k;
      acc += (double)k * cost[j];
      while (b < grid - 1 && acc >= per_block * (b + 1) - 1e-9) starts[++b] = n_items;
    }
  }
  while (b < grid) starts[++b] = n_items;
  return n_items;
}

// Fills the slot's host descriptors for `specs`, uploads them, replays the
// captured graph and copies curves and error words to the slot's pinned
// arena; the slot's `done` event marks completion.
// Books the timing of the slot's previous run (complete: a slot is reused
// only after its done event) and picks the depth of the next run.
int tune_depth(BatchTune& t, Slot& sl) {
  if (sl.tune_cand >= 0) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, sl.t0, sl.t1) == cudaSuccess && ms > 0 && t.chosen < 0) {
      t.vox[sl.tune_cand] += sl.tune_vox;
      t.ms[sl.tune_cand] += ms;
      ++t.runs[sl.tune_cand];
      bool all = true;
      for (int i = 0; i < BatchTune::kCands; ++i) all = all && t.runs[i] >= BatchTune::kTrials;
      if (all) {
        int best = 0;
        for (int i = 1; i < BatchTune::kCands; ++i)
          if (t.vox[i] / t.ms[i] > t.vox[best] / t.ms[best]) best = i;
        t.chosen = best;
      }
    }
    cudaGetLastError();
    sl.tune_cand = -1;
  }
  if (t.fixed > 0) return t.fixed;
  if (t.chosen >= 0) return BatchTune::kDepth[t.chosen];
  sl.tune_cand = t.next;
  t.next = (t.next + 1) % BatchTune::kCands;
  return BatchTune::kDepth[sl.tune_cand];
}

// A batch that does not take part in the depth tuning gives its candidate
// back, so the rotation skips none.
void untune_depth(BatchTune& t, Slot& sl) {
  if (sl.tune_cand < 0) return;
  t.next = sl.tune_cand;
  sl.tune_cand = -1;
}

// h_res: pinned destination of the (curve, error word) records, at the
// offsets sl.res_off (results_bytes(specs) bytes); null = the slot's own
// pinned arena.
int slot_run(ecc_handle* h, Slot& sl, BatchTune& tune, const std::vector<ImgSpec>& specs,
             cudaEvent_t wait_ev, unsigned char* h_res = nullptr, bool profile = false) {
  cudaError_t e;
  const int n = (int)specs.size();
  int depth = tune_depth(tune, sl);
  // A batch too small to give every block a tile at that depth takes thinner
  // tiles (more of them, each with one priming plane more), down to
  // kBatchMinDepth planes: a lone small request then runs on many blocks
  // instead of marching through all its planes on a few. Such a batch is not
  // used to tune the depth.
  auto bits_tiles = [&](int64_t d) {
    int64_t t = 0;
    for (const ImgSpec& sp : specs) {
      if (sp.n[0] * sp.n[1] * sp.n[2] == 0 || !image_nb(h, sp)) continue;
      const int64_t zc = std::min<int64_t>(d, std::max<int64_t>(sp.n[0], 1));
      t += bits_geo(sp.n[2], sp.n[1], sp.n[0], kBatchBitsWarps, zc).n_tiles;
    }
    return t;
  };
  if (tune.fixed == 0 && bits_tiles(depth) < sl.L.grid_b) {
    while (depth > kBatchMinDepth && bits_tiles(depth) < sl.L.grid_b) depth /= 2;
    untune_depth(tune, sl);
  }
  double bits_vox = 0;
  bool large = false;
  // device arena: all VCECs, then all (curve, error word) records, so that
  // only the second part is copied back
  // (each record: a 16-byte header the host fills, the curve, the error word)
  size_t vcec_total = 0, res_total = 0;
  sl.res_off.resize(n);
  for (int i = 0; i < n; ++i) {
    const ImgSpec& sp = specs[i];
    if (sp.bins > kSmallBins && sp.bins <= kSmemBinsMax) large = true;
    vcec_total += sizeof(long long) * sp.bins;
    sl.res_off[i] = res_total + kResultHeader;
    res_total += kResultHeader + sizeof(long long) * (sp.bins + 1);
  }
  // Arenas grow geometrically and without waiting for the device: the device
  // one in stream order on the slot's stream (a plain free would wait for
  // every copy and batch in flight), the pinned one keeping its outgrown
  // buffers until the slot is freed.
  const size_t arena_total = vcec_total + res_total;
  if (arena_total > sl.arena.cap || !sl.arena.p) {
    const size_t want = std::max(arena_total, 2 * sl.arena.cap);
    if (sl.arena.p) cudaFreeAsync(sl.arena.p, sl.stream);
    sl.arena.p = nullptr;
    sl.arena.cap = 0;
    if ((e = cudaMallocAsync(&sl.arena.p, want, sl.stream))) return cuda_err(h, e, "batch arena");
    sl.arena.cap = want;
  }
  if (!h_res && sl.h_arena_cap < res_total) {
    const size_t want = std::max(res_total, 2 * sl.h_arena_cap);
    unsigned char* p = nullptr;
    if ((e = cudaMallocHost(&p, want))) return cuda_err(h, e, "pinned arena");
    if (sl.h_arena) sl.h_retired.push_back(sl.h_arena);
    sl.h_arena = p;
    sl.h_arena_cap = want;
  }
  BHeader* hdr = reinterpret_cast<BHeader*>(sl.h_desc + sl.L.hdr);
  BImage* imgs = reinterpret_cast<BImage*>(sl.h_desc + sl.L.imgs);
  std::vector<int> ib, ig;
  std::vector<int64_t> tb, cb, tg, cg;
  size_t off = 0;
  char* abase = static_cast<char*>(sl.arena.p);
  for (int i = 0; i < n; ++i) {
    const ImgSpec& sp = specs[i];
    BImage& im = imgs[i];
    std::memset(&im, 0, sizeof im);
    im.img = sp.d_img;
    im.n[0] = sp.n[0];
    im.n[1] = sp.n[1];
    im.n[2] = sp.n[2];
    im.bins = sp.bins;
    im.dtype = sp.dtype;
    im.vcec = reinterpret_cast<long long*>(abase + off);
    im.curve = reinterpret_cast<long long*>(abase + vcec_total + sl.res_off[i]);
    im.err = reinterpret_cast<int*>(im.curve + sp.bins);
    off += sizeof(long long) * sp.bins;
    const int64_t vox = sp.n[0] * sp.n[1] * sp.n[2];
    if (vox == 0) continue;
    im.nb = image_nb(h, sp);
    if (im.nb) {
      const int64_t eb = sp.dtype == kU8 ? 1 : 2;
      im.row_pitch = sp.row_pitch > 0 ? sp.row_pitch : sp.n[2] * eb;
      const int64_t zc = std::min<int64_t>(depth, std::max<int64_t>(sp.n[0], 1));
      im.geo = bits_geo(sp.n[2], sp.n[1], sp.n[0], kBatchBitsWarps, zc);
      bits_vox += (double)vox;
      const int64_t width = im.geo.modeB ? 1024 : 32 * im.geo.L;
      ib.push_back(i);
      tb.push_back(im.geo.n_tiles);
      // logic work grows with the value planes: ~9 ops per voxel at 8 bits,
      // ~14 at 14, ~16 at 16 (plus one priming plane per tile)
      const int64_t weight = im.nb == 8 ? 9 : im.nb == 14 ? 14 : 16;
      cb.push_back((im.geo.zc + 1) * im.geo.RB * width * weight);
    } else {
      im.tiles_x = (sp.n[2] + kT3X - 1) / kT3X;
      im.tiles_y = (sp.n[1] + kT3Y - 1) / kT3Y;
      im.zc = std::min<int64_t>(16, std::max<int64_t>(sp.n[0], 1));
      const int64_t tz = (sp.n[0] + im.zc - 1) / im.zc;
      ig.push_back(i);
      tg.push_back(im.tiles_x * im.tiles_y * tz);
      cg.push_back((int64_t)kT3X * kT3Y * (im.zc + 2) * 12 * 9);  // generic: ~12x per voxel
    }
  }
  BItem* items_b = reinterpret_cast<BItem*>(sl.h_desc + sl.L.items_b);
  BItem* items_g = reinterpret_cast<BItem*>(sl.h_desc + sl.L.items_g);
  int* starts_b = reinterpret_cast<int*>(sl.h_desc + sl.L.starts_b);
  int* starts_g = reinterpret_cast<int*>(sl.h_desc + sl.L.starts_g);
  const int n_chunks = sl.L.grid_b * kGrabPerBlock;
  const int nib = partition(ib, tb, cb, n_chunks, items_b, sl.L.item_cap_b, starts_b);
  const int nig = partition(ig, tg, cg, sl.L.grid_g, items_g, sl.L.item_cap_g, starts_g);
  if (nib < 0 || nig < 0) return set_err(h, ECC_ERR_CUDA, "work list overflow");
  hdr->n_images = n;
  hdr->n_items_bits = nib;
  hdr->n_items_gen = nig;
  hdr->n_chunks_b = nib > 0 ? n_chunks : 0;
  hdr->next_b = 0;
  if (wait_ev && (e = cudaStreamWaitEvent(sl.stream, wait_ev, 0))) return cuda_err(h, e, "wait");
  {
    const int64_t n16 = (int64_t)(sl.L.total / 16);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(64, (n16 + 255) / 256));
    k_desc_pull<<<blocks, 256, 0, sl.stream>>>(static_cast<uint4*>(sl.desc.p),
                                               static_cast<const uint4*>(sl.h_desc_dev), n16);
    ++h->launches;
    if ((e = cudaGetLastError())) return cuda_err(h, e, "upload work list");
  }
  cudaGraphExec_t& ex = large ? sl.exec_large : sl.exec_small;
  if (!ex) {
    e = h->cfg.convention == kConvT ? capture_graph<kConvT>(sl, large, &ex)
                                    : capture_graph<kConvV>(sl, large, &ex);
    if (e) return cuda_err(h, e, "capture batch graph");
  }
  // instrumentation (profile): an event pair of the handle's profiling record
  // around the graph
  cudaEvent_t pa = nullptr, pb = nullptr;
  if (profile && (prof_event_take(h, &pa) != cudaSuccess || prof_event_take(h, &pb) != cudaSuccess)) {
    prof_event_give(h, pa);
    prof_event_give(h, pb);
    pa = pb = nullptr;
    cudaGetLastError();
  }
  if ((e = cudaEventRecord(sl.t0, sl.stream)) || (pa && (e = cudaEventRecord(pa, sl.stream))) ||
      (e = cudaGraphLaunch(ex, sl.stream)) || (pb && (e = cudaEventRecord(pb, sl.stream))) ||
      (e = cudaEventRecord(sl.t1, sl.stream))) {
    prof_event_give(h, pa);
    prof_event_give(h, pb);
    return cuda_err(h, e, "graph launch");
  }
  if (pa) h->prof_events.emplace_back(pa, pb);
  h->launches += 4;
  if (sl.tune_cand >= 0) {
    if (bits_vox > 0) sl.tune_vox = bits_vox;
    else sl.tune_cand = -1;  // nothing to learn from a batch without bit-sliced images
  }
  if ((e = cudaMemcpyAsync(h_res ? h_res : sl.h_arena, abase + vcec_total, res_total,
                           cudaMemcpyDeviceToHost, sl.stream)) ||
      (e = cudaEventRecord(sl.done, sl.stream)))
    return cuda_err(h, e, "copy results");
  return ECC_OK;
}

// Bytes of the (header, curve, error word) records of a batch.
size_t results_bytes(const std::vector<ImgSpec>& specs) {
  size_t t = 0;
  for (const ImgSpec& sp : specs) t += kResultHeader + sizeof(long long) * (sp.bins + 1);
  return t;
}

// Status of a (curve, error word) record from its error word.
int record_status(const long long* rec, int64_t bins) {
  const int err = *reinterpret_cast<const int*>(rec + bins);
  if (err & kErrValue) return ECC_ERR_VALUE;
  if (err & kErrOverflow) return ECC_ERR_CUDA;
  return ECC_OK;
}

int view3(const int64_t* dims, int ndim, int64_t n[3]) {
  n[0] = n[1] = n[2] = 1;
  for (int i = 0; i < ndim; ++i) n[3 - ndim + i] = dims[i];
  return ECC_OK;
}

// Row pitch of device copies of a (1-3D, integer) image: dense (the kernels
// read rows at any alignment).
int64_t staged_pitch(const ecc_handle*, int dtype, int64_t, int64_t nx) {
  return nx * (dtype == kU8 ? 1 : 2);
}

}  // namespace

// ---------------------------------------------------------------------------
// Serving
// ---------------------------------------------------------------------------

// Pinned host memory that receives served batches' (header, curve, error
// word) records: each batch takes one contiguous range, bump-allocated. The
// memory is a refcounted ResultBlock: a finished request's curve stays in
// place and ecc_poll hands it out (owned = 2), released by ecc_result_free.
// live counts the batches in flight on the slab (under the server lock); a
// slab with none in flight and no curve left (only the server's reference)
// starts over.
struct PinnedSlab {
  ResultBlock* blk = nullptr;
  size_t used = 0;
  int live = 0;
};
constexpr size_t kSlabBytes = size_t(64) << 20;
constexpr double kServeBatchVoxels = 256e6;

struct Request {
  enum State { kQueuedHost, kOnDevice, kLaunched, kStreaming, kDone, kFailed, kRetired };
  uint64_t id = 0;
  int64_t n[3] = {1, 1, 1};
  int dtype = kU8;
  int64_t bins = 256;
  size_t bytes = 0;       // dense host bytes
  int64_t pitch = 0;      // row pitch of the device copy (bytes)
  size_t dev_bytes = 0;   // bytes of the device copy
  std::vector<unsigned char> host_copy;
  const unsigned char* src = nullptr;  // host image: host_copy, or the caller's borrowed buffer
  void* d_img = nullptr;
  cudaEvent_t copy_done = nullptr;  // device copy still in flight on the copy stream, else null
  State state = kQueuedHost;
  int status = ECC_OK;
  int64_t* result = nullptr;
  int64_t result_bins = 0;
  long long* rec = nullptr;  // or: the curve in place in a result slab (one reference held)
  std::chrono::steady_clock::time_point t_submit, t_done;
  // stages, for ecc_request_trace_us: device copy seen finished, batch
  // launched, batch seen finished (unset: the epoch)
  std::chrono::steady_clock::time_point t_copied, t_launched, t_retired;
  int slot = -1;
  // streamed requests (device copy larger than the ring): z-slab plan
  bool streamed = false;
  int64_t sn[3] = {1, 1, 1};  // view with dims[0] as the marching axis
  int64_t depth = 0;          // planes per slab
  int ring_slots = 0;
  size_t plane_bytes = 0;
};

// A served request whose image is larger than the ring goes through the
// device in z-slabs (the streaming scheme of Sec. 3): its planes move from
// the request's host copy into a ring of slots of (depth + 2) planes on a
// copy stream, the contribution kernel runs on a slot once the next slot's
// first plane (its upper collar) is there, and the partial VCEC stays on the
// device until the last slab. The scheduler advances the job without blocking,
// so batches of other requests keep launching on the batch slots meanwhile.
struct SlabJob {
  Request* r = nullptr;
  int64_t reserved = 0;      // device bytes counted against the cap
  void* ring = nullptr;
  long long* acc = nullptr;  // VCEC (bins), curve (bins), error word
  long long* h_out = nullptr;  // pinned read-back: curve, error word
  cudaEvent_t copied[3] = {}, freed[3] = {}, done = nullptr;
  int64_t z0[3] = {}, nz[3] = {};
  bool used[3] = {};
  int64_t next_z = 0, chunks = 0;
  int pending = -1;
  bool tail = false;  // last slab, scan and read-back enqueued
};

struct Server {
  std::mutex mu;
  std::condition_variable cv;
  std::thread th;
  bool stop = false;
  uint64_t next_id = 1;
  std::deque<Request*> queue;  // waiting for a launch, FIFO
  std::map<uint64_t, Request*> all;
  int64_t bytes_in_use = 0;
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> ev_pool;  // copy-completion events for reuse
  int pending_copies = 0;            // requests with copy_done set
  std::deque<Request*> copying;      // requests whose copies were enqueued, in that order
  std::vector<PinnedSlab*> slabs;   // result slabs (freed at shutdown)
  PinnedSlab* cur_slab = nullptr;   // the slab batches allocate from
  std::vector<std::pair<PinnedSlab*, size_t>> slot_res;  // per slot: its batch's records
  BatchEngine eng;
  std::vector<std::vector<Request*>> in_flight;  // per slot
  std::vector<std::vector<ImgSpec>> specs;       // per slot
  // the streamed request in progress (one at a time) and its streams
  SlabJob* job = nullptr;
  cudaStream_t job_stream = nullptr, job_copy = nullptr;
  std::atomic<uint64_t> submitted{0};  // requests queued so far (wakes the poller)
  // voxels per served batch at most: a burst of ready requests goes out as
  // several batches on the two slots instead of one long one that every
  // request in it waits for (ECC_SERVE_BATCH_VOXELS overrides)
  double max_batch_vox = kServeBatchVoxels;
};

namespace {

int64_t request_cost(const Request* r) {
  return (int64_t)r->dev_bytes + (int64_t)arena_bytes(r->bins);
}

void free_device_image(Server* sv, Request* r) {
  if (r->d_img) {
    cudaFreeAsync(r->d_img, sv->copy_stream);
    r->d_img = nullptr;
    sv->bytes_in_use -= request_cost(r);
  }
}

// Copy-completion events from the pool (caller holds mu); null if none can
// be made.
cudaEvent_t take_event(Server* sv) {
  if (!sv->ev_pool.empty()) {
    cudaEvent_t e = sv->ev_pool.back();
    sv->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Marks r's device copy as in flight behind event e (caller holds mu).
void track_copy(Server* sv, Request* r, cudaEvent_t e) {
  r->copy_done = e;
  ++sv->pending_copies;
  sv->copying.push_back(r);
}

// Whether r's device copy has finished; returns its event to the pool when it
// has (caller holds mu). A failed copy counts as finished: the batch launch
// then reports the error.
bool copy_finished(Server* sv, Request* r) {
  if (!r->copy_done) return true;
  const cudaError_t q = cudaEventQuery(r->copy_done);
  if (q == cudaErrorNotReady) return false;
  if (q != cudaSuccess) cudaGetLastError();
  sv->ev_pool.push_back(r->copy_done);
  r->copy_done = nullptr;
  r->t_copied = std::chrono::steady_clock::now();
  --sv->pending_copies;
  return true;
}

// Retires the finished copies at the front of the copy order (caller holds
// mu), so that admission can enqueue more while both slots compute.
void reap_copies(Server* sv) {
  while (!sv->copying.empty()) {
    Request* r = sv->copying.front();
    if (r->copy_done && !copy_finished(sv, r)) break;
    sv->copying.pop_front();
  }
}

// A range of `need` bytes for one batch's records (caller holds mu): from the
// current slab, else from a slab that can start over, else null (the caller
// adds a slab). The batch holds one live count until it is retired.
PinnedSlab* take_records(Server* sv, size_t need, size_t* off) {
  need = (need + 255) & ~size_t(255);
  auto try_slab = [&](PinnedSlab* sb) {
    if (sb->live == 0 && sb->blk->refs.load(std::memory_order_acquire) == 1) sb->used = 0;
    if (sb->blk->cap - sb->used < need) return false;
    *off = sb->used;
    sb->used += need;
    ++sb->live;
    sv->cur_slab = sb;
    return true;
  };
  if (sv->cur_slab && try_slab(sv->cur_slab)) return sv->cur_slab;
  for (PinnedSlab* sb : sv->slabs)
    if (sb != sv->cur_slab && try_slab(sb)) return sb;
  return nullptr;
}

// Whether the next batch goes now (caller holds mu): at once when no batch
// is in flight, else once it holds kFillRequests requests or kFillVoxels
// voxels or its oldest request has waited kFillWaitUs, so that a stream of
// requests under load fills batches instead of launching one graph (about
// 50 us of fixed GPU time) per request or two.
constexpr int kFillRequests = 32;
constexpr double kFillVoxels = 64e6;
constexpr int64_t kFillWaitUs = 200;
bool batch_worth_launching(Server* sv) {
  bool busy = false;
  for (const auto& fl : sv->in_flight) busy = busy || !fl.empty();
  if (!busy) return true;
  int ready = 0;
  double vox = 0;
  bool in_flight_seen = false;
  auto oldest = std::chrono::steady_clock::time_point::max();
  for (Request* r : sv->queue) {
    if (r->state != Request::kOnDevice) continue;
    if (r->copy_done && (in_flight_seen || !copy_finished(sv, r))) {
      in_flight_seen = true;
      continue;
    }
    ++ready;
    vox += (double)r->n[0] * (double)r->n[1] * (double)r->n[2];
    oldest = std::min(oldest, r->t_submit);
    if (ready >= kFillRequests || vox >= kFillVoxels) return true;
  }
  return ready > 0 && std::chrono::steady_clock::now() - oldest >=
                          std::chrono::microseconds(kFillWaitUs);
}

// Copies queued on the copy stream at a time by admission: enough to keep
// the copy engine busy between two passes of the request loop, few enough
// that enqueueing never waits for room in the stream (a thread blocked there
// holds up every other thread's CUDA calls).
constexpr int kMaxPendingCopies = 64;

// Moves a host-staged request to the device if it fits under the memory cap
// and the copy limit (caller holds mu).
bool admit(ecc_handle* h, Server* sv, Request* r) {
  if (sv->bytes_in_use + request_cost(r) > h->cfg.mem_cap_bytes) return false;
  if (sv->pending_copies >= kMaxPendingCopies) return false;
  void* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, std::max<size_t>(r->dev_bytes, 1), sv->copy_stream);
  if (e) {
    cudaGetLastError();
    return false;
  }
  if (r->bytes) {
    const size_t dense = dtype_bytes(r->dtype) * (size_t)r->n[2];
    if ((size_t)r->pitch != dense)
      e = cudaMemcpy2DAsync(d, (size_t)r->pitch, r->src, dense, dense,
                            (size_t)(r->n[0] * r->n[1]), cudaMemcpyDefault, sv->copy_stream);
    else
      e = cudaMemcpyAsync(d, r->src, r->bytes, cudaMemcpyDefault,
                          sv->copy_stream);
    if (e) {
      cudaFreeAsync(d, sv->copy_stream);
      r->state = Request::kFailed;
      r->status = ECC_ERR_CUDA;
      return true;
    }
  }
  if (r->bytes) {
    cudaEvent_t ev = take_event(sv);
    if (ev && cudaEventRecord(ev, sv->copy_stream) == cudaSuccess) {
      track_copy(sv, r, ev);
    } else {
      // untracked: wait for the copy here (rare)
      cudaGetLastError();
      if (ev) sv->ev_pool.push_back(ev);
      cudaStreamSynchronize(sv->copy_stream);
    }
  }
  r->d_img = d;
  r->host_copy.clear();
  r->host_copy.shrink_to_fit();
  r->src = nullptr;
  r->state = Request::kOnDevice;
  sv->bytes_in_use += request_cost(r);
  return true;
}

// Slab plan of a request (the rule of ecc_stream_begin): dims[0] marches,
// slabs of cfg.slab_depth planes, shrunk until two slots fit the ring.
bool plan_slabs(const ecc_handle* h, Request* r, const int64_t* dims, int ndim) {
  r->sn[0] = dims[0];
  r->sn[1] = ndim >= 3 ? dims[1] : 1;
  r->sn[2] = ndim >= 2 ? dims[ndim - 1] : 1;
  r->plane_bytes = dtype_bytes(r->dtype) * (size_t)(r->sn[1] * r->sn[2]);
  const int64_t ring_planes = h->cfg.ring_bytes / (int64_t)r->plane_bytes;
  int64_t depth = std::max<int64_t>(1, h->cfg.slab_depth);
  if (ring_planes < 2 * (depth + 2)) depth = ring_planes / 2 - 2;
  if (depth < 1) return false;
  r->depth = std::min<int64_t>(depth, r->sn[0]);
  r->ring_slots = (int)std::min<int64_t>(3, ring_planes / (r->depth + 2));
  return true;
}

int64_t job_cost(const Request* r) {
  return (int64_t)r->ring_slots * (r->depth + 2) * (int64_t)r->plane_bytes +
         (int64_t)(sizeof(long long) * (2 * r->bins + 1));
}

void job_release(Server* sv, SlabJob* j) {
  cudaStreamSynchronize(sv->job_stream);
  cudaStreamSynchronize(sv->job_copy);
  for (int k = 0; k < 3; ++k) {
    if (j->copied[k]) cudaEventDestroy(j->copied[k]);
    if (j->freed[k]) cudaEventDestroy(j->freed[k]);
  }
  if (j->done) cudaEventDestroy(j->done);
  if (j->ring) cudaFreeAsync(j->ring, sv->job_stream);
  if (j->acc) cudaFreeAsync(j->acc, sv->job_stream);
  if (j->h_out) cudaFreeHost(j->h_out);
  sv->bytes_in_use -= j->reserved;
  delete j;
}

// Starts the streamed request r if its ring fits under the cap (caller holds
// mu). Returns false when it has to wait for memory.
bool job_start(ecc_handle* h, Server* sv, Request* r) {
  const int64_t cost = job_cost(r);
  if (sv->bytes_in_use + cost > h->cfg.mem_cap_bytes) return false;
  SlabJob* j = new (std::nothrow) SlabJob();
  if (!j) return false;
  j->r = r;
  j->reserved = cost;
  sv->bytes_in_use += cost;
  const size_t acc_bytes = sizeof(long long) * (2 * r->bins + 1);
  cudaError_t e = cudaMallocAsync(&j->ring, (size_t)(cost - (int64_t)acc_bytes), sv->job_stream);
  if (!e) e = cudaMallocAsync(reinterpret_cast<void**>(&j->acc), acc_bytes, sv->job_stream);
  if (!e) e = cudaMemsetAsync(j->acc, 0, acc_bytes, sv->job_stream);
  if (!e) e = cudaHostAlloc(reinterpret_cast<void**>(&j->h_out), sizeof(long long) * (r->bins + 1),
                            cudaHostAllocDefault);
  for (int k = 0; k < r->ring_slots && !e; ++k)
    if (!(e = cudaEventCreateWithFlags(&j->copied[k], cudaEventDisableTiming)))
      e = cudaEventCreateWithFlags(&j->freed[k], cudaEventDisableTiming);
  if (!e) e = cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming);
  if (e) {
    cudaGetLastError();
    job_release(sv, j);
    r->state = Request::kFailed;
    r->status = ECC_ERR_CUDA;
    r->t_done = std::chrono::steady_clock::now();
    return true;
  }
  r->state = Request::kStreaming;
  sv->job = j;
  return true;
}

// Contribution kernel over the slab held in ring slot k (planes z0 - 1 and,
// when has_upper, z0 + nz are its collars).
cudaError_t job_launch(ecc_handle* h, Server* sv, SlabJob& j, int k, bool has_upper) {
  const Request* r = j.r;
  LocalArgs a;
  a.img = static_cast<char*>(j.ring) + (size_t)k * (r->depth + 2) * r->plane_bytes;
  a.dtype = r->dtype;
  a.conv = h->cfg.convention;
  a.view = 3;
  for (int i = 0; i < 3; ++i) a.n[i] = r->sn[i];
  a.w_mem_lo = j.z0[k] - 1;
  a.w_mem_hi = j.z0[k] + j.nz[k] + (has_upper ? 1 : 0);
  a.bins = r->bins;
  a.variant = h->variant;
  a.vcec = j.acc;
  a.err = reinterpret_cast<int*>(j.acc + 2 * r->bins);
  a.stream = sv->job_stream;
  Shape s;
  s.view = 3;
  s.n[0] = r->sn[0];
  s.n[1] = r->sn[1];
  s.n[2] = r->sn[2];
  s.voxels = r->sn[0] * r->sn[1] * r->sn[2];
  const int64_t step = max_planes_per_launch(s, h->num_sms);
  cudaError_t e = cudaSuccess;
  for (int64_t w = j.z0[k]; w < j.z0[k] + j.nz[k] && !e; w += step) {
    a.w_lo = w;
    a.w_hi = std::min(w + step, j.z0[k] + j.nz[k]);
    int64_t cnt = 0;
    e = launch_local(a, h->num_sms, &cnt);
    h->launches += cnt;
  }
  if (!e) e = cudaEventRecord(j.freed[k], sv->job_stream);
  return e;
}

// Advances the streamed request without blocking on the GPU: enqueues the
// slabs whose ring slot is free, then the tail (last slab, scan, read-back),
// then retires the request once the read-back has landed. The host-to-device
// copies run with the lock released. Returns true if anything happened.
bool job_step(ecc_handle* h, Server* sv, std::unique_lock<std::mutex>& lk) {
  SlabJob& j = *sv->job;
  Request* r = j.r;
  cudaError_t e = cudaSuccess;
  bool progressed = false;
  if (j.tail) {
    const cudaError_t q = cudaEventQuery(j.done);
    if (q == cudaErrorNotReady) return false;
    r->status = ECC_OK;
    if (q != cudaSuccess) {
      cudaGetLastError();
      r->status = ECC_ERR_CUDA;
    } else {
      const int err = static_cast<int>(j.h_out[r->bins]);
      if (err & kErrValue) r->status = ECC_ERR_VALUE;
      else if (err & kErrOverflow) r->status = ECC_ERR_CUDA;
    }
    if (r->status == ECC_OK) {
      r->result = static_cast<int64_t*>(std::malloc(sizeof(int64_t) * r->bins));
      if (r->result) std::memcpy(r->result, j.h_out, sizeof(int64_t) * r->bins);
      else r->status = ECC_ERR_OOM;
      r->result_bins = r->bins;
    }
    r->state = r->status == ECC_OK ? Request::kDone : Request::kFailed;
    r->t_done = std::chrono::steady_clock::now();
    r->host_copy.clear();
    r->host_copy.shrink_to_fit();
    r->src = nullptr;
    sv->job = nullptr;
    job_release(sv, &j);
    return true;
  }
  const int R = r->ring_slots;
  while (j.next_z < r->sn[0] && !e) {
    const int k = (int)(j.chunks % R);
    if (j.used[k]) {
      const cudaError_t q = cudaEventQuery(j.freed[k]);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        e = q;
        break;
      }
    }
    const int64_t cnz = std::min<int64_t>(r->depth, r->sn[0] - j.next_z);
    char* base = static_cast<char*>(j.ring) + (size_t)k * (r->depth + 2) * r->plane_bytes;
    const unsigned char* src = r->src + (size_t)j.next_z * r->plane_bytes;
    lk.unlock();
    e = cudaMemcpyAsync(base + r->plane_bytes, src, (size_t)cnz * r->plane_bytes,
                        cudaMemcpyDefault, sv->job_copy);
    lk.lock();
    if (e || (e = cudaEventRecord(j.copied[k], sv->job_copy)) ||
        (e = cudaStreamWaitEvent(sv->job_stream, j.copied[k], 0)))
      break;
    j.z0[k] = j.next_z;
    j.nz[k] = cnz;
    j.used[k] = true;
    if (j.pending >= 0) {
      const int p = j.pending;
      char* pbase = static_cast<char*>(j.ring) + (size_t)p * (r->depth + 2) * r->plane_bytes;
      // collars: this slab's first plane above the previous one, its last below ours
      if ((e = cudaMemcpyAsync(pbase + (j.nz[p] + 1) * r->plane_bytes, base + r->plane_bytes,
                               r->plane_bytes, cudaMemcpyDeviceToDevice, sv->job_stream)) ||
          (e = cudaMemcpyAsync(base, pbase + j.nz[p] * r->plane_bytes, r->plane_bytes,
                               cudaMemcpyDeviceToDevice, sv->job_stream)) ||
          (e = job_launch(h, sv, j, p, true)))
        break;
    }
    j.pending = k;
    ++j.chunks;
    j.next_z += cnz;
    progressed = true;
  }
  if (!e && j.next_z == r->sn[0]) {
    int64_t cnt = 0;
    long long* vcec = j.acc;
    long long* curve = j.acc + r->bins;
    if (!(e = job_launch(h, sv, j, j.pending, false)) &&
        !(e = launch_scan(vcec, curve, r->bins, sv->job_stream, &cnt)) &&
        !(e = cudaMemcpyAsync(j.h_out, curve, sizeof(long long) * (r->bins + 1),
                              cudaMemcpyDeviceToHost, sv->job_stream)))
      e = cudaEventRecord(j.done, sv->job_stream);
    h->launches += cnt;
    j.tail = true;
    progressed = true;
  }
  if (e) {
    cudaGetLastError();
    r->state = Request::kFailed;
    r->status = ECC_ERR_CUDA;
    r->t_done = std::chrono::steady_clock::now();
    sv->job = nullptr;
    job_release(sv, &j);
    return true;
  }
  return progressed;
}

void serve_loop(ecc_handle* h) {
  Server* sv = h->server;
  cudaSetDevice(h->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  const int nslots = (int)sv->eng.slots.size();
  while (true) {
    bool progressed = false;
    // 1. retire finished batches: statuses from the error words in the
    // batch's pinned records (the curves stay there until polled), read
    // without the lock: only this thread launches and retires slots, and no
    // other thread touches a launched request before its state changes.
    for (int s = 0; s < nslots; ++s) {
      if (sv->in_flight[s].empty()) continue;
      cudaError_t q = cudaEventQuery(sv->eng.slots[s].done);
      if (q == cudaErrorNotReady) continue;
      std::vector<Request*> fl;
      fl.swap(sv->in_flight[s]);
      PinnedSlab* sb = sv->slot_res[s].first;
      const size_t base = sv->slot_res[s].second;
      sv->slot_res[s] = {nullptr, 0};
      lk.unlock();
      // statuses from the error words; a finished curve stays where the copy
      // back put it, its header naming the slab's block, and the request holds
      // a reference until ecc_poll hands it out
      for (size_t i = 0; i < fl.size(); ++i) {
        Request* r = fl[i];
        if (q != cudaSuccess) {
          r->status = ECC_ERR_CUDA;
          continue;
        }
        long long* rec = reinterpret_cast<long long*>(sb->blk->p + base + sv->eng.slots[s].res_off[i]);
        r->status = record_status(rec, r->bins);
        if (r->status == ECC_OK) {
          uint64_t* hdr = reinterpret_cast<uint64_t*>(rec) - 2;
          hdr[0] = reinterpret_cast<uint64_t>(sb->blk);
          hdr[1] = kResultMagic;
          sb->blk->refs.fetch_add(1, std::memory_order_relaxed);
          r->rec = rec;
          r->result_bins = r->bins;
        }
      }
      if (q != cudaSuccess) cudaGetLastError();
      const auto now = std::chrono::steady_clock::now();
      // images freed on the slot's stream (idle: its batch is done), not on
      // the copy stream, where a free would queue behind pending copies
      for (Request* r : fl)
        if (r->d_img) cudaFreeAsync(r->d_img, sv->eng.slots[s].stream);
      lk.lock();
      --sb->live;
      for (Request* r : fl) {
        if (r->d_img) {
          r->d_img = nullptr;
          sv->bytes_in_use -= request_cost(r);
        }
        r->t_retired = now;
        r->t_done = now;
        r->state = r->status == ECC_OK ? Request::kDone : Request::kFailed;
      }
      progressed = true;
    }
    if (sv->stop) break;
    // 2. admit host-staged requests in arrival order while memory and the
    // copy limit allow; a streamed request starts when no other one streams
    // and its ring fits
    reap_copies(sv);
    for (auto it = sv->queue.begin(); it != sv->queue.end();) {
      Request* r = *it;
      if (r->state != Request::kQueuedHost) {
        ++it;
        continue;
      }
      if (r->streamed) {
        if (sv->job) {
          ++it;
          continue;
        }
        if (!job_start(h, sv, r)) break;
        it = sv->queue.erase(it);
        progressed = true;
        continue;
      }
      if (!admit(h, sv, r)) break;
      progressed = true;
      ++it;
    }
    // 2b. advance the streamed request
    if (sv->job && job_step(h, sv, lk)) progressed = true;
    // 3. launch the admitted requests on a free slot
    int free_slot = -1;
    for (int s = 0; s < nslots; ++s)
      if (sv->in_flight[s].empty()) {
        free_slot = s;
        break;
      }
    if (free_slot >= 0 && !batch_worth_launching(sv)) free_slot = -1;
    if (free_slot >= 0) {
      // requests whose device copy has finished; copies finish in the order
      // they were enqueued, so after the first one still in flight the later
      // ones are not queried (they wait for the next round)
      std::vector<Request*> batch;
      std::vector<ImgSpec> specs;
      bool in_flight_seen = false;
      size_t rec_bytes = 0;  // the batch's result records fit one slab
      double batch_vox = 0;  // and its voxels stay under the cap (the first request always goes)
      for (auto it = sv->queue.begin(); it != sv->queue.end() && (int)batch.size() < kMaxBatch;) {
        Request* r = *it;
        if (r->state == Request::kFailed) {
          it = sv->queue.erase(it);
          continue;
        }
        if (r->state != Request::kOnDevice ||
            (r->copy_done && (in_flight_seen || !copy_finished(sv, r)))) {
          in_flight_seen = in_flight_seen || r->copy_done != nullptr;
          ++it;
          continue;
        }
        const size_t rb = kResultHeader + sizeof(long long) * (r->bins + 1);
        const double rv = (double)r->n[0] * (double)r->n[1] * (double)r->n[2];
        if (!batch.empty() && (rec_bytes + rb > kSlabBytes || batch_vox + rv > sv->max_batch_vox))
          break;
        rec_bytes += rb;
        batch_vox += rv;
        batch.push_back(r);
        specs.push_back(
            ImgSpec{r->d_img, {r->n[0], r->n[1], r->n[2]}, r->dtype, r->bins, r->pitch});
        it = sv->queue.erase(it);
      }
      if (!batch.empty()) {
        // the work list is built and launched without the lock (the batch's
        // requests are launched: no other thread touches them)
        Slot& sl = sv->eng.slots[free_slot];
        for (Request* r : batch) {
          r->slot = free_slot;
          r->state = Request::kLaunched;
        }
        sv->specs[free_slot] = std::move(specs);
        // the batch's records: a range of a pinned slab (a new slab, if
        // none has room, is allocated without the lock)
        const size_t need = results_bytes(sv->specs[free_slot]);
        size_t off = 0;
        PinnedSlab* sb = take_records(sv, need, &off);
        lk.unlock();
        int rc = ECC_OK;
        std::vector<PinnedSlab*> fresh;
        if (!sb) {
          // The pool grows by a quarter (at least one slab): pinning host
          // memory takes milliseconds and holds up every request behind this
          // batch, so a pool sized by a first burst keeps headroom for the
          // different packing of the next one.
          size_t grow = 1;
          {
            std::lock_guard<std::mutex> lk2(sv->mu);
            grow = std::max<size_t>(1, sv->slabs.size() / 4);
          }
          for (size_t i = 0; i < grow; ++i) {
            PinnedSlab* f = new PinnedSlab();
            f->blk = new ResultBlock();
            f->blk->cap = std::max(kSlabBytes, i == 0 ? (need + 255) & ~size_t(255) : 0);
            if (cudaMallocHost(&f->blk->p, f->blk->cap) != cudaSuccess) {
              cudaGetLastError();
              delete f->blk;
              delete f;
              if (i == 0) rc = set_err(h, ECC_ERR_OOM, "pinned result slab");
              break;
            }
            fresh.push_back(f);
          }
        }
        if (!fresh.empty()) {
          std::lock_guard<std::mutex> lk2(sv->mu);
          for (PinnedSlab* f : fresh) sv->slabs.push_back(f);
          sb = take_records(sv, need, &off);  // fits: the first new slab is empty
        }
        if (!rc) rc = slot_run(h, sl, sv->eng.tune, sv->specs[free_slot], nullptr, sb->blk->p + off);
        lk.lock();
        if (rc) {
          if (sb) --sb->live;
          for (Request* r : batch) {
            r->state = Request::kFailed;
            r->status = rc;
            r->t_done = std::chrono::steady_clock::now();
            free_device_image(sv, r);
          }
        } else {
          const auto now = std::chrono::steady_clock::now();
          for (Request* r : batch) r->t_launched = now;
          sv->in_flight[free_slot] = std::move(batch);
          sv->slot_res[free_slot] = {sb, off};
        }
        progressed = true;
      }
    }
    if (progressed) {
      sv->cv.notify_all();
      continue;
    }
    bool busy = sv->job != nullptr || sv->pending_copies > 0;
    for (int s = 0; s < nslots; ++s) busy = busy || !sv->in_flight[s].empty();
    if (busy) {
      // work on the GPU: poll for a finished batch or a new request without
      // holding the lock, so submitting threads get it at once (a timed wait
      // would cost the timer slack, ~50 us, on every completion). in_flight
      // and job are only changed by this thread.
      const uint64_t seen = sv->submitted.load(std::memory_order_acquire);
      lk.unlock();
      for (int spin = 0; spin < 256 && !sv->job; ++spin) {
        bool finished = false;
        for (int s = 0; s < nslots && !finished; ++s)
          finished = !sv->in_flight[s].empty() &&
                     cudaEventQuery(sv->eng.slots[s].done) != cudaErrorNotReady;
        if (finished || sv->submitted.load(std::memory_order_acquire) != seen) break;
        std::this_thread::yield();
      }
      lk.lock();
    } else {
      sv->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
  }
}

int server_start(ecc_handle* h) {
  if (h->server) return ECC_OK;
  Server* sv = new (std::nothrow) Server();
  if (!sv) return set_err(h, ECC_ERR_OOM, "server");
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&sv->copy_stream, cudaStreamNonBlocking)) ||
      (e = cudaStreamCreateWithFlags(&sv->job_stream, cudaStreamNonBlocking)) ||
      (e = cudaStreamCreateWithFlags(&sv->job_copy, cudaStreamNonBlocking))) {
    delete sv;
    return cuda_err(h, e, "server streams");
  }
  sv->eng.slots.resize(2);
  for (Slot& sl : sv->eng.slots) {
    int rc = slot_init(h, sl, false);
    if (rc) {
      for (Slot& s2 : sv->eng.slots) slot_free(s2);
      delete sv;
      return rc;
    }
  }
  if (const char* v = std::getenv("ECC_SERVE_BATCH_VOXELS")) {
    const double x = std::atof(v);
    if (x > 0) sv->max_batch_vox = x;
  }
  sv->in_flight.resize(2);
  sv->specs.resize(2);
  sv->slot_res.assign(2, {nullptr, 0});
  // keep freed stream-ordered allocations cached in the pool
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, h->device) == cudaSuccess) {
    uint64_t thr = (uint64_t)h->cfg.mem_cap_bytes;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  h->server = sv;
  sv->th = std::thread(serve_loop, h);
  return ECC_OK;
}

}  // namespace

void serve_shutdown(ecc_handle* h) {
  if (h->server) {
    Server* sv = h->server;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stop = true;
    }
    sv->cv.notify_all();
    if (sv->th.joinable()) sv->th.join();
    cudaSetDevice(h->device);
    for (Slot& sl : sv->eng.slots) slot_free(sl);
    if (sv->job) job_release(sv, sv->job);
    sv->job = nullptr;
    for (auto& kv : sv->all) {
      Request* r = kv.second;
      if (r->d_img) cudaFreeAsync(r->d_img, sv->copy_stream);
      if (r->copy_done) cudaEventDestroy(r->copy_done);
      std::free(r->result);
      if (r->rec) result_block_release(
          reinterpret_cast<ResultBlock*>(reinterpret_cast<const uint64_t*>(r->rec)[-2]));
      delete r;
    }
    cudaStreamSynchronize(sv->copy_stream);
    for (cudaEvent_t e : sv->ev_pool) cudaEventDestroy(e);
    for (PinnedSlab* sb : sv->slabs) {
      result_block_release(sb->blk);  // freed now, or with the last result handed out
      delete sb;
    }
    cudaStreamDestroy(sv->copy_stream);
    cudaStreamDestroy(sv->job_stream);
    cudaStreamDestroy(sv->job_copy);
    delete sv;
    h->server = nullptr;
  }
  if (h->batch) {
    for (Slot& sl : h->batch->slots) slot_free(sl);
    if (h->batch->staged) cudaEventDestroy(h->batch->staged);
    delete h->batch;
    h->batch = nullptr;
  }
}

}  // namespace ecc

using namespace ecc;

extern "C" {

int ecc_compute_batch(ecc_handle* h, int n, const ecc_image* images, ecc_result* outs) {
  if (!h) return ECC_ERR_ARG;
  try {
    std::lock_guard<std::mutex> lk(h->api_mu);
    clear_err(h);
    if (n < 0 || (n > 0 && (!images || !outs))) return set_err(h, ECC_ERR_ARG, "bad batch");
    cudaError_t e = cudaSetDevice(h->device);
    if (e) return cuda_err(h, e, "set device");
    for (int i = 0; i < n; ++i) {
      std::memset(&outs[i], 0, sizeof(ecc_result));
      outs[i].owned = 1;
    }
    if (!h->batch) {
      h->batch = new BatchEngine();
      h->batch->slots.resize(2);
      int rc = ECC_OK;
      for (Slot& s2 : h->batch->slots)
        if (!rc) rc = slot_init(h, s2, true);
      if (rc) {
        for (Slot& s2 : h->batch->slots) slot_free(s2);
        delete h->batch;
        h->batch = nullptr;
        return rc;
      }
    }
    Slot& sl = h->batch->slots[0];
    // validate, stage host images into one device buffer
    std::vector<ImgSpec> all(n);
    std::vector<int> ok(n, 0);
    std::vector<size_t> stage_off(n, SIZE_MAX);
    std::vector<char> on_dev(n, 0);
    size_t staged = 0;
    for (int i = 0; i < n; ++i) {
      const ecc_image& im = images[i];
      Shape s;
      int rc = validate_shape(h, im.dims, im.ndim, &s);
      if (rc == ECC_OK && im.ndim > 3) rc = set_err(h, ECC_ERR_ARG, "batched images are 1-3D");
      if (rc == ECC_OK && im.dtype != ECC_U8 && im.dtype != ECC_U16)
        rc = set_err(h, ECC_ERR_DTYPE, "batched images are ECC_U8 or ECC_U16");
      const int64_t bins = im.bins > 0 ? im.bins : default_bins(h, im.dtype);
      if (rc == ECC_OK && (bins > (int64_t(1) << 24))) rc = set_err(h, ECC_ERR_ARG, "bins");
      if (rc == ECC_OK && s.voxels > 0 && !im.data) rc = set_err(h, ECC_ERR_ARG, "null image");
      outs[i].status = rc;
      if (rc) continue;
      ok[i] = 1;
      ImgSpec& sp = all[i];
      sp.dtype = im.dtype;
      sp.bins = bins;
      view3(im.dims, im.ndim, sp.n);
      sp.d_img = im.data;
      sp.row_pitch = 0;
      if (s.voxels == 0) continue;
      // host images are copied into the slot's staging buffer; device
      // images are read in place (the kernels take rows at any alignment)
      const int64_t pitch = staged_pitch(h, im.dtype, bins, sp.n[2]);
      const bool dev = is_device_ptr(h, im.data);
      on_dev[i] = dev;
      if (dev && !elem_aligned(im.data, im.dtype)) {
        outs[i].status = set_err(h, ECC_ERR_ARG, "device image not aligned to its element size");
        ok[i] = 0;
        continue;
      }
      if (!dev) {
        sp.row_pitch = pitch;
        stage_off[i] = staged;
        staged += ((size_t)pitch * (size_t)(sp.n[0] * sp.n[1]) + 255) & ~size_t(255);
      }
    }
    if (staged) {
      if ((e = sl.staging.ensure(staged))) return cuda_err(h, e, "batch staging");
      for (int i = 0; i < n; ++i) {
        if (stage_off[i] == SIZE_MAX) continue;
        ImgSpec& sp = all[i];
        const size_t dense = dtype_bytes(sp.dtype) * (size_t)sp.n[2];
        char* d = static_cast<char*>(sl.staging.p) + stage_off[i];
        const cudaMemcpyKind kind = on_dev[i] ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if ((e = cudaMemcpy2DAsync(d, (size_t)sp.row_pitch, images[i].data, dense, dense,
                                   (size_t)(sp.n[0] * sp.n[1]), kind, sl.stream)))
          return cuda_err(h, e, "copy batch image");
        sp.d_img = d;
      }
    }
    // the second slot's launches read the staged images too
    cudaEvent_t staged_ev = nullptr;
    if (staged) {
      BatchEngine* be = h->batch;
      if (!be->staged && (e = cudaEventCreateWithFlags(&be->staged, cudaEventDisableTiming)))
        return cuda_err(h, e, "event");
      if ((e = cudaEventRecord(be->staged, sl.stream))) return cuda_err(h, e, "record");
      staged_ev = be->staged;
    }
    // Chunks of kMaxBatch valid images alternate between the two slots: a
    // chunk's work list is built and launched while the previous chunk runs.
    // Results stay where the copy back put them, in a pinned block of the
    // slot: each curve is handed out in place (owned = 2) and the block is
    // reused once all of them have been freed.
    std::vector<int> idx;
    for (int i = 0; i < n; ++i)
      if (ok[i]) idx.push_back(i);
    struct Pending {
      bool active = false;
      size_t c0 = 0, c1 = 0;
      std::vector<ImgSpec> specs;
      ResultBlock* blk = nullptr;
    } pend[2];
    auto finish = [&](int si) -> int {
      Pending& pd = pend[si];
      if (!pd.active) return ECC_OK;
      pd.active = false;
      Slot& s2 = h->batch->slots[si];
      const int rc = wait_event(h, s2.done, 300LL * 1000 * 1000);
      if (rc) return rc;
      for (size_t j = pd.c0; j < pd.c1; ++j) {
        const ImgSpec& sp = pd.specs[j - pd.c0];
        unsigned char* rec = pd.blk->p + s2.res_off[j - pd.c0];
        ecc_result& o = outs[idx[j]];
        o.status = record_status(reinterpret_cast<const long long*>(rec), sp.bins);
        if (o.status != ECC_OK) continue;
        uint64_t* hdr = reinterpret_cast<uint64_t*>(rec) - 2;
        hdr[0] = reinterpret_cast<uint64_t>(pd.blk);
        hdr[1] = kResultMagic;
        pd.blk->refs.fetch_add(1, std::memory_order_relaxed);
        o.curve = reinterpret_cast<int64_t*>(rec);
        o.bins = sp.bins;
        o.owned = 2;
      }
      return ECC_OK;
    };
    // a block of the slot that no result refers to any more, else a new one
    auto take_block = [&](Slot& s2, size_t need) -> ResultBlock* {
      for (size_t b = 0; b < s2.blocks.size(); ++b) {
        ResultBlock* blk = s2.blocks[b];
        if (blk->refs.load(std::memory_order_acquire) != 1) continue;
        if (blk->cap >= need) return blk;
        result_block_release(blk);  // too small and unused: drop it
        s2.blocks.erase(s2.blocks.begin() + (long)b);
        --b;
      }
      ResultBlock* blk = new ResultBlock();
      const size_t cap = std::max(need + need / 4, size_t(1) << 20);
      if (cudaMallocHost(&blk->p, cap) != cudaSuccess) {
        cudaGetLastError();
        delete blk;
        return nullptr;
      }
      blk->cap = cap;
      s2.blocks.push_back(blk);
      return blk;
    };
    size_t chunk = 0;
    for (size_t c0 = 0; c0 < idx.size(); c0 += kMaxBatch, ++chunk) {
      const int si = (int)(chunk & 1);
      int rc = finish(si);  // the slot's previous chunk
      if (rc) return rc;
      Slot& s2 = h->batch->slots[si];
      Pending& pd = pend[si];
      pd.c0 = c0;
      pd.c1 = std::min(idx.size(), c0 + kMaxBatch);
      pd.specs.clear();
      for (size_t j = pd.c0; j < pd.c1; ++j) pd.specs.push_back(all[idx[j]]);
      pd.blk = take_block(s2, results_bytes(pd.specs));
      if (!pd.blk) return set_err(h, ECC_ERR_OOM, "pinned result block");
      rc = slot_run(h, s2, h->batch->tune, pd.specs, si == 0 ? nullptr : staged_ev, pd.blk->p,
                    h->prof_on);
      if (rc) return rc;
      pd.active = true;
    }
    for (int si = 0; si < 2; ++si) {
      const int rc = finish(si);
      if (rc) return rc;
    }
    return ECC_OK;
  } catch (const std::bad_alloc&) {
    return set_err(h, ECC_ERR_OOM, "host allocation");
  } catch (...) {
    return set_err(h, ECC_ERR_CUDA, "internal error");
  }
}

// ecc_submit (borrow = false) and ecc_submit_borrowed (borrow = true).
static int submit_request(ecc_handle* h, const void* image, const int64_t* dims, int ndim,
                          ecc_dtype dtype, uint64_t* req_id, bool borrow) {
  if (!h) return ECC_ERR_ARG;
  try {
    Shape s;
    {
      std::lock_guard<std::mutex> lk(h->api_mu);
      clear_err(h);
      if (!req_id) return set_err(h, ECC_ERR_ARG, "req_id is NULL");
      int rc = validate_shape(h, dims, ndim, &s);
      if (rc) return rc;
      if (ndim > 3) return set_err(h, ECC_ERR_ARG, "served images are 1-3D");
      if (dtype != ECC_U8 && dtype != ECC_U16)
        return set_err(h, ECC_ERR_DTYPE, "served images are ECC_U8 or ECC_U16");
      if (s.voxels > 0 && !image) return set_err(h, ECC_ERR_ARG, "image is NULL");
      cudaError_t e = cudaSetDevice(h->device);
      if (e) return cuda_err(h, e, "set device");
      rc = server_start(h);
      if (rc) return rc;
    }
    Server* sv = h->server;
    Request* r = new Request();
    r->dtype = dtype;
    r->bins = default_bins(h, dtype);
    view3(dims, ndim, r->n);
    r->bytes = dtype_bytes(dtype) * (size_t)s.voxels;
    r->pitch = staged_pitch(h, dtype, r->bins, r->n[2]);
    r->dev_bytes = (size_t)r->pitch * (size_t)(r->n[0] * r->n[1]);
    r->t_submit = std::chrono::steady_clock::now();
    if ((int64_t)r->dev_bytes > h->cfg.ring_bytes) {
      // larger than the ring: streamed through it in z-slabs
      r->streamed = true;
      if (!plan_slabs(h, r, dims, ndim) || job_cost(r) > h->cfg.mem_cap_bytes) {
        delete r;
        return set_err(h, ECC_ERR_OOM, "the slab ring of this request does not fit the cap");
      }
    } else if (request_cost(r) > h->cfg.mem_cap_bytes) {
      delete r;
      return set_err(h, ECC_ERR_OOM, "request larger than the device memory cap");
    }
    // An image in pinned host memory or in device (or managed) memory goes
    // straight to the request's device buffer by the copy engine if the cap
    // allows; without borrowing the call waits for that copy. Otherwise a
    // borrowed image is read in place later (admission, or the slabs of a
    // streamed request) and any other is copied into host memory first.
    // A borrowed request joins a batch once its copy's event has completed.
    bool pinned = false, on_dev = false;
    if (r->bytes) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, image) == cudaSuccess) {
        pinned = at.type == cudaMemoryTypeHost;
        on_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
      } else {
        cudaGetLastError();
      }
    }
    const bool direct = pinned || on_dev;  // copied asynchronously by the copy engine
    // The memory (and, when borrowing, a place in the window of copies in
    // flight) is reserved under the lock, the copy enqueued without it. A
    // borrowing caller whose window is full waits for the oldest copy in
    // flight, without the lock.
    cudaEvent_t copied = nullptr;  // the copy's completion event
    bool reserved = false;
    if (direct && !r->streamed) {
      const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(300);
      std::unique_lock<std::mutex> lk(sv->mu);
      while (sv->bytes_in_use + request_cost(r) <= h->cfg.mem_cap_bytes) {
        if (borrow) {
          reap_copies(sv);
          if (sv->pending_copies >= kMaxPendingCopies) {
            cudaEvent_t oldest = sv->copying.empty() ? nullptr : sv->copying.front()->copy_done;
            lk.unlock();
            // (the event may be recycled meanwhile: then this waits for a
            // later copy, which ends too)
            while (oldest && cudaEventQuery(oldest) == cudaErrorNotReady &&
                   std::chrono::steady_clock::now() < deadline)
              std::this_thread::yield();
            if (!oldest) std::this_thread::yield();
            cudaGetLastError();
            lk.lock();
            if (std::chrono::steady_clock::now() >= deadline) break;  // left to admission
            continue;
          }
        }
        if ((copied = take_event(sv)) == nullptr) break;
        sv->bytes_in_use += request_cost(r);
        if (borrow) ++sv->pending_copies;
        reserved = true;
        break;
      }
    }
    if (reserved) {
      void* d = nullptr;
      cudaError_t e = cudaMallocAsync(&d, r->dev_bytes, sv->copy_stream);
      if (e == cudaSuccess &&
          (e = cudaMemcpyAsync(d, image, r->bytes, cudaMemcpyDefault, sv->copy_stream)) ==
              cudaSuccess &&
          (e = cudaEventRecord(copied, sv->copy_stream)) == cudaSuccess) {
        r->d_img = d;
        r->state = Request::kOnDevice;
      } else {
        cudaGetLastError();
        if (d) cudaFreeAsync(d, sv->copy_stream);
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->ev_pool.push_back(copied);
        copied = nullptr;
        sv->bytes_in_use -= request_cost(r);
        if (borrow) --sv->pending_copies;
      }
    }
    if (copied && borrow) {
      // tracked by the request loop (counted in pending_copies above)
      r->copy_done = copied;
      copied = nullptr;
    }
    if (copied) {
      const int rc = wait_event(h, copied, 300LL * 1000 * 1000);
      r->t_copied = std::chrono::steady_clock::now();
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->ev_pool.push_back(copied);
      if (rc) {
        free_device_image(sv, r);
        delete r;
        return rc;
      }
    } else if (r->state != Request::kOnDevice) {
      if (borrow && direct) {
        r->src = static_cast<const unsigned char*>(image);
      } else {
        r->host_copy.resize(r->bytes);
        if (on_dev) {
          const cudaError_t e =
              cudaMemcpy(r->host_copy.data(), image, r->bytes, cudaMemcpyDefault);
          if (e != cudaSuccess) {
            delete r;
            return cuda_err(h, e, "copy device image");
          }
        } else if (r->bytes) {
          std::memcpy(r->host_copy.data(), image, r->bytes);
        }
        r->src = r->host_copy.data();
      }
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      r->id = sv->next_id++;
      sv->all[r->id] = r;
      if (r->copy_done) sv->copying.push_back(r);
      if (r->state == Request::kQueuedHost && !r->streamed) admit(h, sv, r);
      sv->queue.push_back(r);
      *req_id = r->id;
      sv->submitted.fetch_add(1, std::memory_order_release);
    }
    sv->cv.notify_all();
    return ECC_OK;
  } catch (const std::bad_alloc&) {
    return set_err(h, ECC_ERR_OOM, "host allocation");
  } catch (...) {
    return set_err(h, ECC_ERR_CUDA, "internal error");
  }
}

int ecc_submit(ecc_handle* h, const void* image, const int64_t* dims, int ndim, ecc_dtype dtype,
               uint64_t* req_id) {
  return submit_request(h, image, dims, ndim, dtype, req_id, false);
}

int ecc_submit_borrowed(ecc_handle* h, const void* image, const int64_t* dims, int ndim,
                        ecc_dtype dtype, uint64_t* req_id) {
  return submit_request(h, image, dims, ndim, dtype, req_id, true);
}

int ecc_poll(ecc_handle* h, uint64_t req_id, ecc_result* out, int64_t timeout_us) {
  if (!h || !out) return ECC_ERR_ARG;
  Server* sv = h->server;
  if (!sv) return ECC_ERR_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(req_id);
  if (it == sv->all.end() || it->second->state == Request::kRetired) return ECC_ERR_ARG;
  Request* r = it->second;
  auto finished = [&] { return r->state == Request::kDone || r->state == Request::kFailed; };
  if (!finished()) {
    if (timeout_us == 0) return ECC_PENDING;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
    if (!sv->cv.wait_until(lk, deadline, finished)) return ECC_ERR_TIMEOUT;
  }
  std::memset(out, 0, sizeof *out);
  out->status = r->status;
  const int rc = r->status;
  r->state = Request::kRetired;
  if (rc == ECC_OK) {
    out->bins = r->result_bins;
    if (r->rec) {
      out->owned = 2;  // in place in a result slab; the request's reference moves to out
      out->curve = reinterpret_cast<int64_t*>(r->rec);
      r->rec = nullptr;
    } else {
      out->owned = 1;
      out->curve = r->result;
      r->result = nullptr;
    }
  }
  return rc;
}

int ecc_request_trace_us(ecc_handle* h, uint64_t req_id, double* stages) {
  if (!h || !stages || !h->server) return ECC_ERR_ARG;
  Server* sv = h->server;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(req_id);
  if (it == sv->all.end()) return ECC_ERR_ARG;
  Request* r = it->second;
  if (r->state != Request::kDone && r->state != Request::kRetired && r->state != Request::kFailed)
    return ECC_ERR_ARG;
  const std::chrono::steady_clock::time_point ts[4] = {r->t_copied, r->t_launched, r->t_retired,
                                                       r->t_done};
  for (int k = 0; k < 4; ++k)
    stages[k] = ts[k].time_since_epoch().count() == 0
                    ? -1.0
                    : std::chrono::duration<double, std::micro>(ts[k] - r->t_submit).count();
  return ECC_OK;
}

int ecc_request_latency_us(ecc_handle* h, uint64_t req_id, double* us) {
  if (!h || !us || !h->server) return ECC_ERR_ARG;
  Server* sv = h->server;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(req_id);
  if (it == sv->all.end()) return ECC_ERR_ARG;
  Request* r = it->second;
  if (r->state != Request::kDone && r->state != Request::kRetired && r->state != Request::kFailed)
    return ECC_ERR_ARG;
  *us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
  return ECC_OK;
}

}  // extern "C"
