// Host engine: handle lifetime, validation, and the single-image entry points
// of the C ABI (include/ecc.h). No C++ exception crosses the ABI: every entry
// point catches and converts to a status code.
#include "engine.h"

#include <cmath>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

namespace ecc {

cudaError_t launch_local_generic(const LocalArgs& a, int num_sms, int64_t* launches);

namespace {
thread_local const ecc_handle* tl_err_h = nullptr;
thread_local std::string tl_err;
}  // namespace

int set_err(ecc_handle* h, int code, const char* fmt, ...) {
  if (h) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tl_err_h = h;
    tl_err = buf;
  }
  return code;
}

void clear_err(const ecc_handle* h) {
  if (tl_err_h == h) tl_err.clear();
}

const char* last_err(const ecc_handle* h) { return tl_err_h == h ? tl_err.c_str() : ""; }

int cuda_err(ecc_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return ECC_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_err(h, ECC_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return set_err(h, ECC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t dtype_bytes(int dtype) {
  switch (dtype) {
    case kU8: return 1;
    case kU16: return 2;
    case kF32: return 4;
    default: return 0;
  }
}

int64_t default_bins(const ecc_handle* h, int dtype) {
  if (h->cfg.bins > 0) return h->cfg.bins;
  return dtype == kU8 ? 256 : 65536;
}

int validate_shape(ecc_handle* h, const int64_t* dims, int ndim, Shape* s) {
  if (!dims) return set_err(h, ECC_ERR_ARG, "dims is NULL");
  if (ndim < 1 || ndim > 4) return set_err(h, ECC_ERR_ARG, "ndim %d outside 1..4", ndim);
  s->ndim = ndim;
  s->voxels = 1;
  for (int i = 0; i < ndim; ++i) {
    if (dims[i] < 0) return set_err(h, ECC_ERR_ARG, "dims[%d] = %lld < 0", i, (long long)dims[i]);
    if (dims[i] > (int64_t(1) << 40))
      return set_err(h, ECC_ERR_ARG, "dims[%d] too large", i);
    s->dims[i] = dims[i];
    s->voxels *= dims[i];
  }
  // kernel view: 4D stays (w, z, y, x); 1D-3D become (z, y, x) with
  // leading extents 1
  if (ndim == 4) {
    s->view = 4;
    for (int i = 0; i < 4; ++i) s->n[i] = dims[i];
  } else {
    s->view = 3;
    s->n[0] = s->n[1] = s->n[2] = s->n[3] = 1;
    for (int i = 0; i < ndim; ++i) s->n[3 - ndim + i] = dims[i];
  }
  return ECC_OK;
}

bool is_device_ptr(const ecc_handle* h, const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) &&
         at.device == h->device;
}

cudaError_t launch_local_bits(const LocalArgs& a, int num_sms, int64_t* launches);
cudaError_t launch_local_bits4(const LocalArgs& a, int num_sms, int64_t* launches);

// Kernel choice: the bit-sliced kernel where it applies (1-3D integer images
// with 256, 16384 or 65536 bins and 16-byte aligned rows), the generic kernel
// otherwise. variant 1 forces the generic kernel, 2 the bit-sliced one.
cudaError_t launch_local(const LocalArgs& a, int num_sms, int64_t* launches) {
  if (a.variant != 1) {
    cudaError_t e = a.view == 4 ? launch_local_bits4(a, num_sms, launches)
                                : launch_local_bits(a, num_sms, launches);
    if (e != cudaErrorNotSupported || a.variant == 2) return e;
    cudaGetLastError();
  }
  return launch_local_generic(a, num_sms, launches);
}

// Largest number of voxel planes (of n[0]) per contribution launch so that no
// block's int32 shared-memory histogram can overflow: a change is at most 21
// in magnitude (|G_4| <= 3 * 7), and a launch splits its voxels over at least
// `blocks` blocks of which none takes more than twice its share.
int64_t max_planes_per_launch(const Shape& s, int num_sms) {
  const int64_t per_plane = s.voxels / std::max<int64_t>(s.n[0], 1);
  const int64_t budget = (int64_t(1) << 31) / 32 * (int64_t)num_sms / 2;
  if (per_plane <= 0) return s.n[0];
  return std::max<int64_t>(1, budget / per_plane);
}

bool bits_eligible(const ecc_handle* h, const Shape& s, int dtype, int64_t bins) {
  return h->variant != 1 && s.view == 3 &&
         ((dtype == kU8 && bins == 256) || (dtype == kU16 && (bins == 16384 || bins == 65536)));
}

int stage_image(ecc_handle* h, const void* image, bool on_device, const Shape& s, int dtype,
                int64_t bins, cudaStream_t st, const void** d_img, int64_t* row_pitch) {
  (void)bins;
  *row_pitch = 0;
  *d_img = image;
  if (s.voxels == 0 || on_device) return ECC_OK;  // kernels read rows at any alignment
  const size_t bytes = dtype_bytes(dtype) * (size_t)s.voxels;
  cudaError_t e;
  if ((e = h->img.ensure(bytes))) return cuda_err(h, e, "image buffer");
  if ((e = cudaMemcpyAsync(h->img.p, image, bytes, cudaMemcpyHostToDevice, st)))
    return cuda_err(h, e, "copy image");
  *d_img = h->img.p;
  return ECC_OK;
}

// Host images of at least this many bytes are uploaded in plane chunks that
// overlap with the computation (ecc_compute): at most kUploadChunksMax equal
// chunks, the last one then cut in halves.
constexpr size_t kChunkedUploadBytes = size_t(16) << 20;
constexpr int64_t kFusedScanBins = 2048;
constexpr int64_t kUploadChunksMax = 16;
constexpr size_t kUploadChunkBytes = size_t(32) << 20;
constexpr size_t kUploadTailBytes = size_t(2) << 20;

// Uploads a host image of `bytes` into the handle's image buffer in plane
// chunks on the copy stream: equal chunks of about kUploadChunkBytes (at most
// kUploadChunksMax), the last one cut in halves down to about
// kUploadTailBytes (few copies, each with a fixed cost on the copy engine, and
// little work left once the copy has ended). ends[k] is the first plane after
// chunk k, whose arrival h->up_ev[k] marks. The copies wait for the buffer's
// earlier readers (kernels on the compute stream).
cudaError_t prof_event_take(ecc_handle* h, cudaEvent_t* ev) {
  if (!h->prof_pool.empty()) {
    *ev = h->prof_pool.back();
    h->prof_pool.pop_back();
    return cudaSuccess;
  }
  return cudaEventCreate(ev);
}

void prof_event_give(ecc_handle* h, cudaEvent_t ev) {
  if (ev) h->prof_pool.push_back(ev);
}

void result_block_release(ResultBlock* b) {
  if (b && b->refs.fetch_sub(1, std::memory_order_acq_rel) == 1) {
    cudaFreeHost(b->p);
    cudaGetLastError();
    delete b;
  }
}

int upload_chunks(ecc_handle* h, const void* image, size_t bytes, const Shape& s,
                  std::vector<int64_t>* ends) {
  cudaError_t e;
  if ((e = h->img.ensure(bytes))) return cuda_err(h, e, "image buffer");
  const int64_t plane = (int64_t)(bytes / (size_t)s.n[0]);
  const int Keq = (int)std::min<int64_t>(
      {s.n[0], kUploadChunksMax, std::max<int64_t>(2, (int64_t)(bytes / kUploadChunkBytes))});
  ends->clear();
  for (int k = 1; k < Keq; ++k) ends->push_back(s.n[0] * k / Keq);
  int64_t zt = ends->empty() ? 0 : ends->back();
  while (s.n[0] - zt >= 2 && (size_t)(s.n[0] - zt) * (size_t)plane > kUploadTailBytes) {
    zt += (s.n[0] - zt) / 2;
    ends->push_back(zt);
  }
  ends->push_back(s.n[0]);
  const int K = (int)ends->size();
  while ((int)h->up_ev.size() < K) {
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return cuda_err(h, e, "event");
    h->up_ev.push_back(ev);
  }
  if (!h->up_free && (e = cudaEventCreateWithFlags(&h->up_free, cudaEventDisableTiming)))
    return cuda_err(h, e, "event");
  if ((e = cudaEventRecord(h->up_free, h->stream)) ||
      (e = cudaStreamWaitEvent(h->copy_stream, h->up_free, 0)))
    return cuda_err(h, e, "order upload");
  for (int k = 0; k < K; ++k) {
    const int64_t z0 = k > 0 ? (*ends)[k - 1] : 0, z1 = (*ends)[k];
    char* dst = static_cast<char*>(h->img.p) + (size_t)(z0 * plane);
    const char* src = static_cast<const char*>(image) + (size_t)(z0 * plane);
    if ((e = cudaMemcpyAsync(dst, src, (size_t)((z1 - z0) * plane), cudaMemcpyHostToDevice,
                             h->copy_stream)) ||
        (e = cudaEventRecord(h->up_ev[k], h->copy_stream)))
      return cuda_err(h, e, "copy image");
  }
  return ECC_OK;
}

int enqueue_int(ecc_handle* h, const void* d_img, int64_t row_pitch, const Shape& s, int dtype,
                int64_t bins, long long* d_vcec, long long* d_curve, cudaStream_t stream,
                const int64_t* chunk_end, const cudaEvent_t* chunk_ev, int n_chunks) {
  cudaError_t e;
  // entries of d_vcec known to be zero; the buffer counts as dirty until this
  // call has enqueued a launch that leaves it clean (an early error return
  // after a partial launch sequence then forces the next call to clear it)
  int64_t clean = d_vcec == h->clean_vcec ? h->clean_bins : 0;
  h->clean_vcec = nullptr;
  if (bins > clean) {
    if ((e = cudaMemsetAsync(d_vcec, 0, sizeof(long long) * bins, stream)))
      return cuda_err(h, e, "memset vcec");
    clean = bins;
  }
  if (s.voxels > 0) {
    LocalArgs a;
    a.img = d_img;
    a.dtype = dtype;
    a.conv = h->cfg.convention;
    a.view = s.view;
    for (int i = 0; i < 4; ++i) a.n[i] = s.n[i];
    a.bins = bins;
    a.row_pitch = row_pitch;
    a.variant = h->variant;
    a.warps = h->bits_warps;
    a.zc = h->bits_zc;
    a.layout = h->bits_layout;
    a.vcec = d_vcec;
    a.err = h->errw.as<int>();
    a.stream = stream;
    a.w_mem_lo = 0;
    a.w_mem_hi = a.n[0];
    const int64_t step = max_planes_per_launch(s, h->num_sms);
    // launch shape from the tuner (first image of a shape class tunes it)
    if (h->tuner && a.view == 3 && bits_nb(dtype, bins) && h->variant != 1 &&
        h->bits_warps == 0 && h->bits_zc == 0 && h->bits_layout == 0) {
      LocalArgs t = a;
      t.w_lo = 0;
      t.w_hi = std::min(a.n[0], step);
      const std::string k = Tuner::key(t);
      TuneChoice c;
      if (!h->tuner->lookup(k, &c)) {
        // the candidates read the whole first launch's planes: all chunks first
        if (n_chunks > 0 && (e = cudaStreamWaitEvent(stream, chunk_ev[n_chunks - 1], 0)))
          return cuda_err(h, e, "wait upload");
        int rc = tune_bits(h, t, &c);
        if (rc) return rc;
        if (c.warps > 0) h->tuner->store(k, c);
        if ((e = cudaMemsetAsync(d_vcec, 0, sizeof(long long) * bins, stream)))
          return cuda_err(h, e, "memset vcec");
      }
      a.warps = c.warps;
      a.zc = c.zc;
      a.hist = c.hist;
      a.layout = c.layout;
    }
    // one bit-sliced launch over the whole image: its last block also writes
    // the curve and leaves VCEC and the block counter at zero, so neither the
    // clearing memset nor the scan launch is needed while that holds (up to
    // kFusedScanBins bins: one block scans them after all others finished,
    // which for larger histograms costs more than a separate 1024-thread scan)
    const bool fused = n_chunks == 0 && a.n[0] <= step && h->variant != 1 && a.view == 3 &&
                       bins <= kFusedScanBins &&
                       bits_nb(dtype, bins) != 0 && row_pitch == 0 &&
                       (dtype == kU8 || (reinterpret_cast<uintptr_t>(d_img) & 1u) == 0) &&
                       h->done.p != nullptr;
    if (fused) {
      a.fused_curve = d_curve;
      a.done = h->done.as<unsigned int>();
    }
    // profiling events: back to the pool on every return that does not hand
    // them to the handle's record
    struct EventPair {
      ecc_handle* h;
      cudaEvent_t a = nullptr, b = nullptr;
      ~EventPair() {
        prof_event_give(h, a);
        prof_event_give(h, b);
      }
    } prof{h};
    if (h->prof_on) {
      if ((e = prof_event_take(h, &prof.a)) || (e = prof_event_take(h, &prof.b)) ||
          (e = cudaEventRecord(prof.a, stream)))
        return cuda_err(h, e, "profiling event");
    }
    // chunk k's launches take its planes but the last (whose upper neighbour
    // is the next chunk's first plane) and the previous chunk's last plane,
    // so each waits only for its own chunk's copy
    const int K = n_chunks > 0 ? n_chunks : 1;
    for (int k = 0; k < K; ++k) {
      const int64_t lo = n_chunks > 0 && k > 0 ? chunk_end[k - 1] - 1 : 0;
      const int64_t hi = n_chunks > 0 && k < K - 1 ? chunk_end[k] - 1 : a.n[0];
      if (n_chunks > 0 && (e = cudaStreamWaitEvent(stream, chunk_ev[k], 0)))
        return cuda_err(h, e, "wait upload");
      for (int64_t w = lo; w < hi; w += step) {
        a.w_lo = w;
        a.w_hi = std::min(hi, w + step);
        int64_t cnt = 0;
        e = launch_local(a, h->num_sms, &cnt);
        h->launches += cnt;
        if (e != cudaSuccess) return cuda_err(h, e, "contribution kernel");
      }
    }
    if (h->prof_on) {
      if ((e = cudaEventRecord(prof.b, stream))) return cuda_err(h, e, "profiling event");
      h->prof_events.emplace_back(prof.a, prof.b);
      prof.a = prof.b = nullptr;
    }
    if (fused) {
      h->clean_vcec = d_vcec;
      h->clean_bins = clean;
      return ECC_OK;
    }
  }
  int64_t cnt = 0;
  e = launch_scan(d_vcec, d_curve, bins, stream, &cnt);
  h->launches += cnt;
  if (e != cudaSuccess) return cuda_err(h, e, "scan kernel");
  return ECC_OK;
}

int wait_event(ecc_handle* h, cudaEvent_t ev, int64_t timeout_us) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return ECC_OK;
    if (e != cudaErrorNotReady) return cuda_err(h, e, "event");
    const auto dt = std::chrono::duration_cast<std::chrono::microseconds>(
                        std::chrono::steady_clock::now() - t0).count();
    if (timeout_us >= 0 && dt >= timeout_us)
      return set_err(h, ECC_ERR_TIMEOUT, "wait ran out after %lld us", (long long)dt);
    // spin for the first 2 ms (a sleep costs the timer slack, ~50 us), then
    // poll every 100 us
    if (dt < 2000)
      std::this_thread::yield();
    else
      std::this_thread::sleep_for(std::chrono::microseconds(100));
  }
}

// Bounded stream synchronisation through an event (5 minutes).
static int sync_stream(ecc_handle* h, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!h->sync_ev && (e = cudaEventCreateWithFlags(&h->sync_ev, cudaEventDisableTiming)))
    return cuda_err(h, e, "event create");
  e = cudaEventRecord(h->sync_ev, s);
  return e == cudaSuccess ? wait_event(h, h->sync_ev, 300LL * 1000 * 1000) : cuda_err(h, e, "record");
}

static int read_err_word(ecc_handle* h, cudaStream_t s, int* word) {
  cudaError_t e = cudaMemcpyAsync(h->h_err, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_err(h, e, "read error word");
  int rc = sync_stream(h, s);
  if (rc) return rc;
  *word = *h->h_err;
  return ECC_OK;
}

static int err_word_status(ecc_handle* h, int word) {
  if (word & kErrValue)
    return set_err(h, ECC_ERR_VALUE, "a value is >= bins, or a float is NaN/Inf");
  if (word & kErrOverflow)
    return set_err(h, ECC_ERR_CUDA, "internal capacity exceeded (error word %d)", word);
  return ECC_OK;
}

// A pinned block of at least `need` bytes for one float image's pairs, with
// one reference for the result (and one the handle keeps): a block of the
// handle's that no result references any more, else a new one. The handle
// keeps at most kPairBlocks; a block it lets go lives on until its result is
// released.
constexpr size_t kPairBlocks = 3;
// Pair lists up to this size are copied back whole, before their surviving
// count is known (one wait instead of two).
constexpr unsigned long long kSpeculativePairBytes = 32ull << 20;
static ResultBlock* take_pair_block(ecc_handle* h, size_t need) {
  for (ResultBlock* b : h->pair_blocks) {
    // refs == 1: only the handle's reference; no other thread can add one
    if (b->cap >= need && b->refs.load(std::memory_order_acquire) == 1) {
      b->refs.fetch_add(1, std::memory_order_acq_rel);
      return b;
    }
  }
  const size_t cap = std::max<size_t>(need + need / 4, size_t(1) << 20);
  void* p = nullptr;
  if (cudaHostAlloc(&p, cap, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ResultBlock* b = new ResultBlock();
  b->p = static_cast<unsigned char*>(p);
  b->cap = cap;
  b->refs.store(2);
  if (h->pair_blocks.size() >= kPairBlocks) {
    result_block_release(h->pair_blocks.front());
    h->pair_blocks.erase(h->pair_blocks.begin());
  }
  h->pair_blocks.push_back(b);
  return b;
}

// Float pairs of an image on the device. With n_chunks > 0 the image is still
// arriving in plane chunks (upload_chunks): the pairs kernel runs per chunk,
// each launch waiting only for its own chunk (see enqueue_int).
static int compute_float(ecc_handle* h, const void* d_img, const Shape& s, ecc_result* out,
                         const int64_t* chunk_end, const cudaEvent_t* chunk_ev, int n_chunks) {
  cudaStream_t st = h->stream;
  const int64_t n = s.voxels;
  cudaError_t e;
  if ((e = h->pairs.ensure(sizeof(unsigned long long) * std::max<int64_t>(n, 1))) ||
      (e = h->pair_count.ensure(sizeof(unsigned long long))) ||
      (e = h->tmp.ensure(float_tail_tmp_bytes(n))) ||
      (e = h->out_vals.ensure(sizeof(uint32_t) * std::max<int64_t>(n, 1))) ||
      (e = h->out_chi.ensure(sizeof(long long) * std::max<int64_t>(n, 1))) ||
      (e = h->out_count.ensure(sizeof(unsigned long long))))
    return cuda_err(h, e, "float buffers");
  if ((e = cudaMemsetAsync(h->pair_count.p, 0, sizeof(unsigned long long), st)))
    return cuda_err(h, e, "memset");
  LocalArgs a;
  a.img = d_img;
  a.dtype = kF32;
  a.conv = h->cfg.convention;
  a.view = s.view;
  for (int i = 0; i < 4; ++i) a.n[i] = s.n[i];
  a.w_lo = 0; a.w_hi = a.n[0]; a.w_mem_lo = 0; a.w_mem_hi = a.n[0];
  a.err = h->errw.as<int>();
  a.pairs = h->pairs.as<unsigned long long>();
  a.pair_count = h->pair_count.as<unsigned long long>();
  a.pair_cap = n;
  a.stream = st;
  cudaEvent_t pa = nullptr, pb = nullptr;  // profiling: events around the pairs kernel
  if (h->prof_on) {
    if ((e = prof_event_take(h, &pa)) || (e = prof_event_take(h, &pb)) ||
        (e = cudaEventRecord(pa, st))) {
      prof_event_give(h, pa);
      prof_event_give(h, pb);
      return cuda_err(h, e, "profiling event");
    }
  }
  int64_t cnt = 0;
  const int K = n_chunks > 0 ? n_chunks : 1;
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    a.w_lo = n_chunks > 0 && k > 0 ? chunk_end[k - 1] - 1 : 0;
    a.w_hi = n_chunks > 0 && k < K - 1 ? chunk_end[k] - 1 : a.n[0];
    if (n_chunks > 0 && (e = cudaStreamWaitEvent(st, chunk_ev[k], 0))) break;
    if (a.w_lo < a.w_hi) e = launch_local(a, h->num_sms, &cnt);
  }
  if (pa && e == cudaSuccess && (e = cudaEventRecord(pb, st)) == cudaSuccess) {
    h->prof_events.emplace_back(pa, pb);
  } else if (pa) {
    prof_event_give(h, pa);
    prof_event_give(h, pb);
  }
  if (e) return cuda_err(h, e, "pairs kernel");
  h->launches += cnt;
  // the pair count and the error word into pinned memory, one wait
  if ((e = cudaMemcpyAsync(&h->h_cnt[0], h->pair_count.p, 8, cudaMemcpyDeviceToHost, st)))
    return cuda_err(h, e, "copy count");
  int word = 0;
  int rc = read_err_word(h, st, &word);
  if (rc) return rc;
  if ((rc = err_word_status(h, word))) return rc;
  const unsigned long long npairs = h->h_cnt[0];
  cnt = 0;
  if ((e = launch_float_tail(h->pairs.as<unsigned long long>(), (int64_t)npairs, h->tmp.p,
                             h->tmp.cap, h->out_vals.as<uint32_t>(), h->out_chi.as<long long>(),
                             h->out_count.as<unsigned long long>(), st, &cnt)))
    return cuda_err(h, e, "float tail");
  h->launches += cnt;
  // The result: [header][chi][thresholds] in a pinned block. k <= npairs
  // pairs survive the reduction; while npairs pairs are at most
  // kSpeculativePairBytes, all npairs slots are copied together with k
  // behind one wait, else k is read first.
  ResultBlock* blk = nullptr;
  size_t cap_pairs = 0;
  // a block for cap_pairs pairs, handed to the result at once (its header
  // written, so that ecc_result_free releases it on any later error)
  auto take_block = [&]() -> bool {
    if (!(blk = take_pair_block(h, kResultHeader + 12 * cap_pairs))) return false;
    uint64_t* hdr = reinterpret_cast<uint64_t*>(blk->p);
    hdr[0] = reinterpret_cast<uint64_t>(blk);
    hdr[1] = kResultMagic;
    out->owned = 2;  // the result's reference to blk; released by ecc_result_free
    out->chi = reinterpret_cast<int64_t*>(blk->p + kResultHeader);
    return true;
  };
  auto copy_pairs = [&](size_t n) -> cudaError_t {
    cudaError_t ce = cudaMemcpyAsync(blk->p + kResultHeader, h->out_chi.p, 8 * n,
                                     cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(blk->p + kResultHeader + 8 * cap_pairs, h->out_vals.p, 4 * n,
                           cudaMemcpyDeviceToHost, st);
    return ce;
  };
  if ((e = cudaMemcpyAsync(&h->h_cnt[1], h->out_count.p, 8, cudaMemcpyDeviceToHost, st)))
    return cuda_err(h, e, "copy count");
  if (npairs > 0 && 12 * npairs <= kSpeculativePairBytes) {
    cap_pairs = (size_t)npairs;
    if (!take_block()) return set_err(h, ECC_ERR_OOM, "pinned result block");
    if ((e = copy_pairs(cap_pairs))) return cuda_err(h, e, "copy pairs");
  }
  if ((rc = sync_stream(h, st))) return rc;
  const unsigned long long k = h->h_cnt[1];
  out->npairs = (int64_t)k;
  if (k == 0 && !blk) {
    out->thresholds = static_cast<float*>(std::malloc(sizeof(float)));
    out->chi = static_cast<int64_t*>(std::malloc(sizeof(int64_t)));
    if (!out->thresholds || !out->chi) return set_err(h, ECC_ERR_OOM, "host result");
    return ECC_OK;
  }
  if (!blk) {
    cap_pairs = (size_t)k;
    if (!take_block()) return set_err(h, ECC_ERR_OOM, "pinned result block");
    if ((e = copy_pairs(cap_pairs))) return cuda_err(h, e, "copy pairs");
    if ((rc = sync_stream(h, st))) return rc;
  }
  out->thresholds = reinterpret_cast<float*>(blk->p + kResultHeader + 8 * cap_pairs);
  return ECC_OK;
}

}  // namespace ecc

using namespace ecc;

extern "C" {

void ecc_config_default(ecc_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->device = 0;
  c->convention = ECC_CONV_V;
  c->bins = 0;
  c->slab_depth = 64;
  c->ring_bytes = int64_t(4) << 30;
  c->mem_cap_bytes = int64_t(32) << 30;
  c->tuner_cache = nullptr;
}

static thread_local std::string g_create_err;

int ecc_create(const ecc_config* cfg, ecc_handle** out) {
  if (!out) return ECC_ERR_ARG;
  *out = nullptr;
  ecc_handle* h = new (std::nothrow) ecc_handle();
  if (!h) return ECC_ERR_OOM;
  if (cfg)
    h->cfg = *cfg;
  else
    ecc_config_default(&h->cfg);
  if (h->cfg.convention != ECC_CONV_V && h->cfg.convention != ECC_CONV_T) {
    g_create_err = "convention must be ECC_CONV_V or ECC_CONV_T";
    delete h;
    return ECC_ERR_ARG;
  }
  if (h->cfg.bins < 0 || h->cfg.bins > (int64_t(1) << 24) || h->cfg.slab_depth < 0 ||
      h->cfg.ring_bytes < 0 || h->cfg.mem_cap_bytes < 0) {
    g_create_err = "negative or oversized config field";
    delete h;
    return ECC_ERR_ARG;
  }
  if (h->cfg.slab_depth == 0) h->cfg.slab_depth = 64;
  if (h->cfg.ring_bytes == 0) h->cfg.ring_bytes = int64_t(4) << 30;
  if (h->cfg.mem_cap_bytes == 0) h->cfg.mem_cap_bytes = int64_t(32) << 30;
  h->device = h->cfg.device;
  if (const char* kv = std::getenv("ECC_KERNEL")) {
    if (!std::strcmp(kv, "generic")) h->variant = 1;
    else if (!std::strcmp(kv, "bits")) h->variant = 2;
  }
  // launch-shape overrides for tuning sweeps of the bit-sliced kernel
  if (const char* w = std::getenv("ECC_BITS_WARPS")) h->bits_warps = std::atoi(w);
  if (const char* l = std::getenv("ECC_BITS_LAYOUT")) {
    if (!std::strcmp(l, "rows")) h->bits_layout = 1;
    else if (!std::strcmp(l, "columns")) h->bits_layout = 2;
  }
  if (const char* z = std::getenv("ECC_BITS_ZC")) h->bits_zc = std::atoi(z);
  if (h->cfg.tuner_cache || std::getenv("ECC_TUNE")) {
    h->tuner = new (std::nothrow) Tuner();
    if (h->tuner && h->cfg.tuner_cache) h->tuner->load(h->cfg.tuner_cache);
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || h->device < 0 || h->device >= ndev) {
    g_create_err = std::string("no CUDA device ") + std::to_string(h->device) +
                   (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : "");
    cudaGetLastError();
    delete h;
    return ECC_ERR_CUDA;
  }
  if ((e = cudaSetDevice(h->device)) ||
      (e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) ||
      // the compute stream of the blocking calls synchronises with the legacy
      // default stream, so a device image written there (as by PyTorch's
      // default stream) is complete before the kernels read it
      (e = cudaStreamCreate(&h->stream)) ||
      (e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) ||
      (e = h->errw.ensure(sizeof(int))) ||
      (e = cudaMemset(h->errw.p, 0, sizeof(int))) ||
      (e = h->done.ensure(sizeof(unsigned int))) ||
      (e = cudaMemset(h->done.p, 0, sizeof(unsigned int))) ||
      (e = cudaMallocHost(&h->h_err, sizeof(int))) ||
      (e = cudaMallocHost(&h->h_cnt, 2 * sizeof(unsigned long long)))) {
    g_create_err = std::string("CUDA setup: ") + cudaGetErrorString(e);
    ecc_destroy(h);
    return e == cudaErrorMemoryAllocation ? ECC_ERR_OOM : ECC_ERR_CUDA;
  }
  *out = h;
  return ECC_OK;
}

void ecc_destroy(ecc_handle* h) {
  if (!h) return;
  try {
    serve_shutdown(h);
  } catch (...) {
  }
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
  for (DevBuf* b : {&h->img, &h->vcec, &h->curve, &h->errw, &h->pairs, &h->pair_count, &h->tmp,
                    &h->out_vals, &h->out_chi, &h->out_count, &h->batch_desc, &h->batch_items,
                    &h->batch_vcec, &h->batch_curve, &h->codes, &h->done})
    b->release();
  for (auto& pr : h->prof_events) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (cudaEvent_t ev : h->prof_pool) cudaEventDestroy(ev);
  for (ResultBlock* b : h->pair_blocks) result_block_release(b);
  delete h->tuner;
  if (h->h_err) cudaFreeHost(h->h_err);
  if (h->h_cnt) cudaFreeHost(h->h_cnt);
  if (h->h_curve) cudaFreeHost(h->h_curve);
  for (cudaEvent_t ev : h->up_ev) cudaEventDestroy(ev);
  if (h->sync_ev) cudaEventDestroy(h->sync_ev);
  if (h->up_free) cudaEventDestroy(h->up_free);
  if (h->stream) cudaStreamDestroy(h->stream);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
}

const char* ecc_last_error(const ecc_handle* h) {
  return h ? last_err(h) : g_create_err.c_str();
}

void ecc_result_free(ecc_result* r) {
  if (!r) return;
  if (r->owned == 2) {
    // a curve (or the chi array of float pairs, the thresholds after it)
    // inside a pinned result block: drop its reference
    const void* first = r->curve ? static_cast<const void*>(r->curve) : r->chi;
    if (first) {
      const uint64_t* hdr = reinterpret_cast<const uint64_t*>(first) - 2;
      if (hdr[1] == kResultMagic) result_block_release(reinterpret_cast<ResultBlock*>(hdr[0]));
    }
  } else if (r->owned) {
    std::free(r->curve);
    std::free(r->thresholds);
    std::free(r->chi);
  }
  r->curve = nullptr;
  r->thresholds = nullptr;
  r->chi = nullptr;
  r->owned = 0;
  r->bins = 0;
  r->npairs = 0;
}

int ecc_compute(ecc_handle* h, const void* image, const int64_t* dims, int ndim,
                ecc_dtype dtype, ecc_result* out) {
  if (!h) return ECC_ERR_ARG;
  try {
    std::lock_guard<std::mutex> lk(h->api_mu);
    clear_err(h);
    if (!out) return set_err(h, ECC_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof *out);
    out->owned = 1;
    Shape s;
    int rc = validate_shape(h, dims, ndim, &s);
    if (rc) return rc;
    const size_t eb = dtype_bytes(dtype);
    if (!eb) return set_err(h, ECC_ERR_DTYPE, "unknown dtype %d", (int)dtype);
    if (s.voxels > 0 && !image) return set_err(h, ECC_ERR_ARG, "image is NULL");
    cudaError_t e = cudaSetDevice(h->device);
    if (e) return cuda_err(h, e, "set device");
    const bool on_dev = s.voxels > 0 && is_device_ptr(h, image);
    if (on_dev && !elem_aligned(image, dtype))
      return set_err(h, ECC_ERR_ARG, "device image not aligned to its element size");
    if ((e = cudaMemsetAsync(h->errw.p, 0, sizeof(int), h->stream)))
      return cuda_err(h, e, "memset");
    if (dtype == ECC_F32) {
      out->bins = 0;
      if (s.voxels == 0) {
        out->thresholds = static_cast<float*>(std::malloc(sizeof(float)));
        out->chi = static_cast<int64_t*>(std::malloc(sizeof(int64_t)));
        return ECC_OK;
      }
      const void* d_img = image;
      const size_t fbytes = eb * (size_t)s.voxels;
      std::vector<int64_t> ends;
      if (!on_dev && fbytes >= kChunkedUploadBytes && s.n[0] >= 2) {
        // chunked upload overlapping the pairs kernel, as for integer images
        if ((rc = upload_chunks(h, image, fbytes, s, &ends))) return rc;
        d_img = h->img.p;
      } else if (!on_dev) {
        if ((e = h->img.ensure(fbytes))) return cuda_err(h, e, "image buffer");
        if ((e = cudaMemcpyAsync(h->img.p, image, fbytes, cudaMemcpyHostToDevice, h->stream)))
          return cuda_err(h, e, "copy image");
        d_img = h->img.p;
      }
      rc = compute_float(h, d_img, s, out, ends.data(), h->up_ev.data(), (int)ends.size());
      if (rc) ecc_result_free(out);
      return rc;
    }
    const int64_t bins = default_bins(h, dtype);
    if ((e = h->vcec.ensure(sizeof(long long) * bins)) ||
        (e = h->curve.ensure(sizeof(long long) * bins)))
      return cuda_err(h, e, "vcec buffers");
    const void* d_img = nullptr;
    int64_t pitch = 0;
    const size_t bytes = eb * (size_t)s.voxels;
    if (!on_dev && bytes >= kChunkedUploadBytes && s.n[0] >= 2) {
      // large host image: upload in plane chunks on the copy stream and start
      // each chunk's kernels as soon as it (and the next chunk's first plane)
      // has arrived, so the copy and the computation overlap
      std::vector<int64_t> ends;
      if ((rc = upload_chunks(h, image, bytes, s, &ends))) return rc;
      const int K = (int)ends.size();
      rc = enqueue_int(h, h->img.p, 0, s, dtype, bins, h->vcec.as<long long>(),
                       h->curve.as<long long>(), h->stream, ends.data(), h->up_ev.data(), K);
    } else {
      if ((rc = stage_image(h, image, on_dev, s, dtype, bins, h->stream, &d_img, &pitch)))
        return rc;
      rc = enqueue_int(h, d_img, pitch, s, dtype, bins, h->vcec.as<long long>(),
                       h->curve.as<long long>(), h->stream);
    }
    if (rc) return rc;
    out->bins = bins;
    out->curve = static_cast<int64_t*>(std::malloc(sizeof(int64_t) * bins));
    if (!out->curve) return set_err(h, ECC_ERR_OOM, "host curve");
    // through a pinned buffer: an asynchronous copy, one wait for both reads
    if ((size_t)bins > h->h_curve_cap) {
      if (h->h_curve) cudaFreeHost(h->h_curve);
      h->h_curve = nullptr;
      h->h_curve_cap = 0;
      if ((e = cudaMallocHost(&h->h_curve, sizeof(int64_t) * bins)))
        return cuda_err(h, e, "pinned curve");
      h->h_curve_cap = (size_t)bins;
    }
    if ((e = cudaMemcpyAsync(h->h_curve, h->curve.p, sizeof(int64_t) * bins,
                             cudaMemcpyDeviceToHost, h->stream)))
      return cuda_err(h, e, "copy curve");
    int word = 0;
    if ((rc = read_err_word(h, h->stream, &word))) return rc;
    std::memcpy(out->curve, h->h_curve, sizeof(int64_t) * bins);
    if ((rc = err_word_status(h, word))) {
      ecc_result_free(out);
      return rc;
    }
    return ECC_OK;
  } catch (const std::bad_alloc&) {
    return set_err(h, ECC_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(h, ECC_ERR_CUDA, "internal error");
  }
}

int ecc_compute_device(ecc_handle* h, const void* d_image, const int64_t* dims, int ndim,
                       ecc_dtype dtype, int64_t bins, int64_t* d_curve, void* stream) {
  if (!h) return ECC_ERR_ARG;
  try {
    std::lock_guard<std::mutex> lk(h->api_mu);
    clear_err(h);
    Shape s;
    int rc = validate_shape(h, dims, ndim, &s);
    if (rc) return rc;
    if (dtype != ECC_U8 && dtype != ECC_U16)
      return set_err(h, ECC_ERR_DTYPE, "ecc_compute_device takes ECC_U8 or ECC_U16");
    if (bins <= 0) bins = default_bins(h, dtype);
    if (bins > (int64_t(1) << 24)) return set_err(h, ECC_ERR_ARG, "bins too large");
    if (!d_curve || (s.voxels > 0 && !d_image))
      return set_err(h, ECC_ERR_ARG, "null device pointer");
    if (s.voxels > 0 && !elem_aligned(d_image, dtype))
      return set_err(h, ECC_ERR_ARG, "device image not aligned to its element size");
    cudaError_t e = cudaSetDevice(h->device);
    if (e) return cuda_err(h, e, "set device");
    if ((e = h->vcec.ensure(sizeof(long long) * bins))) return cuda_err(h, e, "vcec buffer");
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : h->stream;
    const void* d_img = nullptr;
    int64_t pitch = 0;
    if ((rc = stage_image(h, d_image, true, s, dtype, bins, st, &d_img, &pitch))) return rc;
    return enqueue_int(h, d_img, pitch, s, dtype, bins, h->vcec.as<long long>(),
                       reinterpret_cast<long long*>(d_curve), st);
  } catch (...) {
    return set_err(h, ECC_ERR_CUDA, "internal error");
  }
}

int ecc_compute_quantized(ecc_handle* h, const float* image, const int64_t* dims, int ndim,
                          float lo, float hi, int64_t bins, ecc_result* out) {
  if (!h) return ECC_ERR_ARG;
  try {
    std::lock_guard<std::mutex> lk(h->api_mu);
    clear_err(h);
    if (!out) return set_err(h, ECC_ERR_ARG, "out is NULL");
    std::memset(out, 0, sizeof *out);
    out->owned = 1;
    Shape s;
    int rc = validate_shape(h, dims, ndim, &s);
    if (rc) return rc;
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi))
      return set_err(h, ECC_ERR_ARG, "need finite lo < hi");
    if (bins < 1 || bins > 65536) return set_err(h, ECC_ERR_ARG, "bins must be in 1..65536");
    if (s.voxels > 0 && !image) return set_err(h, ECC_ERR_ARG, "image is NULL");
    // the transform's constants, float32 round-to-nearest like the codes
    const float span = hi - lo;
    const float scale = (float)bins / span;
    if (!std::isfinite(scale)) return set_err(h, ECC_ERR_ARG, "hi - lo too small");
    cudaError_t e = cudaSetDevice(h->device);
    if (e) return cuda_err(h, e, "set device");
    const int code_dtype = bins <= 256 ? ECC_U8 : ECC_U16;
    const size_t code_bytes = dtype_bytes(code_dtype);
    if ((e = h->vcec.ensure(sizeof(long long) * bins)) ||
        (e = h->curve.ensure(sizeof(long long) * bins)) ||
        (e = h->codes.ensure(code_bytes * (size_t)std::max<int64_t>(s.voxels, 1))))
      return cuda_err(h, e, "buffers");
    if ((e = cudaMemsetAsync(h->errw.p, 0, sizeof(int), h->stream))) return cuda_err(h, e, "memset");
    const float* d_in = image;
    const bool in_dev = s.voxels > 0 && is_device_ptr(h, image);
    if (in_dev && !elem_aligned(image, ECC_F32))
      return set_err(h, ECC_ERR_ARG, "device image not aligned to its element size");
    if (s.voxels > 0 && !in_dev) {
      if ((e = h->img.ensure(sizeof(float) * s.voxels))) return cuda_err(h, e, "image buffer");
      if ((e = cudaMemcpyAsync(h->img.p, image, sizeof(float) * s.voxels,
                               cudaMemcpyHostToDevice, h->stream)))
        return cuda_err(h, e, "copy image");
      d_in = h->img.as<float>();
    }
    int64_t cnt = 0;
    e = launch_quantize(d_in, h->codes.p, (int)code_bytes, s.voxels, lo, scale, bins,
                        h->errw.as<int>(), h->num_sms, h->stream, &cnt);
    h->launches += cnt;
    if (e) return cuda_err(h, e, "quantize kernel");
    rc = enqueue_int(h, h->codes.p, 0, s, code_dtype, bins, h->vcec.as<long long>(),
                     h->curve.as<long long>(), h->stream);
    if (rc) return rc;
    out->bins = bins;
    out->curve = static_cast<int64_t*>(std::malloc(sizeof(int64_t) * bins));
    if (!out->curve) return set_err(h, ECC_ERR_OOM, "host curve");
    if ((size_t)bins > h->h_curve_cap) {
      if (h->h_curve) cudaFreeHost(h->h_curve);
      h->h_curve = nullptr;
      h->h_curve_cap = 0;
      if ((e = cudaMallocHost(&h->h_curve, sizeof(int64_t) * bins))) {
        ecc_result_free(out);
        return cuda_err(h, e, "pinned curve");
      }
      h->h_curve_cap = (size_t)bins;
    }
    if ((e = cudaMemcpyAsync(h->h_curve, h->curve.p, sizeof(int64_t) * bins,
                             cudaMemcpyDeviceToHost, h->stream))) {
      ecc_result_free(out);
      return cuda_err(h, e, "copy curve");
    }
    int word = 0;
    if ((rc = read_err_word(h, h->stream, &word)) || (rc = err_word_status(h, word))) {
      ecc_result_free(out);
      return rc;
    }
    std::memcpy(out->curve, h->h_curve, sizeof(int64_t) * bins);
    return ECC_OK;
  } catch (const std::bad_alloc&) {
    return set_err(h, ECC_ERR_OOM, "host allocation failed");
  } catch (...) {
    return set_err(h, ECC_ERR_CUDA, "internal error");
  }
}

int ecc_compute_vcec_chunk(ecc_handle* h, const void* planes, const int64_t* dims, int ndim,
                           ecc_dtype dtype, int64_t z_lo, int64_t z_hi, int64_t* vcec) {
  if (!h) return ECC_ERR_ARG;
  try {
    std::lock_guard<std::mutex> lk(h->api_mu);
    clear_err(h);
    Shape s;
    int rc = validate_shape(h, dims, ndim, &s);
    if (rc) return rc;
    if (dtype != ECC_U8 && dtype != ECC_U16)
      return set_err(h, ECC_ERR_DTYPE, "ecc_compute_vcec_chunk takes ECC_U8 or ECC_U16");
    if (!vcec) return set_err(h, ECC_ERR_ARG, "vcec is NULL");
    if (ndim < 3) {
      // march along dims[0]: a 1D or 2D image viewed as (dims[0], 1, nx), which
      // embeds the same complex with the same linear order as (1, ny, nx)
      s.n[0] = dims[0];
      s.n[1] = 1;
      s.n[2] = ndim == 2 ? dims[1] : 1;
    }
    const int64_t n0 = s.n[0];
    if (z_lo < 0 || z_hi > n0 || z_lo > z_hi)
      return set_err(h, ECC_ERR_ARG, "need 0 <= z_lo <= z_hi <= dims[0]");
    const int64_t bins = default_bins(h, dtype);
    // the chunk and its one-plane collars, where the image has them
    const int64_t p_lo = std::max<int64_t>(z_lo - 1, 0), p_hi = std::min<int64_t>(z_hi + 1, n0);
    const int64_t plane = s.voxels / std::max<int64_t>(n0, 1);
    const size_t bytes = dtype_bytes(dtype) * (size_t)(plane * (p_hi - p_lo));
    if (bytes > 0 && !planes) return set_err(h, ECC_ERR_ARG, "planes is NULL");
    cudaError_t e = cudaSetDevice(h->device);
    if (e) return cuda_err(h, e, "set device");
    if ((e = h->vcec.ensure(sizeof(long long) * bins))) return cuda_err(h, e, "vcec buffer");
    cudaStream_t st = h->stream;
    if ((e = cudaMemsetAsync(h->vcec.p, 0, sizeof(long long) * bins, st)) ||
        (e = cudaMemsetAsync(h->errw.p, 0, sizeof(int), st)))
      return cuda_err(h, e, "memset");
    h->clean_vcec = nullptr;  // this call leaves the VCEC filled
    const void* d_planes = planes;
    if (bytes > 0 && !is_device_ptr(h, planes)) {
      if ((e = h->img.ensure(bytes))) return cuda_err(h, e, "image buffer");
      if ((e = cudaMemcpyAsync(h->img.p, planes, bytes, cudaMemcpyHostToDevice, st)))
        return cuda_err(h, e, "copy planes");
      d_planes = h->img.p;
    } else if (bytes > 0 && !elem_aligned(planes, dtype)) {
      return set_err(h, ECC_ERR_ARG, "device planes not aligned to their element size");
    }
    if (z_hi > z_lo && s.voxels > 0) {
      LocalArgs a;
      a.img = d_planes;
      a.dtype = dtype;
      a.conv = h->cfg.convention;
      a.view = s.view;
      for (int i = 0; i < 4; ++i) a.n[i] = s.n[i];
      a.bins = bins;
      a.variant = h->variant;
      a.warps = h->bits_warps;
      a.zc = h->bits_zc;
      a.layout = h->bits_layout;
      a.vcec = h->vcec.as<long long>();
      a.err = h->errw.as<int>();
      a.stream = st;
      a.w_mem_lo = p_lo;
      a.w_mem_hi = p_hi;
      const int64_t step = max_planes_per_launch(s, h->num_sms);
      for (int64_t w = z_lo; w < z_hi; w += step) {
        a.w_lo = w;
        a.w_hi = std::min(z_hi, w + step);
        int64_t cnt = 0;
        e = launch_local(a, h->num_sms, &cnt);
        h->launches += cnt;
        if (e != cudaSuccess) return cuda_err(h, e, "contribution kernel");
      }
    }
    if ((e = cudaMemcpyAsync(vcec, h->vcec.p, sizeof(long long) * bins, cudaMemcpyDeviceToHost,
                             st)))
      return cuda_err(h, e, "copy vcec");
    int word = 0;
    if ((rc = read_err_word(h, st, &word))) return rc;
    return err_word_status(h, word);
  } catch (...) {
    return set_err(h, ECC_ERR_CUDA, "internal error");
  }
}

int ecc_device_status(ecc_handle* h) {
  if (!h) return ECC_ERR_ARG;
  try {
    std::lock_guard<std::mutex> lk(h->api_mu);
    cudaError_t e = cudaSetDevice(h->device);
    if (e) return cuda_err(h, e, "set device");
    if ((e = cudaDeviceSynchronize())) return cuda_err(h, e, "synchronize");
    int word = 0;
    int rc = read_err_word(h, h->stream, &word);
    if (rc) return rc;
    if ((e = cudaMemsetAsync(h->errw.p, 0, sizeof(int), h->stream)))
      return cuda_err(h, e, "memset");
    if ((rc = sync_stream(h, h->stream))) return rc;
    return err_word_status(h, word);
  } catch (...) {
    return set_err(h, ECC_ERR_CUDA, "internal error");
  }
}

int64_t ecc_launch_count(const ecc_handle* h) { return h ? h->launches.load() : 0; }

int ecc_set_profiling(ecc_handle* h, int on) {
  if (!h) return ECC_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->api_mu);
  h->prof_on = on != 0;
  return ECC_OK;
}

int ecc_profile_read(ecc_handle* h, double* contrib_ms, int64_t* count) {
  if (!h || !contrib_ms || !count) return ECC_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->api_mu);
  double total = 0.0, lo = 0.0, hi = 0.0;
  int rc = ECC_OK;
  const auto& ev = h->prof_events;
  for (size_t i = 0; i < ev.size(); ++i) {
    if (rc == ECC_OK) rc = wait_event(h, ev[i].second, 300LL * 1000 * 1000);
    float ms = 0.f, a = 0.f, b = 0.f;
    if (rc == ECC_OK) {
      // this pair's duration, and its start and end relative to the first
      // pair's start (for the span the recorded work covered)
      cudaError_t e = cudaEventElapsedTime(&ms, ev[i].first, ev[i].second);
      if (!e && i > 0) e = cudaEventElapsedTime(&a, ev[0].first, ev[i].first);
      if (!e) b = a + ms;
      if (e) rc = cuda_err(h, e, "elapsed time");
    }
    total += ms;
    lo = i == 0 ? a : std::min(lo, (double)a);
    hi = i == 0 ? b : std::max(hi, (double)b);
  }
  for (auto& pr : h->prof_events) {
    prof_event_give(h, pr.first);
    prof_event_give(h, pr.second);
  }
  *count = (int64_t)h->prof_events.size();
  h->prof_events.clear();
  *contrib_ms = total;
  h->prof_span_ms = rc == ECC_OK ? hi - lo : 0.0;
  return rc;
}

int ecc_profile_span(ecc_handle* h, double* span_ms) {
  if (!h || !span_ms) return ECC_ERR_ARG;
  std::lock_guard<std::mutex> lk(h->api_mu);
  *span_ms = h->prof_span_ms;
  return ECC_OK;
}

}  // extern "C"
