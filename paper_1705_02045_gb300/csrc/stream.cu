// Streaming (Sec. 3, "Streaming" and "Processing one Chunk"): the image
// arrives as chunks of consecutive planes along dims[0]; each chunk is
// processed with a one-plane collar on each side, and the per-chunk VCECs add
// up to the whole image's (the cell partition by axis-0 coordinate).
//
// Device side: a ring of R slots, each holding (depth + 2) planes: the collar
// plane below, the chunk, the collar plane above. Host planes go to their slot
// by cudaMemcpyAsync on the copy stream; the compute stream waits for the
// copy, copies the two collar planes device-to-device between neighbouring
// slots, and runs the contribution kernel on the previous chunk (whose upper
// collar has just arrived). The partial VCEC stays on the device until finish.
// A slot is reused once the kernel that read it has finished (event wait on
// the copy stream, no host blocking).
#include "engine.h"

#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <atomic>
#include <cerrno>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

namespace ecc {

struct StreamSlot {
  cudaEvent_t copied = nullptr;  // host planes landed in the slot
  cudaEvent_t freed = nullptr;   // contribution kernel on this slot finished
  int64_t z0 = 0, nz = 0;
  bool used = false;
};

}  // namespace ecc

using namespace ecc;

struct ecc_stream {
  ecc_handle* h = nullptr;
  Shape s;          // kernel view: marching axis n[0] = dims[0]
  int dtype = kU8;
  int64_t bins = 256;
  size_t plane_bytes = 0;   // bytes of one plane in a ring slot
  size_t src_row = 0;       // bytes of one dense row in the caller's planes
  size_t rows_per_plane = 0;
  int64_t row_pitch = 0;    // slot row pitch (0 = dense)
  int64_t depth = 64;
  int R = 0;
  DevBuf ring, vcec, curve;
  std::vector<StreamSlot> slots;
  int64_t next_z = 0;
  int64_t chunks = 0;
  int pending = -1;  // slot whose kernel waits for the next chunk's first plane
  bool failed = false;
};

namespace {

char* slot_base(ecc_stream* st, int k) {
  return static_cast<char*>(st->ring.p) + (size_t)k * (st->depth + 2) * st->plane_bytes;
}

// Contribution kernel over the chunk held in slot k; planes z0-1 .. z0+nz are
// readable from the slot (the collar planes outside the image are never read).
int launch_slot(ecc_stream* st, int k, bool has_upper) {
  ecc_handle* h = st->h;
  StreamSlot& sl = st->slots[k];
  LocalArgs a;
  a.img = slot_base(st, k);
  a.dtype = st->dtype;
  a.conv = h->cfg.convention;
  a.view = st->s.view;
  for (int i = 0; i < 4; ++i) a.n[i] = st->s.n[i];
  a.w_lo = sl.z0;
  a.w_hi = sl.z0 + sl.nz;
  a.w_mem_lo = sl.z0 - 1;
  a.w_mem_hi = sl.z0 + sl.nz + (has_upper ? 1 : 0);
  a.bins = st->bins;
  a.row_pitch = st->row_pitch;
  a.variant = h->variant;
  a.vcec = st->vcec.as<long long>();
  a.err = h->errw.as<int>();
  a.stream = h->stream;
  int64_t cnt = 0;
  cudaError_t e = launch_local(a, h->num_sms, &cnt);
  h->launches += cnt;
  if (e) return cuda_err(h, e, "contribution kernel (slab)");
  if ((e = cudaEventRecord(sl.freed, h->stream))) return cuda_err(h, e, "record");
  return ECC_OK;
}

void release(ecc_stream* st) {
  if (!st) return;
  if (st->h) {
    cudaSetDevice(st->h->device);
    cudaStreamSynchronize(st->h->stream);
    cudaStreamSynchronize(st->h->copy_stream);
  }
  for (StreamSlot& sl : st->slots) {
    if (sl.copied) cudaEventDestroy(sl.copied);
    if (sl.freed) cudaEventDestroy(sl.freed);
  }
  st->ring.release();
  st->vcec.release();
  st->curve.release();
  delete st;
}

}  // namespace

extern "C" {

int ecc_stream_begin(ecc_handle* h, const int64_t* dims, int ndim, ecc_dtype dtype,
                     ecc_stream** out) {
  if (!h) return ECC_ERR_ARG;
  try {
    std::lock_guard<std::mutex> lk(h->api_mu);
    clear_err(h);
    if (!out) return set_err(h, ECC_ERR_ARG, "out is NULL");
    *out = nullptr;
    Shape s;
    int rc = validate_shape(h, dims, ndim, &s);
    if (rc) return rc;
    if (dtype != ECC_U8 && dtype != ECC_U16)
      return set_err(h, ECC_ERR_DTYPE, "streaming takes ECC_U8 or ECC_U16");
    // View with the streamed axis dims[0] as the marching axis: an extent-1
    // axis inserted between keeps the complex (product with a unit interval).
    if (ndim < 4) {
      s.view = 3;
      s.n[0] = dims[0];
      s.n[1] = ndim >= 3 ? dims[1] : 1;
      s.n[2] = ndim >= 2 ? dims[ndim - 1] : 1;
      s.n[3] = 1;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e) return cuda_err(h, e, "set device");
    ecc_stream* st = new (std::nothrow) ecc_stream();
    if (!st) return set_err(h, ECC_ERR_OOM, "stream state");
    st->h = h;
    st->s = s;
    st->dtype = dtype;
    st->bins = default_bins(h, dtype);
    st->src_row = dtype_bytes(dtype) * (size_t)s.n[s.view - 1];
    st->rows_per_plane = s.voxels > 0 ? (size_t)(s.voxels / s.n[0] / s.n[s.view - 1]) : 0;
    size_t slot_row = st->src_row;  // dense slot rows (kernels take any alignment)
    st->plane_bytes = slot_row * st->rows_per_plane;
    if (s.voxels == 0) st->plane_bytes = 0;
    st->depth = std::max<int64_t>(1, h->cfg.slab_depth);
    if (st->plane_bytes > 0) {
      const int64_t ring_planes = h->cfg.ring_bytes / (int64_t)st->plane_bytes;
      // at least two slots; shrink the depth if the ring is small
      if (ring_planes < 2 * (st->depth + 2)) st->depth = ring_planes / 2 - 2;
      if (st->depth < 1) {
        delete st;
        return set_err(h, ECC_ERR_OOM, "ring of %lld bytes holds fewer than 6 planes",
                       (long long)h->cfg.ring_bytes);
      }
      st->depth = std::min<int64_t>(st->depth, std::max<int64_t>(dims[0], 1));
      st->R = (int)std::min<int64_t>(3, ring_planes / (st->depth + 2));
    } else {
      st->R = 0;
    }
    st->slots.resize(st->R);
    if ((e = st->vcec.ensure(sizeof(long long) * st->bins)) ||
        (e = st->curve.ensure(sizeof(long long) * st->bins)) ||
        (st->R && (e = st->ring.ensure((size_t)st->R * (st->depth + 2) * st->plane_bytes)))) {
      release(st);
      return cuda_err(h, e, "stream buffers");
    }
    for (StreamSlot& sl : st->slots) {
      if ((e = cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming)) ||
          (e = cudaEventCreateWithFlags(&sl.freed, cudaEventDisableTiming))) {
        release(st);
        return cuda_err(h, e, "events");
      }
    }
    if ((e = cudaMemsetAsync(st->vcec.p, 0, sizeof(long long) * st->bins, h->stream)) ||
        (e = cudaMemsetAsync(h->errw.p, 0, sizeof(int), h->stream))) {
      release(st);
      return cuda_err(h, e, "memset");
    }
    *out = st;
    return ECC_OK;
  } catch (...) {
    return set_err(h, ECC_ERR_OOM, "stream begin failed");
  }
}

int ecc_stream_push_slab(ecc_stream* st, const void* host_planes, int64_t z0, int64_t nz) {
  if (!st) return ECC_ERR_ARG;
  ecc_handle* h = st->h;
  try {
    std::lock_guard<std::mutex> lk(h->api_mu);
    clear_err(h);
    if (st->failed) return set_err(h, ECC_ERR_STATE, "stream failed earlier");
    if (z0 != st->next_z)
      return set_err(h, ECC_ERR_STATE, "expected plane %lld, got %lld", (long long)st->next_z,
                     (long long)z0);
    if (nz < 1 || z0 + nz > st->s.n[0] || !host_planes)
      return set_err(h, ECC_ERR_ARG, "bad slab [%lld, +%lld)", (long long)z0, (long long)nz);
    if (st->R == 0) {  // planes of zero voxels: nothing to copy
      st->next_z = z0 + nz;
      return ECC_OK;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e) return cuda_err(h, e, "set device");
    const char* src = static_cast<const char*>(host_planes);
    int last_slot = -1;
    for (int64_t off = 0; off < nz; off += st->depth) {
      const int64_t cnz = std::min<int64_t>(st->depth, nz - off);
      const int k = (int)(st->chunks % st->R);
      StreamSlot& sl = st->slots[k];
      char* base = slot_base(st, k);
      if (sl.used && (e = cudaStreamWaitEvent(h->copy_stream, sl.freed, 0))) break;
      const size_t src_plane = st->src_row * st->rows_per_plane;
      if (st->row_pitch)
        e = cudaMemcpy2DAsync(base + st->plane_bytes, (size_t)st->row_pitch, src + off * src_plane,
                              st->src_row, st->src_row, cnz * st->rows_per_plane,
                              cudaMemcpyDefault, h->copy_stream);
      else
        e = cudaMemcpyAsync(base + st->plane_bytes, src + off * src_plane, cnz * src_plane,
                            cudaMemcpyDefault, h->copy_stream);
      if (e ||
          (e = cudaEventRecord(sl.copied, h->copy_stream)) ||
          (e = cudaStreamWaitEvent(h->stream, sl.copied, 0)))
        break;
      sl.z0 = z0 + off;
      sl.nz = cnz;
      sl.used = true;
      if (st->pending >= 0) {
        const int p = st->pending;
        StreamSlot& ps = st->slots[p];
        char* pbase = slot_base(st, p);
        // collars: our first plane above the previous chunk, its last below ours
        if ((e = cudaMemcpyAsync(pbase + (ps.nz + 1) * st->plane_bytes, base + st->plane_bytes,
                                 st->plane_bytes, cudaMemcpyDeviceToDevice, h->stream)) ||
            (e = cudaMemcpyAsync(base, pbase + ps.nz * st->plane_bytes, st->plane_bytes,
                                 cudaMemcpyDeviceToDevice, h->stream)))
          break;
        int rc = launch_slot(st, p, true);
        if (rc) {
          st->failed = true;
          return rc;
        }
      }
      st->pending = k;
      ++st->chunks;
      last_slot = k;
    }
    if (e) {
      st->failed = true;
      return cuda_err(h, e, "slab copy");
    }
    st->next_z = z0 + nz;
    // the caller's buffer is free once its copies are done
    if (last_slot >= 0) {
      int rc = wait_event(h, st->slots[last_slot].copied, 300LL * 1000 * 1000);
      if (rc) {
        st->failed = true;
        return rc;
      }
    }
    return ECC_OK;
  } catch (...) {
    st->failed = true;
    return set_err(h, ECC_ERR_CUDA, "push failed");
  }
}

int ecc_stream_finish(ecc_stream* st, ecc_result* out) {
  if (!st) return ECC_ERR_ARG;
  ecc_handle* h = st->h;
  int rc = ECC_OK;
  try {
    std::unique_lock<std::mutex> lk(h->api_mu);
    clear_err(h);
    if (!out) {
      rc = set_err(h, ECC_ERR_ARG, "out is NULL");
    } else if (st->failed) {
      rc = set_err(h, ECC_ERR_STATE, "stream failed earlier");
    } else if (st->next_z != st->s.n[0] && st->s.voxels > 0) {
      rc = set_err(h, ECC_ERR_STATE, "planes [%lld, %lld) were never pushed",
                   (long long)st->next_z, (long long)st->s.n[0]);
    }
    if (rc == ECC_OK) {
      std::memset(out, 0, sizeof *out);
      cudaError_t e = cudaSetDevice(h->device);
      if (e) rc = cuda_err(h, e, "set device");
      if (!rc && st->pending >= 0) rc = launch_slot(st, st->pending, false);
      int64_t cnt = 0;
      if (!rc && (e = launch_scan(st->vcec.as<long long>(), st->curve.as<long long>(), st->bins,
                                  h->stream, &cnt)))
        rc = cuda_err(h, e, "scan");
      h->launches += cnt;
      if (!rc) {
        out->owned = 1;
        out->bins = st->bins;
        out->curve = static_cast<int64_t*>(std::malloc(sizeof(int64_t) * st->bins));
        if (!out->curve) rc = set_err(h, ECC_ERR_OOM, "host curve");
      }
      if (!rc && (e = cudaMemcpyAsync(out->curve, st->curve.p, sizeof(int64_t) * st->bins,
                                      cudaMemcpyDeviceToHost, h->stream)))
        rc = cuda_err(h, e, "copy curve");
      if (!rc && (e = cudaMemcpyAsync(h->h_err, h->errw.p, sizeof(int), cudaMemcpyDeviceToHost,
                                      h->stream)))
        rc = cuda_err(h, e, "copy error word");
      cudaEvent_t ev = nullptr;
      if (!rc && !(e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) &&
          !(e = cudaEventRecord(ev, h->stream)))
        rc = wait_event(h, ev, 300LL * 1000 * 1000);
      else if (!rc)
        rc = cuda_err(h, e, "event");
      if (ev) cudaEventDestroy(ev);
      if (!rc && (*h->h_err & kErrValue))
        rc = set_err(h, ECC_ERR_VALUE, "a value is >= bins");
      if (!rc && (*h->h_err & kErrOverflow))
        rc = set_err(h, ECC_ERR_CUDA, "a collar plane was missing (internal)");
      if (rc) ecc_result_free(out);
    }
    lk.unlock();
    release(st);
    return rc;
  } catch (...) {
    release(st);
    return set_err(h, ECC_ERR_CUDA, "finish failed");
  }
}

void ecc_stream_abort(ecc_stream* st) {
  if (!st) return;
  try {
    release(st);
  } catch (...) {
  }
}

// Out-of-core streaming from a file (Sec. 3, "Streaming": chunks read from
// disk; the terabyte images of Sec. 5 are processed this way). A reader
// thread fills two pinned slab buffers with pread (each slab split over up to
// kReadThreads parallel readers) while the caller's thread pushes the other
// one through the device ring, so disk reads, host-to-device copies and
// kernels overlap.
constexpr int kReadThreads = 8;

int ecc_stream_file(ecc_handle* h, const char* path, int64_t offset, const int64_t* dims,
                    int ndim, ecc_dtype dtype, ecc_result* out) {
  if (!h) return ECC_ERR_ARG;
  if (!out || !path || offset < 0) return set_err(h, ECC_ERR_ARG, "bad path, offset or out");
  std::memset(out, 0, sizeof *out);
  ecc_stream* st = nullptr;
  int rc = ecc_stream_begin(h, dims, ndim, dtype, &st);
  if (rc) return rc;
  const int64_t nz = st->s.n[0];
  const size_t plane = st->src_row * st->rows_per_plane;
  const int fd = ::open(path, O_RDONLY);
  if (fd < 0) {
    ecc_stream_abort(st);
    return set_err(h, ECC_ERR_ARG, "cannot open %s: %s", path, std::strerror(errno));
  }
  struct stat sb;
  if (::fstat(fd, &sb) != 0 ||
      (uint64_t)sb.st_size < (uint64_t)offset + (uint64_t)plane * (uint64_t)nz) {
    ::close(fd);
    ecc_stream_abort(st);
    return set_err(h, ECC_ERR_ARG, "%s is shorter than offset + image bytes", path);
  }
#ifdef POSIX_FADV_SEQUENTIAL
  posix_fadvise(fd, 0, 0, POSIX_FADV_SEQUENTIAL);
#endif
  const int64_t depth = std::max<int64_t>(1, std::min<int64_t>(st->depth, nz));
  void* buf[2] = {nullptr, nullptr};
  if (plane > 0 && nz > 0) {
    for (int i = 0; i < 2; ++i) {
      cudaError_t e = cudaHostAlloc(&buf[i], plane * (size_t)depth, cudaHostAllocDefault);
      if (e) {
        cudaGetLastError();
        for (int j = 0; j < 2; ++j)
          if (buf[j]) cudaFreeHost(buf[j]);
        ::close(fd);
        ecc_stream_abort(st);
        return set_err(h, ECC_ERR_OOM, "pinned slab buffers");
      }
    }
  }
  // slab k lives in buf[k & 1]; full[i] = slab index held by buffer i, or -1
  std::mutex mu;
  std::condition_variable cv;
  int64_t full[2] = {-1, -1};
  bool stop = false;
  int read_err = 0;
  const int64_t slabs = plane > 0 ? (nz + depth - 1) / depth : 0;
  std::thread reader([&] {
    for (int64_t k = 0; k < slabs; ++k) {
      const int i = (int)(k & 1);
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return stop || full[i] < 0; });
        if (stop) return;
      }
      const int64_t z0 = k * depth, n = std::min(depth, nz - z0);
      const size_t want = plane * (size_t)n;
      char* dst = static_cast<char*>(buf[i]);
      const off_t base = (off_t)(offset + (int64_t)plane * z0);
      // the slab in parts of >= 32 MiB read by parallel preads (one thread
      // copying out of the page cache is far slower than the ring)
      const size_t part = std::max<size_t>(size_t(32) << 20, (want + kReadThreads - 1) / kReadThreads);
      std::atomic<int> err{0};
      auto read_range = [&](size_t lo, size_t hi) {
        while (lo < hi && !err.load()) {
          const ssize_t r = ::pread(fd, dst + lo, hi - lo, base + (off_t)lo);
          if (r < 0 && errno == EINTR) continue;
          if (r <= 0) {
            err = r < 0 ? errno : EIO;
            return;
          }
          lo += (size_t)r;
        }
      };
      std::vector<std::thread> parts;
      for (size_t lo = part; lo < want; lo += part)
        parts.emplace_back(read_range, lo, std::min(want, lo + part));
      read_range(0, std::min(want, part));
      for (std::thread& t : parts) t.join();
      std::lock_guard<std::mutex> lk(mu);
      if (err.load()) {
        read_err = err.load();
      } else {
        full[i] = k;
      }
      cv.notify_all();
      if (read_err) return;
    }
  });
  rc = ECC_OK;
  for (int64_t k = 0; k < slabs && rc == ECC_OK; ++k) {
    const int i = (int)(k & 1);
    {
      std::unique_lock<std::mutex> lk(mu);
      // a read of one slab: bounded at 10 minutes
      if (!cv.wait_for(lk, std::chrono::minutes(10), [&] { return full[i] == k || read_err; }))
        rc = set_err(h, ECC_ERR_TIMEOUT, "reading slab %lld timed out", (long long)k);
      else if (read_err)
        rc = set_err(h, ECC_ERR_ARG, "reading %s failed: %s", path, std::strerror(read_err));
    }
    if (rc) break;
    const int64_t z0 = k * depth, n = std::min(depth, nz - z0);
    rc = ecc_stream_push_slab(st, buf[i], z0, n);
    std::lock_guard<std::mutex> lk(mu);
    full[i] = -1;  // the push returned: the buffer may be refilled
    cv.notify_all();
  }
  {
    std::lock_guard<std::mutex> lk(mu);
    stop = true;
    cv.notify_all();
  }
  reader.join();
  ::close(fd);
  if (rc == ECC_OK) {
    rc = ecc_stream_finish(st, out);
  } else {
    ecc_stream_abort(st);  // keeps this thread's message
  }
  for (int j = 0; j < 2; ++j)
    if (buf[j]) cudaFreeHost(buf[j]);
  return rc;
}

}  // extern "C"
