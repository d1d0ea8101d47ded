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

#include <cstring>
#include <new>

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
    h->err.clear();
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
    h->err.clear();
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
                              cudaMemcpyHostToDevice, h->copy_stream);
      else
        e = cudaMemcpyAsync(base + st->plane_bytes, src + off * src_plane, cnz * src_plane,
                            cudaMemcpyHostToDevice, h->copy_stream);
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
    h->err.clear();
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

}  // extern "C"
