/*
 * ecc.h -- C ABI of libecc_gb300: Euler characteristic curves (ECC) of 1-4D
 * gray-scale images on one NVIDIA GB300 (sm_103a).
 *
 * Method: Heiss & Wagner, "Streaming Algorithm for Euler Characteristic Curves
 * of Multidimensional Images".
 *   - The image complex and its filtration: Sec. 2 ("Consecutive Thresholded
 *     Images as Sublevel Set Filtrations", "Sublevel Set Filtration"): voxel
 *     (i_1..i_d) is the top cell prod_k [i_k - 1, i_k]; every other cell enters
 *     at the minimum of the voxels that contain it (convention V, the default).
 *   - The curve: Sec. 2 ("Euler Characteristic Curve"): chi(K_t) for every
 *     threshold t, chi = sum_k (-1)^k n_k.
 *   - How it is computed: Sec. 3 ("Tracking the Changes", Algorithm 1): each
 *     voxel adds, at its own gray value, the signed count of the faces it
 *     introduces (ties broken by linear index); the vector of changes (VCEC) is
 *     prefix-summed ("Post-Processing").
 *   - Streaming: Sec. 3 ("Streaming", "Processing one Chunk"): chunks along
 *     the slowest axis with a one-voxel collar.
 *   - Float images: Sec. 3 ("Other Ranges of Gray Values").
 *
 * Layout of every image argument: C order, dims[0] slowest, dims[ndim-1]
 * contiguous; 1 <= ndim <= 4. Linear index = the paper's lexicographic order.
 * Integer images are unsigned (ECC_U8, ECC_U16); values must be < bins.
 * Float images (ECC_F32) must be finite; -0.0 and +0.0 are one value.
 *
 * Pointers: an "image" argument may be a host pointer (pageable or pinned) or
 * a device pointer of the handle's device; the library tells them apart with
 * cudaPointerGetAttributes. The caller keeps ownership of every argument. The
 * blocking calls run on streams that synchronise with the legacy default
 * stream: a device image written there is complete before it is read; one
 * written on another stream must be synchronised by the caller first.
 * Every call returns an int status (ECC_OK or a negative ECC_ERR_*); no C++
 * exception ever crosses this boundary. ecc_last_error() gives a message.
 *
 * Threads: a handle may be used from one thread at a time, except that
 * ecc_submit / ecc_submit_borrowed / ecc_poll may be called concurrently from
 * any threads.
 */
#ifndef ECC_GB300_H
#define ECC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum ecc_status {
  ECC_OK = 0,
  ECC_PENDING = 1,        /* ecc_poll: request not finished yet             */
  ECC_ERR_ARG = -1,       /* null pointer, ndim outside 1..4, dim < 0, ...   */
  ECC_ERR_DTYPE = -2,     /* dtype not supported by this call               */
  ECC_ERR_VALUE = -3,     /* integer value >= bins; NaN or Inf in a float   */
  ECC_ERR_OOM = -4,       /* device or host allocation failed / over cap    */
  ECC_ERR_TIMEOUT = -5,   /* a bounded wait ran out                         */
  ECC_ERR_STATE = -6,     /* call out of order (e.g. push after finish)     */
  ECC_ERR_CUDA = -7       /* a CUDA runtime call failed                     */
};

typedef enum ecc_dtype { ECC_U8 = 1, ECC_U16 = 2, ECC_F32 = 3 } ecc_dtype;

/* Cell convention. V: the paper's (voxels are top cells, faces enter at the
 * min of their voxels; (3^d-1)-connectivity, Sec. 2 footnote on closed
 * cells). T: the dual complex the same section names in a footnote (voxels as
 * vertices, a cell enters at the max of its vertices). */
typedef enum ecc_convention { ECC_CONV_V = 0, ECC_CONV_T = 1 } ecc_convention;

typedef struct ecc_config {
  int device;             /* CUDA device ordinal (default 0)                */
  int convention;         /* ecc_convention (default ECC_CONV_V)            */
  int64_t bins;           /* thresholds 0..bins-1 of integer images;
                             0 = 256 for ECC_U8, 65536 for ECC_U16          */
  int64_t slab_depth;     /* planes per streamed slab (default 64)          */
  int64_t ring_bytes;     /* device ring for streamed slabs (default 4 GiB) */
  int64_t mem_cap_bytes;  /* device memory cap of queued requests (32 GiB)  */
  const char* tuner_cache;/* JSON file of tuned launch shapes, or NULL      */
} ecc_config;

/* Result of one image. Integer images: curve[t] = chi(K_t), t < bins.
 * Float images: the (threshold, chi) pairs at every value t where the VCEC
 * is non-zero, ascending in t; the curve is constant between them and 0 below
 * the first. Arrays are allocated by the library (owned = 1), or lie in a
 * pinned host block of the library (owned = 2): the curves of
 * ecc_compute_batch and ecc_poll share one per batch, and the pairs of a float
 * image from ecc_compute get one (chi first, thresholds after it) that the
 * handle reuses for a later float image once this result is released. Either
 * way they are released with ecc_result_free (a block once all its results
 * are released, also after ecc_destroy). */
typedef struct ecc_result {
  int64_t bins;
  int64_t* curve;
  int64_t npairs;
  float* thresholds;
  int64_t* chi;
  int32_t owned;
  int32_t status;         /* per-request status for batch/poll results      */
} ecc_result;

typedef struct ecc_handle ecc_handle;
typedef struct ecc_stream ecc_stream;

/* One image of a batch: host or device pointer, C order. */
typedef struct ecc_image {
  const void* data;
  int64_t dims[4];
  int32_t ndim;
  int32_t dtype;          /* ecc_dtype                                      */
  int64_t bins;           /* 0 = the handle's default                       */
} ecc_image;

/* Fills *cfg with the defaults listed above. */
void ecc_config_default(ecc_config* cfg);

/* Creates a handle on cfg->device (cfg may be NULL for the defaults). The
 * handle owns its streams, device pools and tuner cache. Errors: ECC_ERR_ARG,
 * ECC_ERR_CUDA (no such device), ECC_ERR_OOM. */
int ecc_create(const ecc_config* cfg, ecc_handle** out);

/* Waits for the handle's work, stops its scheduler, frees everything. NULL is
 * a no-op. Pending requests are cancelled. */
void ecc_destroy(ecc_handle* h);

/* Message of the last error of this thread's calls on the handle ("" if
 * none); valid until this thread's next call on the handle. h may be NULL
 * for errors of ecc_create (also per thread). */
const char* ecc_last_error(const ecc_handle* h);

/* Frees the arrays of a result the library allocated; safe on zeroed or
 * already-freed results. */
void ecc_result_free(ecc_result* r);

/* ECC of one image (Sec. 3, Algorithm 1 then "Post-Processing"). Blocks until
 * the result is in *out (host memory, owned by the library). A dimension of 0
 * gives the empty complex: an all-zero curve / no pairs. A device image must
 * be aligned to its element size (host images may start anywhere). Errors:
 * ECC_ERR_ARG,
 * ECC_ERR_DTYPE, ECC_ERR_VALUE (value >= bins, NaN/Inf), ECC_ERR_OOM,
 * ECC_ERR_CUDA. */
int ecc_compute(ecc_handle* h, const void* image, const int64_t* dims, int ndim,
                ecc_dtype dtype, ecc_result* out);

/* Same for an integer image already on the device, enqueued on `stream`
 * (a cudaStream_t; NULL = the handle's stream) without any host
 * synchronisation. d_image must be aligned to its element size (else
 * ECC_ERR_ARG). d_curve: device int64[bins], written by the call. The
 * library's device scratch is shared by all calls on the handle, so calls on
 * different streams must not overlap. Out-of-range values are not
 * reported by this call: ecc_device_status() reports them. */
int ecc_compute_device(ecc_handle* h, const void* d_image, const int64_t* dims,
                       int ndim, ecc_dtype dtype, int64_t bins,
                       int64_t* d_curve, void* stream);

/* Partial VCEC of one chunk of an integer image, for computations that cut
 * an image along dims[0] and combine the parts elsewhere (Sec. 3, "Parallel
 * Computations": each chunk's VCEC is computed on its own and the VCECs are
 * summed in "Post-Processing"; Sec. 6 notes the method fits map-reduce).
 * vcec[t], t < bins (the handle's default bins for dtype), receives the sum
 * of the changes of Algorithm 1 of the voxels in planes [z_lo, z_hi) of the
 * image at value t: summed over any partition of [0, dims[0]) they give the
 * image's VCEC, whose prefix sum is the curve. dims: the whole image's
 * dimensions (1-4D). planes: host or device memory holding planes
 * [max(z_lo - 1, 0), min(z_hi + 1, dims[0])) of the image, C order: the chunk
 * and the one-plane collar on each side where the image has one (a device
 * pointer aligned to its element size). vcec: host int64[bins], written.
 * Blocks until done. Errors: ECC_ERR_ARG (z range outside 0..dims[0], null
 * pointers), ECC_ERR_DTYPE, ECC_ERR_VALUE (a value >= bins), ECC_ERR_OOM,
 * ECC_ERR_CUDA. */
int ecc_compute_vcec_chunk(ecc_handle* h, const void* planes, const int64_t* dims, int ndim,
                           ecc_dtype dtype, int64_t z_lo, int64_t z_hi, int64_t* vcec);

/* ECC of a float32 image through the value transform of Sec. 3 ("Other
 * Ranges of Gray Values": shift, scale and round the values into 0..m-1, then
 * run the integer algorithm): code(v) = clamp(floor((v - lo) * s), 0, bins-1)
 * with s = bins / (hi - lo), each step a float32 operation rounded to nearest
 * (hi - lo, s, v - lo, the product). curve[k] = chi of {voxels with code <= k},
 * which is the exact float curve read at the largest image value of code k.
 * image: host or device float32, C order, 1-4D. bins: 1..65536 (codes are
 * uint8 up to 256 bins, else uint16). Blocks until *out holds the curve
 * (owned by the library). Errors: ECC_ERR_ARG (lo >= hi, non-finite lo / hi,
 * bins out of range), ECC_ERR_VALUE (NaN or Inf in the image), ECC_ERR_OOM,
 * ECC_ERR_CUDA. */
int ecc_compute_quantized(ecc_handle* h, const float* image, const int64_t* dims, int ndim,
                          float lo, float hi, int64_t bins, ecc_result* out);

/* Synchronises the handle's device work and returns ECC_ERR_VALUE if any
 * ecc_compute_device call since the last ecc_device_status saw a value
 * >= bins, else ECC_OK (or ECC_ERR_CUDA). Clears the flag. */
int ecc_device_status(ecc_handle* h);

/* Streaming (Sec. 3, "Streaming"): the image arrives as z-slabs (runs of
 * consecutive planes along dims[0]) in order, with no gaps. The library keeps
 * the one-plane collar itself, so slabs do not overlap. Slabs are copied
 * through a device ring buffer of cfg->ring_bytes on a copy stream; the
 * partial VCEC stays on the device. Integer dtypes only. */
int ecc_stream_begin(ecc_handle* h, const int64_t* dims, int ndim, ecc_dtype dtype,
                     ecc_stream** out);

/* Pushes planes [z0, z0 + nz) of the image (host memory, pinned for full
 * copy speed, or device memory; C order, dims of one plane as given to
 * ecc_stream_begin). Returns once the buffer may be reused; the computation continues in
 * the background. Errors: ECC_ERR_STATE (z0 not the next plane, after finish),
 * ECC_ERR_ARG, ECC_ERR_CUDA. */
int ecc_stream_push_slab(ecc_stream* s, const void* host_planes, int64_t z0, int64_t nz);

/* Finishes a stream whose planes have all been pushed, writes the curve to
 * *out and releases the stream (also on error). ECC_ERR_STATE if planes are
 * missing; ECC_ERR_VALUE if a value was >= bins. */
int ecc_stream_finish(ecc_stream* s, ecc_result* out);

/* Drops a stream without a result. */
void ecc_stream_abort(ecc_stream* s);

/* Out-of-core streaming from a file (Sec. 3, "Streaming", where chunks are
 * read from disk; Sec. 5 runs terabyte images this way): the image is stored
 * raw at byte `offset` of the file at `path` (C order, native byte order, no
 * padding, dims and integer dtype as for ecc_stream_begin). A reader thread
 * fills two pinned slab buffers of cfg->slab_depth planes with pread while
 * the other is pushed through the device ring. Blocks until *out holds the
 * curve (owned by the library). Errors: ECC_ERR_ARG (file missing, shorter
 * than offset + image bytes, or a read failed), ECC_ERR_DTYPE, ECC_ERR_VALUE,
 * ECC_ERR_OOM, ECC_ERR_TIMEOUT (a slab read took over 10 minutes),
 * ECC_ERR_CUDA. */
int ecc_stream_file(ecc_handle* h, const char* path, int64_t offset, const int64_t* dims,
                    int ndim, ecc_dtype dtype, ecc_result* out);

/* Batched computation: all images of the batch in one persistent launch
 * whose blocks take (image, tile) items from a work list (batches of more
 * than 1024 images run in launches of 1024, each built while the previous
 * one runs). Images of 1-3 dimensions and integer dtypes, host or device
 * pointers (a device image aligned to its element size); outs[i] receives
 * image i's curve (owned = 2: see ecc_result) and outs[i].status its status.
 * Blocks until done. */
int ecc_compute_batch(ecc_handle* h, int n, const ecc_image* images, ecc_result* outs);

/* Serving: queues one request. The image (integer dtype; pageable or pinned
 * host memory, or device memory of the handle's device) is copied before the
 * call returns (pinned and device images straight to the device, the call
 * waiting for that copy). A scheduler thread admits
 * queued requests while their device memory fits under cfg->mem_cap_bytes,
 * launches the requests whose copies have finished as one batched launch on
 * one of two slots, and keeps launching while earlier batches run; with one
 * batch in flight the next one waits to hold 32 requests or 64 M voxels, or
 * until its oldest request has waited 200 us. A request whose image is larger than
 * cfg->ring_bytes is streamed instead (Sec. 3, "Streaming"): slabs of
 * dims[0] planes pass through a ring of at most cfg->ring_bytes under the
 * cap, one such request at a time, its partial VCEC kept on the device, while
 * batches of the other requests go on. ECC_ERR_OOM if the request (or its
 * ring) cannot fit under the cap. *req_id identifies the request. */
int ecc_submit(ecc_handle* h, const void* image, const int64_t* dims, int ndim,
               ecc_dtype dtype, uint64_t* req_id);

/* As ecc_submit, but an image in pinned host memory (cudaHostAlloc'd or
 * registered) or in device memory is borrowed instead of copied before the
 * call returns: its
 * device copy is enqueued on the server's copy stream (ordered before the
 * request's batch) or, over the memory cap, made when the scheduler admits
 * the request, and a streamed request reads its slabs from it. The caller
 * keeps the buffer allocated and unchanged until ecc_poll has returned a
 * status other than ECC_PENDING / ECC_ERR_TIMEOUT for the request (or the
 * handle is destroyed). The call does not wait for the copy, so a submitting
 * thread queues copies back to back. An image in pageable host memory is
 * copied before the call returns, as by ecc_submit. Errors as ecc_submit. */
int ecc_submit_borrowed(ecc_handle* h, const void* image, const int64_t* dims, int ndim,
                        ecc_dtype dtype, uint64_t* req_id);

/* Waits up to timeout_us microseconds (0 = just check) for request req_id.
 * ECC_OK: *out holds the curve and the request is retired (the curve of a
 * batched request lies in place in a pinned result slab of the library,
 * owned = 2, that of a streamed one in its own allocation, owned = 1; either
 * is released by ecc_result_free). ECC_PENDING: not
 * done and timeout_us == 0. ECC_ERR_TIMEOUT: not done when the wait ran out.
 * ECC_ERR_ARG: unknown id. A failed request returns its error status once. */
int ecc_poll(ecc_handle* h, uint64_t req_id, ecc_result* out, int64_t timeout_us);

/* Latency record of a retired request, in microseconds from ecc_submit to the
 * completion event, for p50/p99 reporting. ECC_ERR_ARG if unknown. */
int ecc_request_latency_us(ecc_handle* h, uint64_t req_id, double* us);

/* Stages of a retired request, in microseconds from ecc_submit (-1 where a
 * stage did not happen, e.g. a streamed request has no batch): stages[0] its
 * device copy seen finished, [1] its batch launched, [2] its batch seen
 * finished, [3] its curve ready (the latency). Instrumentation, no
 * counterpart in the paper. ECC_ERR_ARG if unknown or not retired. */
int ecc_request_trace_us(ecc_handle* h, uint64_t req_id, double* stages);

/* Number of kernel launches this handle issued since it was created. */
int64_t ecc_launch_count(const ecc_handle* h);

/* Instrumentation (no counterpart in the paper). With profiling on, every
 * single-image computation (integer curve or float pairs) records CUDA events
 * on its launching stream around its contribution kernel(s), and every
 * launch of ecc_compute_batch around its graph (clear, contribution, scan). ecc_profile_read synchronises, returns the summed
 * elapsed milliseconds and the number of computations recorded since the
 * last read, and clears the record. */
int ecc_set_profiling(ecc_handle* h, int on);
int ecc_profile_read(ecc_handle* h, double* contrib_ms, int64_t* count);

/* Milliseconds from the earliest start to the latest end among the event
 * pairs of the record the last ecc_profile_read returned: the device time
 * the recorded work spanned, work that overlapped (the two slots of a batched
 * computation) counted once. */
int ecc_profile_span(ecc_handle* h, double* span_ms);

/* ECC of an integer image already on the device, for callers that cannot
 * allocate device memory: for example a host program that has handed all of
 * the GPU's memory to its own pool allocator and may not let a library
 * allocate beside it, or one that must stay inside a fixed, pre-planned
 * memory budget. It needs no handle and allocates nothing. The paper has no
 * counterpart of this entry point.
 *
 * What the computation needs besides the caller's image and curve (the int64
 * change vector and an error word) sits in file-scope device arrays of this
 * library: 65536 int64 counters (512 KiB) plus 256 bytes, held by every GPU
 * that loads the library until the process exits. Hence bins must lie in
 * 1..65536; a larger bins returns ECC_ERR_ARG.
 *
 * d_image: device (or managed) memory of the current device, layout as
 * everywhere in this header (ECC_U8 or ECC_U16, 1 <= ndim <= 4), its address
 * a multiple of the element size. convention: ECC_CONV_V or ECC_CONV_T.
 * d_curve: device int64[bins] of the current device, 8-byte aligned, written
 * with chi(K_t). stream: a cudaStream_t (NULL = the legacy default stream);
 * the call enqueues its work there, copies the error word back and
 * synchronises the stream before returning, also when it fails after
 * enqueueing. Errors: ECC_ERR_ARG (also for a pointer that is not device
 * memory of the current device, or misaligned), ECC_ERR_DTYPE, ECC_ERR_VALUE
 * (a value >= bins), ECC_ERR_CUDA.
 *
 * The first call on a device (with that device current) looks up the
 * arrays' device address; make that first call before any stream capture.
 * All calls on a device share the arrays, and each call clears them first:
 * calls that overlap on the GPU (from several host threads or streams) race
 * and give wrong results. */
int ecc_compute_device_noalloc(const void* d_image, const int64_t* dims, int ndim,
                               ecc_dtype dtype, int64_t bins, int convention,
                               int64_t* d_curve, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ECC_GB300_H */
