"""Python binding of libecc_gb300.so (include/ecc.h), argument marshalling only.

Every function keeps the C name. Images may be numpy arrays (host) or torch
tensors (host or CUDA); the library itself tells host from device pointers.
There is no Python or CPU fallback: if the library is missing, ``load()``
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ECC_OK, ECC_PENDING = 0, 1
ECC_ERR_ARG, ECC_ERR_DTYPE, ECC_ERR_VALUE, ECC_ERR_OOM = -1, -2, -3, -4
ECC_ERR_TIMEOUT, ECC_ERR_STATE, ECC_ERR_CUDA = -5, -6, -7
ECC_U8, ECC_U16, ECC_F32 = 1, 2, 3
ECC_CONV_V, ECC_CONV_T = 0, 1

_STATUS = {0: "ECC_OK", 1: "ECC_PENDING", -1: "ECC_ERR_ARG", -2: "ECC_ERR_DTYPE",
           -3: "ECC_ERR_VALUE", -4: "ECC_ERR_OOM", -5: "ECC_ERR_TIMEOUT",
           -6: "ECC_ERR_STATE", -7: "ECC_ERR_CUDA"}


class EccError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class ecc_config(C.Structure):
    _fields_ = [("device", C.c_int), ("convention", C.c_int), ("bins", C.c_int64),
                ("slab_depth", C.c_int64), ("ring_bytes", C.c_int64),
                ("mem_cap_bytes", C.c_int64), ("tuner_cache", C.c_char_p)]


class ecc_result(C.Structure):
    _fields_ = [("bins", C.c_int64), ("curve", C.POINTER(C.c_int64)),
                ("npairs", C.c_int64), ("thresholds", C.POINTER(C.c_float)),
                ("chi", C.POINTER(C.c_int64)), ("owned", C.c_int32), ("status", C.c_int32)]


class ecc_image(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dims", C.c_int64 * 4), ("ndim", C.c_int32),
                ("dtype", C.c_int32), ("bins", C.c_int64)]


_P = C.c_void_p
_I64P = C.POINTER(C.c_int64)
_SIGNATURES = {
    "ecc_config_default": (None, [C.POINTER(ecc_config)]),
    "ecc_create": (C.c_int, [C.POINTER(ecc_config), C.POINTER(_P)]),
    "ecc_destroy": (None, [_P]),
    "ecc_last_error": (C.c_char_p, [_P]),
    "ecc_result_free": (None, [C.POINTER(ecc_result)]),
    "ecc_compute": (C.c_int, [_P, _P, _I64P, C.c_int, C.c_int, C.POINTER(ecc_result)]),
    "ecc_compute_device": (C.c_int, [_P, _P, _I64P, C.c_int, C.c_int, C.c_int64, _P, _P]),
    "ecc_device_status": (C.c_int, [_P]),
    "ecc_compute_vcec_chunk": (C.c_int, [_P, _P, _I64P, C.c_int, C.c_int, C.c_int64, C.c_int64,
                                         _I64P]),
    "ecc_compute_quantized": (C.c_int, [_P, _P, _I64P, C.c_int, C.c_float, C.c_float, C.c_int64,
                                        C.POINTER(ecc_result)]),
    "ecc_stream_begin": (C.c_int, [_P, _I64P, C.c_int, C.c_int, C.POINTER(_P)]),
    "ecc_stream_push_slab": (C.c_int, [_P, _P, C.c_int64, C.c_int64]),
    "ecc_stream_finish": (C.c_int, [_P, C.POINTER(ecc_result)]),
    "ecc_stream_abort": (None, [_P]),
    "ecc_stream_file": (C.c_int, [_P, C.c_char_p, C.c_int64, _I64P, C.c_int, C.c_int,
                                  C.POINTER(ecc_result)]),
    "ecc_compute_batch": (C.c_int, [_P, C.c_int, C.POINTER(ecc_image), C.POINTER(ecc_result)]),
    "ecc_submit": (C.c_int, [_P, _P, _I64P, C.c_int, C.c_int, C.POINTER(C.c_uint64)]),
    "ecc_submit_borrowed": (C.c_int, [_P, _P, _I64P, C.c_int, C.c_int, C.POINTER(C.c_uint64)]),
    "ecc_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(ecc_result), C.c_int64]),
    "ecc_request_latency_us": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_double)]),
    "ecc_request_trace_us": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_double)]),
    "ecc_launch_count": (C.c_int64, [_P]),
    "ecc_set_profiling": (C.c_int, [_P, C.c_int]),
    "ecc_profile_read": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "ecc_profile_span": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "ecc_compute_device_noalloc": (C.c_int, [_P, _I64P, C.c_int, C.c_int, C.c_int64, C.c_int,
                                             _P, _P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads the CUDA library (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build_library()
        else:
            raise RuntimeError(
                f"{path} is missing: build it with __graft_entry__.build() "
                "(there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


_DTYPE_CODES = {}


def _dtype_code(dt) -> int:
    """ECC dtype code of a numpy dtype / scalar type or a torch dtype; other
    types map to 0, which the library rejects with ECC_ERR_DTYPE."""
    code = _DTYPE_CODES.get(dt)
    if code is None:
        try:
            name = np.dtype(dt).name
        except TypeError:
            name = str(dt).replace("torch.", "")
        code = {"uint8": ECC_U8, "uint16": ECC_U16, "float32": ECC_F32}.get(name, 0)
        _DTYPE_CODES[dt] = code
    return code


def _check(h, rc: int) -> int:
    if rc < 0:
        msg = load().ecc_last_error(h)
        raise EccError(rc, msg.decode() if msg else "")
    return rc


def _dims(shape):
    return (C.c_int64 * max(1, len(shape)))(*[int(s) for s in shape])


def _data_ptr(image):
    """(pointer, keepalive) of a numpy array or torch tensor (C order)."""
    if isinstance(image, np.ndarray):
        arr = np.ascontiguousarray(image)
        return arr.ctypes.data_as(C.c_void_p), arr
    if not image.is_contiguous():
        image = image.contiguous()
    return C.c_void_p(image.data_ptr()), image


class _ResultOwner:
    """Holds a library-allocated ecc_result whose buffers numpy arrays view;
    releases them (ecc_result_free) when the last view is gone."""
    __slots__ = ("r",)

    def __init__(self, r: ecc_result):
        self.r = ecc_result()
        C.memmove(C.byref(self.r), C.byref(r), C.sizeof(ecc_result))

    def __del__(self):
        try:
            if _lib is not None:
                _lib.ecc_result_free(C.byref(self.r))
        except Exception:  # interpreter shutdown: the process frees everything
            pass


def _view(owner, ptr, n: int, ctype, dtype):
    buf = (ctype * n).from_address(C.cast(ptr, C.c_void_p).value)
    buf._owner = owner  # the buffer lives while any array viewing it does
    return np.frombuffer(buf, dtype=dtype)


def _result_to_numpy(r: ecc_result):
    """The curve (or (thresholds, chi) pairs) of r as numpy arrays. Buffers
    the library allocated are viewed in place and taken over (r is left
    empty, so a later ecc_result_free of it is a no-op); others are copied."""
    bins, npairs = int(r.bins), int(r.npairs)
    if not r.owned or (bins <= 0 and npairs <= 0):
        if bins > 0:
            return np.ctypeslib.as_array(r.curve, shape=(bins,)).copy()
        if npairs > 0:
            return (np.ctypeslib.as_array(r.thresholds, shape=(npairs,)).copy(),
                    np.ctypeslib.as_array(r.chi, shape=(npairs,)).copy())
        return np.zeros(0, np.float32), np.zeros(0, np.int64)
    owner = _ResultOwner(r)
    C.memset(C.byref(r), 0, C.sizeof(ecc_result))
    if bins > 0:
        return _view(owner, owner.r.curve, bins, C.c_int64, np.int64)
    return (_view(owner, owner.r.thresholds, npairs, C.c_float, np.float32),
            _view(owner, owner.r.chi, npairs, C.c_int64, np.int64))


def ecc_config_default() -> ecc_config:
    cfg = ecc_config()
    load().ecc_config_default(C.byref(cfg))
    return cfg


def ecc_create(config: ecc_config | None = None, **fields):
    lib = load()
    cfg = config if config is not None else ecc_config_default()
    for k, v in fields.items():
        setattr(cfg, k, v)
    h = C.c_void_p()
    rc = lib.ecc_create(C.byref(cfg), C.byref(h))
    if rc != ECC_OK:
        msg = lib.ecc_last_error(None)
        raise EccError(rc, msg.decode() if msg else "")
    return h


def ecc_destroy(h) -> None:
    load().ecc_destroy(h)
    for key in [k for k in _borrowed if k[0] == h.value]:
        del _borrowed[key]


def ecc_last_error(h) -> str:
    msg = load().ecc_last_error(h)
    return msg.decode() if msg else ""


def ecc_compute(h, image):
    """Curve of an integer image (int64[bins]) or (thresholds, chi) of a float
    image; `image` is a numpy array or a torch tensor (host or CUDA)."""
    lib = load()
    ptr, keep = _data_ptr(image)
    dims = _dims(image.shape)
    r = ecc_result()
    _check(h, lib.ecc_compute(h, ptr, dims, len(image.shape), _dtype_code(image.dtype),
                              C.byref(r)))
    try:
        return _result_to_numpy(r)
    finally:
        lib.ecc_result_free(C.byref(r))
        del keep


def ecc_compute_quantized(h, image, lo: float, hi: float, bins: int):
    """Curve (int64[bins]) of a float32 image (numpy array or torch tensor,
    host or CUDA) through the value transform code = clamp(floor((v - lo) *
    bins / (hi - lo)), 0, bins - 1)."""
    if _dtype_code(image.dtype) != ECC_F32:
        raise TypeError("ecc_compute_quantized takes a float32 image")
    lib = load()
    ptr, keep = _data_ptr(image)
    r = ecc_result()
    _check(h, lib.ecc_compute_quantized(h, ptr, _dims(image.shape), len(image.shape),
                                        C.c_float(lo), C.c_float(hi), int(bins), C.byref(r)))
    try:
        return _result_to_numpy(r)
    finally:
        lib.ecc_result_free(C.byref(r))
        del keep


def ecc_compute_device(h, d_image, bins: int, d_curve, stream=None) -> None:
    """Enqueues an integer CUDA-tensor image; writes the int64 CUDA tensor
    ``d_curve[bins]``; ``stream`` is a torch.cuda.Stream or None."""
    lib = load()
    dims = _dims(d_image.shape)
    st = C.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(h, lib.ecc_compute_device(h, C.c_void_p(d_image.data_ptr()), dims,
                                     len(d_image.shape), _dtype_code(d_image.dtype),
                                     int(bins), C.c_void_p(d_curve.data_ptr()), st))


def ecc_compute_vcec_chunk(h, planes, shape, z_lo: int, z_hi: int, bins: int):
    """Partial VCEC (int64[bins]) of planes [z_lo, z_hi) of an integer image of
    `shape`; `planes` holds planes [max(z_lo-1, 0), min(z_hi+1, shape[0]))
    (numpy or torch, host or CUDA)."""
    ptr, keep = _data_ptr(planes)
    out = np.zeros(int(bins), dtype=np.int64)
    _check(h, load().ecc_compute_vcec_chunk(h, ptr, _dims(shape), len(shape),
                                            _dtype_code(planes.dtype), int(z_lo), int(z_hi),
                                            out.ctypes.data_as(_I64P)))
    del keep
    return out


def ecc_device_status(h) -> int:
    return _check(h, load().ecc_device_status(h))


def ecc_stream_begin(h, shape, dtype):
    s = C.c_void_p()
    _check(h, load().ecc_stream_begin(h, _dims(shape), len(shape), _dtype_code(dtype),
                                      C.byref(s)))
    return s


def ecc_stream_push_slab(h, s, planes, z0: int) -> None:
    ptr, keep = _data_ptr(planes)
    _check(h, load().ecc_stream_push_slab(s, ptr, int(z0), int(planes.shape[0])))
    del keep


def ecc_stream_finish(h, s):
    lib = load()
    r = ecc_result()
    _check(h, lib.ecc_stream_finish(s, C.byref(r)))
    try:
        return _result_to_numpy(r)
    finally:
        lib.ecc_result_free(C.byref(r))


def ecc_stream_abort(s) -> None:
    load().ecc_stream_abort(s)


def ecc_stream_file(h, path, shape, dtype, offset: int = 0):
    """Curve of a raw C-order integer image stored at byte `offset` of the
    file `path`, streamed slab by slab."""
    lib = load()
    r = ecc_result()
    _check(h, lib.ecc_stream_file(h, os.fsencode(path), int(offset), _dims(shape), len(shape),
                                  _dtype_code(dtype), C.byref(r)))
    try:
        return _result_to_numpy(r)
    finally:
        lib.ecc_result_free(C.byref(r))


def ecc_compute_batch(h, images, bins=None):
    """Curves of a list of integer images (numpy or torch, host or CUDA) from
    one batched launch. Returns a list of int64 arrays (or EccError objects
    for images that failed)."""
    lib = load()
    n = len(images)
    descs = (ecc_image * max(n, 1))()
    keep = []
    for i, im in enumerate(images):
        ptr, k = _data_ptr(im)
        keep.append(k)
        descs[i].data = ptr.value
        for j, s in enumerate(im.shape):
            descs[i].dims[j] = int(s)
        descs[i].ndim = len(im.shape)
        descs[i].dtype = _dtype_code(im.dtype)
        descs[i].bins = int(bins[i]) if bins is not None else 0
    outs = (ecc_result * max(n, 1))()
    _check(h, lib.ecc_compute_batch(h, n, descs, outs))
    res = []
    for i in range(n):
        o = outs[i]
        if o.status != ECC_OK:
            res.append(EccError(o.status, f"image {i}"))
            lib.ecc_result_free(C.byref(o))
        else:
            res.append(_result_to_numpy(o))  # takes the buffers over
    return res


def ecc_submit(h, image) -> int:
    lib = load()
    ptr, keep = _data_ptr(image)
    rid = C.c_uint64()
    _check(h, lib.ecc_submit(h, ptr, _dims(image.shape), len(image.shape),
                             _dtype_code(image.dtype), C.byref(rid)))
    del keep
    return rid.value


# images of borrowed requests, kept alive until their request has finished
_borrowed = {}


def ecc_submit_borrowed(h, image) -> int:
    """ecc_submit without the copy on return: the library reads the image
    (pinned host memory) until the request has finished; the binding holds a
    reference to it until ecc_poll reports the request done or failed."""
    lib = load()
    ptr, keep = _data_ptr(image)
    rid = C.c_uint64()
    _check(h, lib.ecc_submit_borrowed(h, ptr, _dims(image.shape), len(image.shape),
                                      _dtype_code(image.dtype), C.byref(rid)))
    _borrowed[(h.value, rid.value)] = keep
    return rid.value


def ecc_poll(h, req_id: int, timeout_us: int = 0):
    """(status, curve or None)."""
    lib = load()
    r = ecc_result()
    rc = lib.ecc_poll(h, C.c_uint64(req_id), C.byref(r), int(timeout_us))
    if rc not in (ECC_PENDING, ECC_ERR_TIMEOUT):
        _borrowed.pop((h.value, req_id), None)
    if rc == ECC_OK:
        try:
            return rc, _result_to_numpy(r)
        finally:
            lib.ecc_result_free(C.byref(r))
    if rc in (ECC_PENDING, ECC_ERR_TIMEOUT):
        return rc, None
    _check(h, rc)
    return rc, None


def ecc_request_latency_us(h, req_id: int) -> float:
    v = C.c_double()
    _check(h, load().ecc_request_latency_us(h, C.c_uint64(req_id), C.byref(v)))
    return v.value


def ecc_request_trace_us(h, req_id: int):
    """(copied, launched, batch finished, done) microseconds after submit; -1
    for a stage that did not happen."""
    st = (C.c_double * 4)()
    _check(h, load().ecc_request_trace_us(h, C.c_uint64(req_id), st))
    return tuple(st)


def ecc_launch_count(h) -> int:
    return int(load().ecc_launch_count(h))


def ecc_set_profiling(h, on: bool) -> None:
    _check(h, load().ecc_set_profiling(h, 1 if on else 0))


def ecc_profile_read(h):
    """(summed contribution-kernel milliseconds, number of computations)."""
    ms, n = C.c_double(), C.c_int64()
    _check(h, load().ecc_profile_read(h, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def ecc_profile_span(h) -> float:
    """Device milliseconds spanned by the record the last ecc_profile_read returned."""
    ms = C.c_double()
    _check(h, load().ecc_profile_span(h, C.byref(ms)))
    return ms.value


def ecc_compute_device_noalloc(d_image, bins: int, d_curve, convention: int = ECC_CONV_V,
                               stream=None) -> int:
    """Status of the allocation-free integer entry point on CUDA tensors
    (``d_curve``: int64 CUDA tensor of ``bins`` entries)."""
    st = C.c_void_p(stream.cuda_stream) if stream is not None else None
    return int(load().ecc_compute_device_noalloc(
        C.c_void_p(d_image.data_ptr()), _dims(d_image.shape), len(d_image.shape),
        _dtype_code(d_image.dtype), int(bins), int(convention),
        C.c_void_p(d_curve.data_ptr()), st))
