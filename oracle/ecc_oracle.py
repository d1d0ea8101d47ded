"""Plain CPU oracle: Euler characteristic curve by explicit cell enumeration.

TEST INFRASTRUCTURE ONLY (see the package docstring): not importable from the
product path, never called by the CUDA library.

What it computes, and the passage each step follows (Heiss & Wagner,
"Streaming Algorithm for Euler Characteristic Curves of Multidimensional
Images"):

* Cells (Sec. 2, "Cubical Cell"): a product of d factors, each a unit interval
  [a, a+1] or a singleton {b}; dim = number of interval factors.
* The image complex (Sec. 2, "Consecutive Thresholded Images as Sublevel Set
  Filtrations"): voxel i = (i_1..i_d) is the top cell prod_k [i_k - 1, i_k]
  (here shifted to 0-based: voxel i covers prod_k [i_k, i_k + 1]); the complex is
  all voxels with all their faces.
* Filtration value (Sec. 2, "Sublevel Set Filtration", the extension f~): a voxel
  carries its gray value; any other cell the MINIMUM over the voxels that
  contain it. This is convention "V", the paper's.
* Euler characteristic (Sec. 2, "Euler Characteristic"): chi = sum_k (-1)^k n_k.
* VCEC and curve (Sec. 3, "Tracking the Changes"): a_t = chi(K_t) - chi(K_{t-1})
  with chi(empty) = 0, and the curve is the running sum (a_0, a_0 + a_1, ...).
  a_t is therefore the signed count of cells whose filtration value equals t.
* Integer range (Sec. 3, "Range of Values"): thresholds t in {0..m-1}.
* Other ranges (Sec. 3, "Other Ranges of Gray Values"): for float images the
  VCEC is keyed by the value itself (the paper's hash map); output is the list
  of (t, chi(K_t)) at the values t where a_t != 0, ascending. The same passage
  offers the alternative of transforming the values (shift, scale, round) into
  {0..m-1} and running the integer algorithm: `quantize_f32` is that
  transform, `ecc_quantized` its curve.

Convention "T" is the alternative the same section names in a footnote: the
dual complex, voxels as vertices, lower-star filtration. A cell is a box of
2^k voxel centres spanned by unit steps and takes the MAXIMUM of its vertices.

Nothing here uses neighbour masks, tie-breaks, or the per-voxel block
decomposition of Sec. 3 ("Tracking the Changes", Algorithm 1). Library
primitives used as steps: numpy minimum/maximum, bincount, unique, cumsum.
"""
from __future__ import annotations

import itertools

import numpy as np

# Stands for the value +inf of voxels outside the image (integer images).
SENTINEL_INT = np.iinfo(np.int32).max


def _exact_values(img: np.ndarray):
    """Return (values, sentinel) in a type where min/max and equality are exact.

    Unsigned/signed integers up to 31 bits go to int32 (sentinel 2^31-1 is
    above every representable input value); floats go to float64 with -0.0
    normalised to +0.0 (IEEE equality already treats them as one value; the
    normalisation only fixes which bit pattern represents it) and +inf as the
    sentinel. NaN and +-inf inputs are rejected: the paper reserves infinity for
    the collar of outside voxels (Sec. 4, limitations).
    """
    if img.dtype.kind in "ui":
        if img.size and (int(img.max()) >= SENTINEL_INT or int(img.min()) < 0):
            raise ValueError("integer values must lie in [0, 2^31 - 1)")
        return img.astype(np.int32), SENTINEL_INT
    if img.dtype.kind == "f":
        v = img.astype(np.float64) + 0.0
        if not np.all(np.isfinite(v)):
            raise ValueError("NaN or infinite values are not gray values")
        return v, np.inf
    raise TypeError(f"unsupported dtype {img.dtype}")


def _sl(a: np.ndarray, axis: int, lo: int, hi: int) -> np.ndarray:
    idx = [slice(None)] * a.ndim
    idx[axis] = slice(lo, hi)
    return a[tuple(idx)]


def cells_V(img: np.ndarray, lo: int = 0, hi: int | None = None):
    """Yield (dim, values) for every cell type of the paper's complex (conv. V).

    A cell type picks, per axis k, an interval [a, a+1] with 0 <= a < n_k or a
    singleton {b} with 0 <= b <= n_k. The voxels containing such a cell are, per
    axis, {a} for an interval and {b-1, b} intersected with [0, n_k) for a
    singleton. Its value is the minimum over those voxels. ``values`` holds that
    minimum for every cell of the type (one array entry per cell).

    ``lo``/``hi`` restrict the axis-0 coordinate (a or b) of the enumerated
    cells to [lo, hi); the default enumerates all cells. Disjoint ranges
    partition the cell set, which is what the chunked streaming of Sec. 3
    ("Streaming") relies on.
    """
    n0 = img.shape[0]
    if hi is None:
        hi = n0 + 1
    lo, hi = max(lo, 0), min(hi, n0 + 1)
    if img.size == 0 or lo >= hi:
        return
    # Padded coordinate p along every axis stands for voxel p - 1; padded
    # entries outside the image hold the sentinel (+inf). Along axis 0 only
    # padded rows [lo, hi + 1) are needed.
    p_lo, p_hi = lo, min(hi + 1, n0 + 2)
    v_lo, v_hi = max(p_lo - 1, 0), min(p_hi - 1, n0)
    vals, sentinel = _exact_values(img[v_lo:v_hi])
    pad = [(1 if p_lo == 0 else 0, 1 if p_hi == n0 + 2 else 0)]
    pad += [(1, 1)] * (img.ndim - 1)
    P = np.pad(vals, pad, constant_values=sentinel)
    for kinds in itertools.product("IS", repeat=img.ndim):
        A = P
        for axis, kind in enumerate(kinds):
            n = img.shape[axis]
            if axis == 0:
                a_hi, b_hi = min(hi, n), min(hi, n + 1)
                if kind == "I":          # a in [lo, a_hi): padded a + 1
                    A = _sl(A, 0, lo + 1 - p_lo, a_hi + 1 - p_lo)
                else:                    # b in [lo, b_hi): padded b and b + 1
                    A = np.minimum(_sl(A, 0, lo - p_lo, b_hi - p_lo),
                                   _sl(A, 0, lo + 1 - p_lo, b_hi + 1 - p_lo))
            elif kind == "I":            # a in [0, n): padded a + 1
                A = _sl(A, axis, 1, n + 1)
            else:                        # b in [0, n]: padded b and b + 1
                A = np.minimum(_sl(A, axis, 0, n + 1), _sl(A, axis, 1, n + 2))
        if A.size == 0:
            continue
        # every cell contains at least one voxel of the image
        assert not np.any(A == sentinel)
        yield kinds.count("I"), A


def cells_T(img: np.ndarray, lo: int = 0, hi: int | None = None):
    """Yield (dim, values) for every cell type of the dual complex (conv. T).

    Voxel centres are the vertices. A cell type picks, per axis, a point a
    (0 <= a < n_k) or an edge [a, a+1] (0 <= a < n_k - 1); the cell's vertices
    are all voxels with coordinate a (point) or a, a+1 (edge) on each axis, and
    its value is their MAXIMUM (lower-star filtration). ``lo``/``hi`` restrict
    the axis-0 coordinate a to [lo, hi).
    """
    n0 = img.shape[0]
    if hi is None:
        hi = n0
    lo, hi = max(lo, 0), min(hi, n0)
    if img.size == 0 or lo >= hi:
        return
    vals, _ = _exact_values(img[lo:min(hi + 1, n0)])
    for kinds in itertools.product("PE", repeat=img.ndim):
        A = vals
        for axis, kind in enumerate(kinds):
            n = A.shape[axis]
            if axis == 0:
                if kind == "P":          # a in [lo, hi)
                    A = _sl(A, 0, 0, hi - lo)
                else:                    # a in [lo, min(hi, n0 - 1)): a, a + 1
                    e_hi = min(hi, n0 - 1)
                    A = np.maximum(_sl(A, 0, 0, e_hi - lo),
                                   _sl(A, 0, 1, e_hi - lo + 1))
            elif kind == "E":
                A = np.maximum(_sl(A, axis, 0, n - 1), _sl(A, axis, 1, n))
        if A.size == 0:
            continue
        yield kinds.count("E"), A


def _cells(img, convention, lo=0, hi=None):
    if convention == "V":
        return cells_V(img, lo, hi)
    if convention == "T":
        return cells_T(img, lo, hi)
    raise ValueError(f"unknown convention {convention!r}")


def vcec_int(img: np.ndarray, bins: int, convention: str = "V") -> np.ndarray:
    """VCEC a[0..bins-1] of an integer image: a_t = sum over cells with value t
    of (-1)^dim (Sec. 2 "Euler Characteristic" with Sec. 3 "Tracking the
    Changes"). Values >= bins raise ValueError (no clamping)."""
    return vcec_int_zrange(img, bins, 0, None, convention)


def vcec_int_zrange(img: np.ndarray, bins: int, lo: int, hi: int | None,
                    convention: str = "V") -> np.ndarray:
    """VCEC restricted to the cells whose axis-0 coordinate lies in [lo, hi).

    Summing this over a partition of the axis-0 coordinates gives
    ``vcec_int`` of the whole image: the chunk decomposition of Sec. 3
    ("Streaming", "Processing one Chunk").
    """
    if img.dtype.kind not in "ui":
        raise TypeError("integer image expected")
    a = np.zeros(bins, dtype=np.int64)
    for dim, A in _cells(img, convention, lo, hi):
        flat = A.ravel()
        if flat.size and int(flat.max()) >= bins:
            raise ValueError("a gray value is >= bins")
        a += (-1) ** dim * np.bincount(flat, minlength=bins).astype(np.int64)
    return a


def ecc_from_vcec(a: np.ndarray) -> np.ndarray:
    """Curve (a_0, a_0 + a_1, ..., sum_t a_t) (Sec. 3, "Post-Processing")."""
    return np.cumsum(np.asarray(a, dtype=np.int64), dtype=np.int64)


def ecc_int(img: np.ndarray, bins: int, convention: str = "V") -> np.ndarray:
    """Euler characteristic curve chi(K_t), t = 0..bins-1, of an integer image."""
    return ecc_from_vcec(vcec_int(img, bins, convention))


def ecc_pairs_float(img: np.ndarray, convention: str = "V"):
    """Float image: (thresholds, chi) at every value t with a_t != 0, ascending.

    The VCEC is keyed by the value itself (Sec. 3, "Other Ranges of Gray
    Values", the hash-map variant); chi(K_t) at a listed t is the running sum
    of a over all values <= t. Between two listed thresholds the curve is
    constant. Returns (float32 array, int64 array).
    """
    keys, weights = [], []
    for dim, A in _cells(img, convention):
        u, c = np.unique(A.ravel(), return_counts=True)
        keys.append(u)
        weights.append((-1) ** dim * c.astype(np.int64))
    if not keys:
        return np.zeros(0, np.float32), np.zeros(0, np.int64)
    k = np.concatenate(keys)
    w = np.concatenate(weights)
    order = np.argsort(k, kind="stable")
    k, w = k[order], w[order]
    starts = np.flatnonzero(np.r_[True, k[1:] != k[:-1]])
    a = np.add.reduceat(w, starts)
    t = k[starts]
    keep = a != 0
    return t[keep].astype(np.float32), np.cumsum(a[keep], dtype=np.int64)


def _chunk_voxel_planes(n0: int, lo: int, hi: int, convention: str):
    """Voxel planes [p0, p1) along axis 0 that contain the cells whose axis-0
    coordinate lies in [lo, hi): for V a singleton {b} lies in voxels b - 1
    and b, an interval [a, a + 1] in voxel a; for T a point a is voxel a and
    an edge [a, a + 1] joins voxels a and a + 1."""
    if convention == "V":
        return max(lo - 1, 0), min(hi, n0)
    return lo, min(hi + 1, n0)


def vcec_float_zrange(img: np.ndarray, lo: int, hi: int | None,
                      convention: str = "V"):
    """Float VCEC of the cells whose axis-0 coordinate lies in [lo, hi): the
    distinct values of those cells, ascending (float64), and the signed count
    sum (-1)^dim of the cells at each value, entries of count 0 left out.

    This is the hash map of Sec. 3 ("Other Ranges of Gray Values") restricted
    to one chunk of the partition of Sec. 3 ("Streaming"): the maps of a
    partition of the axis-0 coordinates, merged by value
    (`merge_vcec_float`), give the whole image's map.

    Every cell value is the value of one of the voxels the chunk's cells
    contain (the minimum of some of them for V, the maximum for T). Those
    voxels' values are first replaced by their rank among the distinct values
    present, a strictly increasing relabelling, with which minimum and maximum
    commute; the integer VCEC of the rank image (`vcec_int_zrange`, bins = the
    number of distinct values) is then the float map indexed by rank.
    """
    if img.dtype.kind != "f":
        raise TypeError("float image expected")
    n0 = img.shape[0]
    top = n0 + 1 if convention == "V" else n0  # one past the last axis-0 coordinate
    if convention not in ("V", "T"):
        raise ValueError(f"unknown convention {convention!r}")
    hi = top if hi is None else min(hi, top)
    lo = max(lo, 0)
    if img.size == 0 or lo >= hi:
        return np.zeros(0, np.float64), np.zeros(0, np.int64)
    p0, p1 = _chunk_voxel_planes(n0, lo, hi, convention)
    vals, _ = _exact_values(img[p0:p1])
    u, rank = np.unique(vals.ravel(), return_inverse=True)
    rank = rank.reshape(vals.shape).astype(np.int32)
    a = vcec_int_zrange(rank, len(u), lo - p0, hi - p0, convention)
    keep = a != 0
    return u[keep], a[keep]


def merge_vcec_float(parts):
    """Sum of float VCEC maps given as (values, counts) pairs: counts at equal
    values add up (Sec. 3, "Post-Processing": the partial VCECs are summed);
    values whose sum is 0 are left out."""
    parts = list(parts)
    if not parts:
        return np.zeros(0, np.float64), np.zeros(0, np.int64)
    k = np.concatenate([np.asarray(p[0], np.float64) for p in parts])
    w = np.concatenate([np.asarray(p[1], np.int64) for p in parts])
    if k.size == 0:
        return k, w
    order = np.argsort(k, kind="stable")
    k, w = k[order], w[order]
    starts = np.flatnonzero(np.r_[True, k[1:] != k[:-1]])
    a = np.add.reduceat(w, starts)
    t = k[starts]
    keep = a != 0
    return t[keep], a[keep]


def pairs_from_vcec_float(values: np.ndarray, a: np.ndarray):
    """(t, chi(K_t)) at every value t with a_t != 0, ascending: the running
    sum of the map (Sec. 3, "Post-Processing"). Returns (float32, int64)."""
    values = np.asarray(values, np.float64)
    a = np.asarray(a, np.int64)
    keep = a != 0
    return values[keep].astype(np.float32), np.cumsum(a[keep], dtype=np.int64)


def quantize_f32(img: np.ndarray, lo: float, hi: float, bins: int) -> np.ndarray:
    """The value transform of Sec. 3 ("Other Ranges of Gray Values": shift,
    scale, round into {0..m-1}), in the reading used here:

        q(v) = clamp(floor((v - lo) * s), 0, bins - 1),  s = bins / (hi - lo),

    every operation in float32 with round-to-nearest: hi - lo, then s, then
    v - lo, then the product; floor and clamp are exact. Values below lo go to
    0, values at or above hi to bins - 1. q is non-decreasing in v, so by the
    paper's remark the integer curve of q(f) is the float curve read at the
    largest value of each bin. NaN / +-inf and lo >= hi are rejected.
    Pinned in tests/test_oracle_pins.py (hand-computed codes, identity
    scaling, the transform relation against `ecc_pairs_float`)."""
    x = np.asarray(img, dtype=np.float32)
    if not np.all(np.isfinite(x)):
        raise ValueError("NaN or infinite value")
    lo32, hi32 = np.float32(lo), np.float32(hi)
    if not (np.isfinite(lo32) and np.isfinite(hi32) and lo32 < hi32):
        raise ValueError("need finite lo < hi")
    if not 1 <= bins <= 65536:
        raise ValueError("bins must be in 1..65536")
    span = np.float32(hi32 - lo32)
    scale = np.float32(np.float32(bins) / span)
    d = (x - lo32).astype(np.float32)
    p = (d * scale).astype(np.float32)
    code = np.floor(p.astype(np.float64))
    return np.clip(code, 0, bins - 1).astype(np.int64)


def ecc_quantized(img: np.ndarray, lo: float, hi: float, bins: int,
                  convention: str = "V") -> np.ndarray:
    """Curve chi({q(f) <= k}), k = 0..bins-1, of the transformed image."""
    return ecc_int(quantize_f32(img, lo, hi, bins), bins, convention)


def cell_counts(img_shape, convention: str = "V"):
    """n_k, the number of k-dimensional cells of the full complex of an image
    of this shape (every cell present, i.e. the threshold above all values)."""
    d = len(img_shape)
    n = np.zeros(d + 1, dtype=np.int64)
    if any(s == 0 for s in img_shape):
        return n
    for kinds in itertools.product((0, 1), repeat=d):
        # 1 = interval (V) / edge (T) factor
        cnt = 1
        for s, k in zip(img_shape, kinds):
            if convention == "V":
                cnt *= s if k else s + 1
            else:
                cnt *= s - 1 if k else s
        n[sum(kinds)] += cnt
    return n
