"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each pin is a closed form, a textbook topological value, an invariant of the
Euler characteristic, or a connected-component count by a library labeller
(scipy.ndimage.label) combined with the Euler-Poincare formula
chi = b0 - b1 (+ b2) of Sec. 2 ("Euler Characteristic"). The last test plants
plausible mistakes in the oracle and checks that some pin catches each one.
"""
import itertools

import numpy as np
import pytest
from scipy import ndimage

import oracle
from oracle import ecc_oracle

CONVS = ("V", "T")


# --------------------------------------------------------------------------
# independent reference quantities
# --------------------------------------------------------------------------

def runs_1d(mask: np.ndarray) -> int:
    """Number of maximal runs of True in a 1D mask (its connected components;
    a 1D set has no holes, so this is its Euler characteristic)."""
    m = np.r_[False, mask.astype(bool)]
    return int(np.sum(m[1:] & ~m[:-1]))


def chi_2d_unionfind(mask: np.ndarray, conv: str) -> int:
    """chi = b0 - b1 of the thresholded 2D set, by component labelling.

    V (closed pixels, 8-connected set; the footnote on connectivity in Sec. 2):
    b0 = 8-components of the set, b1 = bounded 4-components of the complement.
    T (pixels as vertices of the dual grid): b0 = 4-components of the set,
    b1 = bounded 8-components of the complement.
    """
    four = ndimage.generate_binary_structure(2, 1)
    eight = ndimage.generate_binary_structure(2, 2)
    s_set, s_comp = (eight, four) if conv == "V" else (four, eight)
    b0 = ndimage.label(mask, structure=s_set)[1]
    comp = np.pad(~mask.astype(bool), 1, constant_values=True)
    b1 = ndimage.label(comp, structure=s_comp)[1] - 1
    return b0 - b1


def curve_from(img, chi_of_mask, bins):
    return np.array([chi_of_mask(img <= t) for t in range(bins)], dtype=np.int64)


# --------------------------------------------------------------------------
# closed forms and invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("shape", [(5,), (3, 4), (2, 3, 4), (2, 2, 3, 2), (1, 1, 1)])
def test_constant_image(conv, shape):
    """A constant image c: the box is contractible, so chi = 1 from t = c on."""
    c = 3
    img = np.full(shape, c, dtype=np.uint8)
    e = oracle.ecc_int(img, 8, conv)
    assert e.tolist() == [0] * c + [1] * (8 - c)


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("shape", [(7,), (6, 5), (4, 3, 5), (3, 2, 3, 3)])
def test_zero_below_min_one_at_top(conv, shape):
    rng = np.random.default_rng(1)
    img = rng.integers(3, 9, size=shape).astype(np.uint8)
    e = oracle.ecc_int(img, 12, conv)
    assert np.all(e[: int(img.min())] == 0)
    assert np.all(e[int(img.max()):] == 1)


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("shape", [(1,), (4,), (3, 5), (2, 3, 4), (2, 3, 2, 2)])
def test_full_complex_counts(conv, shape):
    """n_k of the complete complex: the vertex count (n+1)^d (V) or n^d (T),
    and chi = 1 (the closed box is contractible)."""
    n = oracle.cell_counts(shape, conv)
    if conv == "V":
        assert n[0] == np.prod([s + 1 for s in shape])
        assert n[-1] == np.prod(shape)
    else:
        assert n[0] == np.prod(shape)
    assert int(np.sum(n * (-1) ** np.arange(len(n)))) == 1
    img = np.zeros(shape, np.uint8)
    cnt = np.zeros(len(shape) + 1, np.int64)
    cells = oracle.cells_V(img) if conv == "V" else oracle.cells_T(img)
    for dim, A in cells:
        cnt[dim] += A.size
    assert cnt.tolist() == n.tolist()


def test_empty_image():
    for conv in CONVS:
        assert oracle.ecc_int(np.zeros((0, 4), np.uint8), 4, conv).tolist() == [0] * 4


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("seed", range(6))
def test_1d_runs(conv, seed):
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 6, size=int(rng.integers(1, 40))).astype(np.uint8)
    ref = curve_from(img, runs_1d, 6)
    assert oracle.ecc_int(img, 6, conv).tolist() == ref.tolist()


@pytest.mark.parametrize("n", range(2, 10))
@pytest.mark.parametrize("phase", [0, 1])
def test_checkerboard(n, phase):
    """0/1 checkerboard at t = 0. V: the zero pixels' closed squares meet only at
    corners: vertices (n+1)^2 - k (k = corner pixels equal to 1, whose outer
    vertex is missing), edges 4Z, squares Z, so chi = (n+1)^2 - k - 3Z.
    T: the zero pixels are isolated vertices, chi = Z."""
    i, j = np.indices((n, n))
    img = ((i + j + phase) % 2).astype(np.uint8)
    z = int(np.sum(img == 0))
    corners = [img[0, 0], img[0, -1], img[-1, 0], img[-1, -1]]
    k = int(sum(int(c) for c in corners))
    assert oracle.ecc_int(img, 2, "V")[0] == (n + 1) ** 2 - k - 3 * z
    assert oracle.ecc_int(img, 2, "T")[0] == z


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("seed", range(12))
def test_2d_euler_poincare(conv, seed):
    rng = np.random.default_rng(100 + seed)
    shape = tuple(int(x) for x in rng.integers(1, 12, size=2))
    img = rng.integers(0, 5, size=shape).astype(np.uint8)
    ref = curve_from(img, lambda m: chi_2d_unionfind(m, conv), 5)
    assert oracle.ecc_int(img, 5, conv).tolist() == ref.tolist()


def _chi_of_factor(img, conv, bins):
    if img.ndim == 1:
        return curve_from(img, runs_1d, bins)
    return curve_from(img, lambda m: chi_2d_unionfind(m, conv), bins)


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("dims", [(1, 1), (2, 1), (1, 2), (2, 2), (1, 1, 1), (2, 1, 1)])
@pytest.mark.parametrize("seed", range(3))
def test_product_formula(conv, dims, seed):
    """f(x, y) = max(g(x), h(y)) has sublevel sets G_t x H_t, and the Euler
    characteristic is multiplicative on products; f = min(g, h) has sublevel
    sets G_t x box + box x H_t, whose chi is chi_G + chi_H - chi_G chi_H.
    The factors' curves come from run counts (1D) or labelling (2D)."""
    rng = np.random.default_rng(200 + seed)
    bins = 5
    factors = []
    for d in dims:
        shape = tuple(int(x) for x in rng.integers(2, 6 if d == 2 else 9, size=d))
        factors.append(rng.integers(0, bins, size=shape).astype(np.uint8))
    f_max, f_min = factors[0], factors[0]
    ref_max = _chi_of_factor(factors[0], conv, bins)
    ref_min = ref_max.copy()
    for g in factors[1:]:
        eg = _chi_of_factor(g, conv, bins)
        ext = (slice(None),) * f_max.ndim + (None,) * g.ndim
        f_max = np.maximum(f_max[ext], g)
        f_min = np.minimum(f_min[ext], g)
        ref_max = ref_max * eg
        ref_min = ref_min + eg - ref_min * eg
    assert f_max.ndim <= 4
    assert oracle.ecc_int(f_max, bins, conv).tolist() == ref_max.tolist()
    assert oracle.ecc_int(f_min, bins, conv).tolist() == ref_min.tolist()


def _box(shape, inner):
    """Binary image: value 0 on the set ``inner`` (a boolean array), 1 elsewhere."""
    img = np.ones(shape, np.uint8)
    img[inner] = 0
    return img


def designed_shapes_3d():
    """(name, image, chi_V, chi_T) with textbook Euler characteristics: ball 1,
    sphere shell 2, solid torus 0, genus-2 handlebody -1, ball with k point
    cavities 1 + k. Shapes are thick so both conventions agree, except the two
    touching boxes: closed cubes meeting at a vertex or an edge are connected
    and contractible (V), voxel centres without a unit step between them are
    not (T)."""
    S = (9, 11, 12)
    out = []
    m = np.zeros(S, bool); m[2:7, 2:9, 2:10] = True
    out.append(("ball", _box(S, m), 1, 1))
    shell = m.copy(); shell[3:6, 3:8, 3:9] = False
    out.append(("shell", _box(S, shell), 2, 2))
    torus = m.copy(); torus[:, 5, 5] = False
    out.append(("solid torus", _box(S, torus), 0, 0))
    g2 = torus.copy(); g2[:, 5, 8] = False
    out.append(("genus 2", _box(S, g2), -1, -1))
    cav = m.copy(); cav[4, 4, 4] = False; cav[4, 6, 7] = False; cav[3, 4, 7] = False
    out.append(("three cavities", _box(S, cav), 4, 4))
    two = np.zeros(S, bool); two[1:4, 1:4, 1:4] = True; two[4:7, 4:7, 4:7] = True
    out.append(("boxes touching at a vertex", _box(S, two), 1, 2))
    two_e = np.zeros(S, bool); two_e[1:4, 1:4, 1:4] = True; two_e[1:4, 4:7, 4:7] = True
    out.append(("boxes touching at an edge", _box(S, two_e), 1, 2))
    return out


@pytest.mark.parametrize("case", designed_shapes_3d(), ids=lambda c: c[0])
def test_designed_shapes_3d(case):
    _, img, chi_v, chi_t = case
    assert oracle.ecc_int(img, 2, "V")[0] == chi_v
    assert oracle.ecc_int(img, 2, "T")[0] == chi_t
    assert oracle.ecc_int(img, 2, "V")[1] == 1


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_point_cavity(conv, d):
    """A box missing one interior voxel deformation-retracts onto a sphere
    S^{d-1}: chi = 1 + (-1)^(d-1)."""
    shape = (5,) * d
    m = np.ones(shape, bool)
    m[(2,) * d] = False
    assert oracle.ecc_int(_box(shape, m), 2, conv)[0] == 1 + (-1) ** (d - 1)


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("shape", [(13,), (9, 7), (6, 5, 7), (5, 4, 3, 4)])
def test_chunk_additivity(conv, shape):
    """Cells partitioned by their axis-0 coordinate (the chunks of Sec. 3,
    "Streaming") give VCECs that sum to the whole image's."""
    rng = np.random.default_rng(7)
    img = rng.integers(0, 9, size=shape).astype(np.uint16)
    whole = oracle.vcec_int(img, 9, conv)
    n0 = shape[0]
    cuts = sorted(set([0, n0 + 1] + [int(x) for x in rng.integers(0, n0 + 1, size=3)]))
    parts = sum(oracle.vcec_int_zrange(img, 9, lo, hi, conv)
                for lo, hi in zip(cuts[:-1], cuts[1:]))
    assert parts.tolist() == whole.tolist()


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("shape", [(17,), (7, 6), (4, 5, 3), (3, 3, 3, 4)])
def test_float_monotone_transform(conv, shape):
    """Sec. 3 ("Other Ranges of Gray Values"): a strictly increasing transform
    of the values moves the curve's domain and nothing else. The float pairs of
    phi(img) must be (phi(t), chi(t)) at the integer thresholds with a_t != 0."""
    rng = np.random.default_rng(11)
    img = rng.integers(0, 10, size=shape).astype(np.uint8)
    phi = lambda t: np.float32(np.exp(0.37 * t) - 3.0)  # noqa: E731
    a = oracle.vcec_int(img, 10, conv)
    e = oracle.ecc_from_vcec(a)
    nz = np.flatnonzero(a)
    t, chi = oracle.ecc_pairs_float(phi(img.astype(np.float64)).astype(np.float32), conv)
    assert t.tolist() == [phi(x) for x in nz]
    assert chi.tolist() == e[nz].tolist()


def _float_chunk_pin(conv, shape, seed):
    """Sec. 3 ("Streaming" with "Other Ranges of Gray Values"): the float maps
    of the chunks of any partition of the axis-0 coordinates, merged by value,
    give the whole image's pairs as the plain per-cell-type enumeration
    (`ecc_pairs_float`) computes them. Values repeat (ties across chunks)."""
    rng = np.random.default_rng(seed)
    img = rng.normal(size=shape).astype(np.float32)
    flat = img.reshape(-1)
    flat[rng.integers(0, flat.size, size=flat.size // 3)] = flat[0]  # ties
    flat[rng.integers(0, flat.size, size=2)] = -0.0
    want_t, want_chi = oracle.ecc_pairs_float(img, conv)
    n0 = shape[0]
    top = n0 + 1 if conv == "V" else n0
    cuts = sorted(set([0, top] + [int(x) for x in rng.integers(0, top + 1, size=3)]))
    for cc in (cuts, [0, top], list(range(top + 1))):
        parts = [oracle.vcec_float_zrange(img, lo, hi, conv) for lo, hi in zip(cc[:-1], cc[1:])]
        t, chi = oracle.pairs_from_vcec_float(*oracle.merge_vcec_float(parts))
        assert t.tolist() == want_t.tolist()
        assert chi.tolist() == want_chi.tolist()


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("shape", [(13,), (9, 7), (6, 5, 7), (5, 4, 3, 4), (1, 3, 3), (2, 1, 4, 3)])
def test_float_chunk_additivity(conv, shape):
    _float_chunk_pin(conv, shape, 17)


@pytest.mark.parametrize("name", ["lower collar plane dropped", "upper collar plane dropped"])
def test_planted_float_chunk_mistake_is_caught(name, monkeypatch):
    """A chunk that misses the voxel plane below (V) or above (T) its cells
    gets the values of its boundary cells wrong: the chunk pin must fail."""
    good = ecc_oracle._chunk_voxel_planes
    if name == "lower collar plane dropped":
        bad = lambda n0, lo, hi, c: (lo, good(n0, lo, hi, c)[1]) if c == "V" \
            else good(n0, lo, hi, c)  # noqa: E731
        conv = "V"
    else:
        bad = lambda n0, lo, hi, c: (lo, min(hi, n0)) if c == "T" \
            else good(n0, lo, hi, c)  # noqa: E731
        conv = "T"
    monkeypatch.setattr(ecc_oracle, "_chunk_voxel_planes", bad)
    with pytest.raises((AssertionError, ValueError, IndexError)):
        _float_chunk_pin(conv, (6, 5, 7), 17)


def test_float_negative_zero_is_zero():
    img = np.array([[0.0, -0.0], [1.0, -0.0]], dtype=np.float32)
    t, chi = oracle.ecc_pairs_float(img, "V")
    assert np.signbit(t).tolist() == [False] * len(t)
    t2, chi2 = oracle.ecc_pairs_float(np.abs(img), "V")
    assert t.tolist() == t2.tolist() and chi.tolist() == chi2.tolist()


def test_rejects_bad_values():
    with pytest.raises(ValueError):
        oracle.ecc_int(np.array([1, 9], np.uint8), 8)
    with pytest.raises(ValueError):
        oracle.ecc_pairs_float(np.array([1.0, np.nan], np.float32))


# --------------------------------------------------------------------------
# the value transform (Sec. 3, "Other Ranges of Gray Values")
# --------------------------------------------------------------------------

def test_quantize_hand_codes():
    """q(v) = clamp(floor((v - lo) * bins / (hi - lo)), 0, bins - 1) on values
    where every float32 step is exact: lo = -1, hi = 1, bins = 4 (scale 2)."""
    v = np.array([-3.0, -1.0, -0.75, -0.5, -0.25, 0.0, 0.25, 0.5, 0.75, 0.999, 1.0, 7.5],
                 np.float32)
    want = [0, 0, 0, 1, 1, 2, 2, 3, 3, 3, 3, 3]
    assert oracle.quantize_f32(v, -1.0, 1.0, 4).tolist() == want


def test_quantize_identity_scale():
    """lo = 0, hi = bins (scale 1): integer-valued floats map to themselves,
    so the transformed curve is the integer curve of the same values."""
    rng = np.random.default_rng(21)
    img = rng.integers(0, 50, size=(5, 6, 7))
    f = img.astype(np.float32)
    assert oracle.quantize_f32(f, 0.0, 50.0, 50).tolist() == img.tolist()
    for conv in CONVS:
        assert (oracle.ecc_quantized(f, 0.0, 50.0, 50, conv).tolist() ==
                oracle.ecc_int(img, 50, conv).tolist())


@pytest.mark.parametrize("conv", CONVS)
@pytest.mark.parametrize("shape", [(23,), (9, 8), (5, 4, 6), (3, 4, 3, 3)])
def test_quantized_curve_is_float_curve_at_bin_tops(conv, shape):
    """Sec. 3: the integer algorithm on transformed values gives the float
    curve with its domain transformed. q is non-decreasing, so {q(f) <= k} =
    {f <= m_k} with m_k the largest image value whose code is <= k: the
    transformed curve at k is the float curve (the independent float-keyed
    enumeration) read at m_k, and 0 where no value has a code <= k."""
    rng = np.random.default_rng(31 + len(shape))
    img = rng.normal(size=shape).astype(np.float32)
    lo, hi, bins = -1.3, 1.1, 37
    qc = oracle.ecc_quantized(img, lo, hi, bins, conv)
    t, chi = oracle.ecc_pairs_float(img, conv)
    codes = oracle.quantize_f32(img, lo, hi, bins).ravel()
    vals = img.ravel()
    for k in range(bins):
        sel = vals[codes <= k]
        want = 0
        if sel.size:
            i = np.searchsorted(t, sel.max(), side="right") - 1
            want = int(chi[i]) if i >= 0 else 0
        assert qc[k] == want


def test_quantize_monotone_and_rejects():
    v = np.sort(np.random.default_rng(5).normal(size=10000).astype(np.float32) * 3)
    q = oracle.quantize_f32(v, -2.0, 2.5, 1000)
    assert np.all(np.diff(q) >= 0) and q.min() == 0 and q.max() == 999
    with pytest.raises(ValueError):
        oracle.quantize_f32(np.array([np.nan], np.float32), 0.0, 1.0, 4)
    with pytest.raises(ValueError):
        oracle.quantize_f32(np.zeros(3, np.float32), 1.0, 1.0, 4)
    with pytest.raises(ValueError):
        oracle.quantize_f32(np.zeros(3, np.float32), 0.0, 1.0, 70000)


def test_quantize_float32_rounding():
    """The code is decided in float32: 0.7f = 0.69999998807..., times 10 is
    6.9999998807... exactly, which rounds to 7.0 in float32 (the nearest
    float32 values are 6.99999952... and 7.0), so the code is 7, not the 6 of
    exact arithmetic."""
    v = np.array([0.7, 0.3, 0.1], np.float32)
    assert oracle.quantize_f32(v, 0.0, 1.0, 10).tolist() == [7, 3, 1]


def _quant_pins_pass() -> bool:
    try:
        test_quantize_hand_codes()
        test_quantize_identity_scale()
        test_quantize_float32_rounding()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("name", ["ceil instead of floor", "no clamp", "no float32 rounding"])
def test_planted_quantizer_mistake_is_caught(name, monkeypatch):
    swap = {"ceil instead of floor": {"floor": np.ceil},
            "no clamp": {"clip": lambda a, lo, hi: a},
            "no float32 rounding": {"float32": np.float64}}[name]
    monkeypatch.setattr(ecc_oracle, "np", _NumpyWith(**swap))
    assert not _quant_pins_pass(), f"no pin catches: {name}"


# --------------------------------------------------------------------------
# planted mistakes: each must be caught by at least one pin above
# --------------------------------------------------------------------------

class _NumpyWith:
    """numpy with one function swapped, to plant a mistake in the oracle."""

    def __init__(self, **swap):
        self._swap = swap

    def __getattr__(self, name):
        return self._swap.get(name, getattr(np, name))


def _mutations():
    def max_for_min(mp):
        mp.setattr(ecc_oracle, "np", _NumpyWith(minimum=np.maximum))

    def min_for_max(mp):
        mp.setattr(ecc_oracle, "np", _NumpyWith(maximum=np.minimum))

    def wrap_cells(transform):
        def plant(mp):
            orig_v, orig_t = ecc_oracle.cells_V, ecc_oracle.cells_T
            mp.setattr(ecc_oracle, "cells_V", lambda *a: transform(orig_v(*a)))
            mp.setattr(ecc_oracle, "cells_T", lambda *a: transform(orig_t(*a)))
        return plant

    drop_vertices = wrap_cells(lambda g: ((d, A) for d, A in g if d != 0))
    flip_parity = wrap_cells(lambda g: ((d + 1, A) for d, A in g))
    drop_top = wrap_cells(lambda g: ((d, A) for d, A in g if d != A.ndim))
    off_by_one = wrap_cells(lambda g: ((d, A[..., :-1] if d < A.ndim else A) for d, A in g))

    def bad_scan(mp):
        mp.setattr(ecc_oracle, "ecc_from_vcec",
                   lambda a: np.cumsum(np.asarray(a, np.int64)[::-1])[::-1].copy())

    return {
        "max instead of min (V)": max_for_min,
        "min instead of max (T)": min_for_max,
        "vertices dropped": drop_vertices,
        "dimension parity flipped": flip_parity,
        "top cells dropped": drop_top,
        "last boundary layer dropped": off_by_one,
        "reversed prefix sum": bad_scan,
    }


def _all_pins_pass() -> bool:
    checks = [
        lambda: test_constant_image("V", (2, 3, 4)),
        lambda: test_constant_image("T", (2, 3, 4)),
        lambda: test_zero_below_min_one_at_top("V", (4, 3, 5)),
        lambda: test_zero_below_min_one_at_top("T", (4, 3, 5)),
        lambda: test_checkerboard(5, 0),
        lambda: test_2d_euler_poincare("V", 3),
        lambda: test_2d_euler_poincare("T", 3),
        lambda: test_product_formula("V", (2, 1), 0),
        lambda: test_product_formula("T", (2, 1), 0),
        lambda: test_point_cavity("V", 3),
        lambda: test_point_cavity("T", 3),
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return False
    return True


def test_pins_pass_unmutated():
    assert _all_pins_pass()


@pytest.mark.parametrize("name", list(_mutations()))
def test_planted_mistake_is_caught(name, monkeypatch):
    _mutations()[name](monkeypatch)
    assert not _all_pins_pass(), f"no pin catches: {name}"


def test_oracle_package_imports_nothing_from_the_product():
    src = open(ecc_oracle.__file__).read()
    assert "paper_1705_02045_gb300" not in src
    assert "ctypes" not in src


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_itertools_cell_types(d):
    """2^d cell types, each counted once (sanity of the enumeration helper)."""
    img = np.zeros((2,) * d, np.uint8)
    types = [dim for dim, _ in oracle.cells_V(img)]
    assert sorted(types) == sorted(sum(k) for k in itertools.product((0, 1), repeat=d))


def test_golden_fixtures_reproduce():
    """The stored fixtures (written by tests/golden/make_golden.py from the
    oracle) still come out of the oracle unchanged."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_small.json")
    for rec in json.load(open(path)):
        img = np.array(rec["values"], dtype=rec["dtype"]).reshape(rec["shape"])
        for conv in CONVS:
            if rec["dtype"] == "float32":
                t, chi = oracle.ecc_pairs_float(img, conv)
                assert [[float(a), int(b)] for a, b in zip(t, chi)] == rec["pairs_" + conv]
            else:
                a = oracle.vcec_int(img, rec["bins"], conv)
                nz = np.flatnonzero(a)
                assert [[int(x), int(a[x])] for x in nz] == rec["vcec_" + conv]
