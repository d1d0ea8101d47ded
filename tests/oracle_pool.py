"""The CPU oracle over a large image in parallel: the image is a raw file,
each task computes the VCEC of the cells whose axis-0 coordinate lies in a
plane range (the chunk partition of Sec. 3, "Streaming") from a memory map,
and the task VCECs add up to the image's (integer images: a vector over the
bins; float images: maps keyed by value, merged by value). Test
infrastructure only."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _task(args):
    path, shape, dtype, bins, lo, hi, conv = args
    import oracle
    img = np.memmap(path, dtype=dtype, mode="r", shape=shape)
    return oracle.vcec_int_zrange(img, bins, lo, hi, conv)


def ecc_int_parallel(path, shape, dtype, bins: int, planes_per_task: int = 4,
                     procs: int | None = None, conv: str = "V") -> np.ndarray:
    """Curve of the raw C-order image in `path` by the oracle, one spawned
    process per host core."""
    procs = procs or max(1, os.cpu_count() or 1)
    n0 = shape[0]
    tasks = [(str(path), tuple(shape), np.dtype(dtype).str, bins, lo,
              min(lo + planes_per_task, n0 + 1), conv)
             for lo in range(0, n0 + 1, planes_per_task)]
    total = np.zeros(bins, dtype=np.int64)
    with mp.get_context("spawn").Pool(procs) as pool:
        for part in pool.imap_unordered(_task, tasks):
            total += part
    import oracle
    return oracle.ecc_from_vcec(total)


def _task_float(args):
    path, shape, dtype, lo, hi, conv = args
    import oracle
    img = np.memmap(path, dtype=dtype, mode="r", shape=shape)
    return oracle.vcec_float_zrange(img, lo, hi, conv)


def ecc_pairs_float_parallel(path, shape, planes_per_task: int = 8,
                             procs: int | None = None, conv: str = "V"):
    """(thresholds, chi) pairs of the raw C-order float32 image in `path` by
    the oracle, one spawned process per host core."""
    procs = procs or max(1, os.cpu_count() or 1)
    n0 = shape[0]
    top = n0 + 1 if conv == "V" else n0
    tasks = [(str(path), tuple(shape), np.dtype(np.float32).str, lo,
              min(lo + planes_per_task, top), conv)
             for lo in range(0, top, planes_per_task)]
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = list(pool.imap_unordered(_task_float, tasks))
    import oracle
    return oracle.pairs_from_vcec_float(*oracle.merge_vcec_float(parts))
