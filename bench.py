"""Benchmark: Euler characteristic curves on one GB300, every configured workload.

Headline (one "step"): the whole hot path -- per-voxel change of Algorithm 1
(contribution kernel, block-private histogram, int64 merge) and the prefix
scan -- on a 512 x 512 x 512 uint8 image (seeded white noise, Gaussian
sigma = 4, requantised to 0..255; 256 thresholds), resident in HBM.

  value      Gvoxel/s from CUDA events around each step on the launching
             stream; L2 is flushed (256 MiB write) between steps, outside
             the timed events.
  e2e        same metric through ecc_compute() with the image in pinned host
             memory: host->device copy, kernels, device->host curve, all timed.
  roofline   contribution kernel, integer-logic bound (see alu_ops_per_voxel),
             with the HBM view (algorithmic bytes over its duration against
             the measured copy bandwidth) beside it.
  cpu_baseline  the CPU oracle on a bounded slab of the same image.

The same line carries the other workloads, each with its own value, roofline,
e2e and CPU baseline: ``configs`` holds the 2D 512^2 uint8 call, the 14-bit
3072 x 3072 x 1536 volume (resident, and streamed in z-slabs from pinned host
memory) and the 4D 128^4 float32 field (exact pairs); ``batched`` and
``serving`` the 4096-request mixed stream; ``h2d_peak`` the host-to-device
copy rate the streamed and end-to-end fractions are taken against.

N > 1 (torchrun): replicas, one image per rank, weak scaling; value is the
voxels of all ranks / the slowest rank's time (headline only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (512, 512, 512)
BINS = 256
SIGMA = 4.0
METRIC = "ECC Gvoxel/s & % HBM roofline; batched vs per-image launch; p50/p99 latency"
WORKLOAD = "3D 512x512x512 uint8, seeded white noise * Gaussian(sigma=4) requantised 0..255, 256 bins, HBM-resident"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, world: int) -> float:
    """Max of a per-rank scalar over the process group (NCCL on CUDA, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(voxels_per_rank: int, step_ms: float, world: int):
    """Replicas: every rank processes its own image; the job's throughput is
    all ranks' voxels over the slowest rank's step time. Returns
    (Gvoxel/s, slowest ms per step)."""
    slowest = _max_over_ranks(step_ms, world)
    return world * voxels_per_rank / (slowest * 1e-3) / 1e9, slowest


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits"], capture_output=True, text=True,
                    timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for name, v in zip(names, s[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def make_image(seed_offset: int = 1):
    from paper_1705_02045_gb300 import synth
    return synth.smooth_u8(SHAPE, SIGMA, synth.SEED_BASE + seed_offset)


# Integer logic pipe: 32-bit lanes per SM per clock. The bit-sliced
# contribution kernel is bound by it (ncu: ALU pipe ~78 % busy at 56 % issue
# activity, which puts the pipe at half the issue rate: 64 lanes/SM/clock).
ALU_LANES_PER_SM_CLK = 64
SM_MAX_MHZ_DEFAULT = 2070.0


def alu_ops_per_voxel(nb: int) -> float:
    """32-bit logic operations per voxel of the bit-sliced formulation, from
    its formulas (32 voxels per operation): 13 pair comparisons of nb planes
    plus the outside-mask op each; 12 edge triples (1 op) and 8 vertex boxes
    (2 ops); the 26-term count (21 full + 3 half adders, 2 ops each); the
    zero test (3); the byte -> bit-plane transpose (60 for 8 bits; two of
    them and 16 byte permutes for 16 bits); the centre row shifted left and
    right (2 nb funnel shifts) and the 10 shifted comparison words (2 ops)."""
    transpose = 60 if nb <= 8 else 2 * 60 + 16
    ops = 13 * (nb + 1) + (12 + 16) + 48 + 3 + transpose + 2 * nb + 20
    return ops / 32.0


def alu_peak_tops(num_sms: int, sm_max_mhz) -> float:
    return num_sms * ALU_LANES_PER_SM_CLK * float(sm_max_mhz or SM_MAX_MHZ_DEFAULT) * 1e6 / 1e12


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _oracle_planes(task):
    """Worker of the CPU baselines: the oracle's VCEC (integer image) or
    value-keyed map (float image) of the cells whose axis-0 coordinate lies
    in [lo, hi), reading the image from shared memory."""
    name, shape, dtype, bins, lo, hi = task
    from multiprocessing import shared_memory
    import oracle
    shm = shared_memory.SharedMemory(name=name)
    try:
        img = np.ndarray(shape, dtype=dtype, buffer=shm.buf)
        if img.dtype.kind == "f":
            oracle.vcec_float_zrange(img, lo, hi, "V")
        else:
            oracle.vcec_int_zrange(img, bins, lo, hi, "V")
    finally:
        shm.close()
    return hi - lo


def oracle_on_host_cores(img, bins: int, seconds: float):
    """The oracle, as it stands, over plane ranges of the image on every host
    core (a spawned process pool: one process per core, the image in shared
    memory), for about `seconds` of CPU work in all: one task of k planes per
    process, in as many rounds as that takes. Returns (voxels, wall seconds,
    processes, planes per task, rounds)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import oracle
    procs = max(1, os.cpu_count() or 1)
    t0 = time.perf_counter()
    if img.dtype.kind == "f":
        oracle.vcec_float_zrange(img, 0, 1, "V")
    else:
        oracle.vcec_int_zrange(img, bins, 0, 1, "V")
    one = max(time.perf_counter() - t0, 1e-3)
    # planes per task so that one round of tasks (one per process) takes
    # about `seconds`, at most the whole image split over the processes
    k = int(max(1, min(img.shape[0] // procs or 1, seconds / one)))
    rounds = int(max(1, min(16, round(seconds / (procs * k * one)))))
    shm = shared_memory.SharedMemory(create=True, size=img.nbytes)
    try:
        np.ndarray(img.shape, dtype=img.dtype, buffer=shm.buf)[...] = img
        tasks = [(shm.name, img.shape, img.dtype.str, bins, (i * k) % img.shape[0],
                  (i * k) % img.shape[0] + k) for i in range(procs)] * rounds
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map(_oracle_planes, [(shm.name, img.shape, img.dtype.str, bins, 0, 1)] * procs)
            t0 = time.perf_counter()
            planes = sum(pool.map(_oracle_planes, tasks, chunksize=1))
            wall = time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()
    return planes * int(np.prod(img.shape[1:])), wall, procs, k, rounds


def cpu_baseline(img, bins: int = BINS, seconds: float = 15.0, what: str = "the same 512^3 image"):
    """The oracle on a bounded sample of the same image, on all host cores."""
    vox, wall, procs, k, rounds = oracle_on_host_cores(img, bins, seconds)
    return {"value": vox / wall / 1e9, "unit": "Gvoxel/s", "cores": procs, "kind": "oracle",
            "sample": f"{rounds} rounds of {procs} processes x cells of {k} consecutive planes "
                      f"of {what}: {vox} voxels in {wall:.1f} s "
                      f"(~{wall * procs:.0f} s of CPU work; numpy oracle, one process per "
                      "host core)"}


def _numa_info(ptr: int):
    """NUMA node of the page at host address ptr, the GPU's node and the
    number of nodes (None where the system does not say)."""
    import ctypes
    info = {"buffer_node": None, "gpu_node": None, "nodes": None}
    try:
        info["nodes"] = len([n for n in os.listdir("/sys/devices/system/node")
                             if n.startswith("node") and n[4:].isdigit()])
    except OSError:
        pass
    try:
        libc = ctypes.CDLL(None, use_errno=True)
        nr = {"aarch64": 236, "x86_64": 239}.get(os.uname().machine)
        node = ctypes.c_int(-1)
        if nr is not None and libc.syscall(nr, ctypes.byref(node), None, ctypes.c_ulong(0),
                                           ctypes.c_void_p(ptr), ctypes.c_ulong(3)) == 0:
            info["buffer_node"] = node.value
    except Exception:
        pass
    try:
        bus = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=10).stdout.strip().lower()
        if bus:
            path = f"/sys/bus/pci/devices/{bus[-12:]}/numa_node"
            info["gpu_node"] = int(open(path).read().strip())
    except Exception:
        pass
    return info


def h2d_peak():
    """Pinned host -> device copy rate: one 4 GiB pinned buffer copied whole by
    one stream, and in equal parts by 2 and 4 concurrent streams (best of 3
    each), with the NUMA placement of the buffer and of the GPU."""
    import torch
    size = 4 << 30
    host = torch.empty(size, dtype=torch.uint8, pin_memory=True)
    host.fill_(1)
    dev = torch.empty(size, dtype=torch.uint8, device="cuda")
    rates = {}
    for ns in (1, 2, 4):
        streams = [torch.cuda.Stream() for _ in range(ns)]
        part = size // ns
        best = 0.0
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for i, st in enumerate(streams):
                with torch.cuda.stream(st):
                    dev[i * part:(i + 1) * part].copy_(host[i * part:(i + 1) * part],
                                                       non_blocking=True)
            torch.cuda.synchronize()
            best = max(best, size / (time.perf_counter() - t0) / 1e9)
        rates[str(ns)] = best
    info = _numa_info(host.data_ptr())
    del host, dev
    torch.cuda.empty_cache()
    return {"gbs": max(rates.values()), "by_streams": rates, "buffer_bytes": size, **info}


def alu_roofline(nvox: int, ops_per_voxel: float, kernel_s: float, alu_pk: float,
                 hbm_bytes: float, hbm_pk: float, hbm_kind: str, what: str):
    """Roofline object of an integer-logic bound kernel, with the HBM view of
    its algorithmic bytes beside it."""
    achieved = nvox * ops_per_voxel / kernel_s / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": alu_pk, "unit": "Tops/s",
            "frac": achieved / alu_pk, "traffic": None, "kernel": what,
            "kernel_ms": kernel_s * 1e3, "ops_per_voxel": ops_per_voxel,
            "peak_kind": "derived: SMs x 64 logic lanes/clock x max SM clock",
            "hbm": {"achieved": hbm_bytes / kernel_s / 1e9, "peak": hbm_pk, "unit": "GB/s",
                    "frac": hbm_bytes / kernel_s / 1e9 / hbm_pk, "peak_kind": hbm_kind}}


def make_requests(n: int, seed: int):
    """The mixed request stream (shapes/dtypes of synth.request_mix, smoothed
    fields sigma = 2 requantised to each dtype's range), generated on the GPU
    and returned as host numpy arrays with their bin counts."""
    from paper_1705_02045_gb300 import synth
    out = []
    for i, (shape, dt, bins) in enumerate(synth.request_mix(n, seed)):
        t = synth.smooth_int_torch(shape, 2.0, bins - 1, seed + 1 + i)
        out.append((t.cpu().numpy().astype(dt), bins))
    return out


def bench_batched(h, reqs, stream):
    """One launch sequence per image vs one batched launch, same device images.
    Both include copying every curve back to the host."""
    import torch
    from paper_1705_02045_gb300 import ecc
    dev = [torch.from_numpy(a).cuda() for a, _ in reqs]
    bins = [b for _, b in reqs]
    curves = [torch.empty(b, dtype=torch.int64, device="cuda") for b in bins]
    vox = sum(a.size for a, _ in reqs)

    def per_image():
        for d, b, c in zip(dev, bins, curves):
            ecc.ecc_compute_device(h, d, b, c, stream=stream)
        stream.synchronize()
        return [c.cpu() for c in curves]

    def batched():
        return ecc.ecc_compute_batch(h, dev, bins)

    # the C call alone, its image descriptors built once (as a caller
    # reusing them would), the results released after the timing
    import ctypes as C
    lib = ecc.load()
    n = len(dev)
    descs = (ecc.ecc_image * n)()
    for i, (d, b) in enumerate(zip(dev, bins)):
        descs[i].data = d.data_ptr()
        for j, sz in enumerate(d.shape):
            descs[i].dims[j] = int(sz)
        descs[i].ndim = d.dim()
        descs[i].dtype = ecc.ECC_U8 if d.dtype == torch.uint8 else ecc.ECC_U16
        descs[i].bins = int(b)
    outs = (ecc.ecc_result * n)()

    def batched_c():
        t0 = time.perf_counter()
        assert lib.ecc_compute_batch(h, n, descs, outs) == ecc.ECC_OK
        dt = time.perf_counter() - t0
        for i in range(n):
            lib.ecc_result_free(C.byref(outs[i]))
        return dt

    per_image()
    batched()
    batched_c()
    torch.cuda.synchronize()
    t_per, t_bat, t_c, k_ms = [], [], [], []
    for _ in range(3):
        t0 = time.perf_counter()
        ref = per_image()
        t_per.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        res = batched()
        t_bat.append(time.perf_counter() - t0)
        ecc.ecc_set_profiling(h, True)
        ecc.ecc_profile_read(h)
        t_c.append(batched_c())
        ecc.ecc_profile_read(h)
        ecc.ecc_set_profiling(h, False)
        k_ms.append(ecc.ecc_profile_span(h))
    same = all(np.array_equal(r.numpy(), b) for r, b in zip(ref, res))
    assert same, "batched curves differ from per-image curves"
    bench_batched.curves = [np.array(b) for b in res]
    tp, tb, tc = min(t_per), min(t_bat), min(t_c)
    kernel_s = k_ms[int(np.argmin(t_c))] / 1e3
    return {"images": len(reqs), "voxels": int(vox), "per_image_s": tp, "batched_s": tb,
            "speedup": tp / tb, "gvox_s_batched": vox / tb / 1e9,
            "gvox_s_per_image": vox / tp / 1e9, "identical": bool(same),
            "c_call_s": tc, "graphs_span_s": kernel_s, "c_call_over_graphs": tc / kernel_s,
            "timing": "per_image_s / batched_s: the Python calls (ecc_compute_device per "
                      "image then each curve to the host / ecc_compute_batch with its "
                      "argument marshalling and curve views), best of 3; c_call_s: "
                      "ecc_compute_batch itself with prepared descriptors; graphs_span_s: the "
                      "device time from the first of its batched graphs' start to the last "
                      "one's end (profiling events; the two slots' graphs overlap)"}


def _same_curve(served, batched) -> bool:
    """served (over at least as many bins) equals batched, then holds its last
    value: thresholds past the largest image value add no cells."""
    n = len(batched)
    return (len(served) >= n and np.array_equal(served[:n], batched)
            and bool(np.all(served[n:] == batched[-1])))


def bench_serving(h, reqs, rate_hz: float, seed: int, borrowed: bool = False, ref=None):
    """Requests submitted at Poisson arrival times (rate_hz), polled to
    completion; latency = submit -> completion as recorded by the library.
    rate_hz = 0: all submitted at once (saturated). Request images are in
    pinned host memory (as from a receive buffer registered with CUDA);
    borrowed: ecc_submit_borrowed, which reads them in place instead of
    copying each before it returns. One untimed pass of the same requests on
    the same handle comes first (the warm-up of a long-running server: batch
    graphs captured, result slabs and the device memory pool sized). ref:
    the curves of the same images from the batched call; every served curve
    of the warm-up pass and every 16th of the timed pass must equal them (a
    served curve spans the handle's default bins, 65536 for uint16, and past
    the last batched bin it stays at the whole image's characteristic)."""
    from paper_1705_02045_gb300 import ecc
    submit = ecc.ecc_submit_borrowed if borrowed else ecc.ecc_submit
    warm = [submit(h, img) for img, _ in reqs]
    checked = 0
    for i, rid in enumerate(warm):
        st, curve = ecc.ecc_poll(h, rid, timeout_us=600_000_000)
        assert st == ecc.ECC_OK
        if ref is not None and i < len(ref):
            assert _same_curve(curve, ref[i]), f"served curve {i} differs from the batched one"
            checked += 1
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=len(reqs)) if rate_hz > 0 else np.zeros(len(reqs))
    arrivals = np.cumsum(gaps)
    ids = [None] * len(reqs)

    def submitter():
        t0 = time.perf_counter()
        for i, (img, _) in enumerate(reqs):
            dt = arrivals[i] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids[i] = submit(h, img)

    t0 = time.perf_counter()
    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    kept = {}
    for i, rid in enumerate(ids):
        st, curve = ecc.ecc_poll(h, rid, timeout_us=600_000_000)
        assert st == ecc.ECC_OK
        if i % 16 == 0:
            # a copy: a served curve is a view into a pinned result slab of
            # the library, and a live view keeps the whole slab from reuse
            kept[i] = np.array(curve)
        del curve
    wall = time.perf_counter() - t0
    if ref is not None:
        for i, curve in kept.items():
            if i < len(ref):
                assert _same_curve(curve, ref[i]), f"served curve {i} differs from the batched one"
                checked += 1
    del kept
    lat = np.array([ecc.ecc_request_latency_us(h, rid) for rid in ids]) / 1e3
    # where the time went: submit -> copy seen done -> batch launched -> batch
    # seen done -> curve ready, for the median request and the slowest 1 %
    st = np.array([ecc.ecc_request_trace_us(h, rid) for rid in ids]) / 1e3
    seg = np.diff(np.concatenate([np.zeros((len(st), 1)), st], axis=1), axis=1)
    slow = lat >= np.percentile(lat, 99)
    names = ["copy", "wait_launch", "batch", "complete"]
    vox = sum(int(np.prod(a.shape)) for a, _ in reqs)
    sizes = np.array([int(np.prod(a.shape)) for a, _ in reqs], dtype=np.float64)
    return {"requests": len(reqs), "rate_hz": rate_hz, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "gvox_s": vox / wall / 1e9, "wall_s": wall,
            "curves_checked_against_batched": checked,
            "mean_mvox_all": float(sizes.mean() / 1e6),
            "mean_mvox_slowest_1pct": float(sizes[slow].mean() / 1e6),
            "stages_ms_median": {k: float(np.median(seg[:, i])) for i, k in enumerate(names)},
            "stages_ms_slowest_1pct": {k: float(seg[slow, i].mean()) for i, k in enumerate(names)}}


def config_volume14(steps: int, volume, h2d: dict):
    """14-bit two-phase volume (default 1536 x 3072 x 3072 uint16, 27 GiB,
    16384 bins), the same bytes fully resident in HBM (value: events around
    ecc_compute_device on the device image) and streamed from pinned host
    memory in z-slabs of 64 planes through a 4 GiB device ring (e2e: the
    wall time of begin / push every slab / finish, min and median over the
    repetitions)."""
    import torch
    from paper_1705_02045_gb300 import ecc, synth
    shape = tuple(int(s) for s in volume)
    nvox = int(np.prod(shape))
    host = torch.empty(shape, dtype=torch.int16, pin_memory=True)
    hview = host.numpy().view(np.uint16)
    t0 = time.perf_counter()
    for z0, slab in synth.two_phase_u16_slabs(shape, 6.0, synth.SEED_BASE + 2, 64):
        hview[z0:z0 + slab.shape[0]] = slab
    gen_s = time.perf_counter() - t0
    hu = host.view(torch.uint16)
    # streamed
    h = ecc.ecc_create(device=0, bins=16384, slab_depth=64, ring_bytes=4 << 30)
    times, curve_s = [], None
    for rep in range(steps + 1):
        t0 = time.perf_counter()
        s = ecc.ecc_stream_begin(h, shape, np.uint16)
        for z0 in range(0, shape[0], 64):
            ecc.ecc_stream_push_slab(h, s, hu[z0:z0 + 64], z0)
        curve_s = ecc.ecc_stream_finish(h, s)
        if rep:
            times.append(time.perf_counter() - t0)
    ecc.ecc_destroy(h)
    # resident
    d = hu.cuda()
    torch.cuda.synchronize()
    h = ecc.ecc_create(device=0, bins=16384)
    c = torch.empty(16384, dtype=torch.int64, device="cuda")
    st = torch.cuda.Stream()
    ecc.ecc_compute_device(h, d, 16384, c, stream=st)
    st.synchronize()
    ecc.ecc_set_profiling(h, True)
    ecc.ecc_profile_read(h)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for e0, e1 in evs:
        e0.record(st)
        ecc.ecc_compute_device(h, d, 16384, c, stream=st)
        e1.record(st)
    st.synchronize()
    t_res = float(np.median([e0.elapsed_time(e1) for e0, e1 in evs])) / 1e3
    kms, n = ecc.ecc_profile_read(h)
    assert ecc.ecc_device_status(h) == ecc.ECC_OK
    curve_r = c.cpu().numpy()
    ecc.ecc_destroy(h)
    del d
    torch.cuda.empty_cache()
    same = bool(np.array_equal(curve_s, curve_r))
    assert same and curve_r[-1] == 1
    peak, peak_kind = measured_peak_hbm()
    kernel_s = kms / max(n, 1) / 1e3
    alu_pk = alu_peak_tops(torch.cuda.get_device_properties(0).multi_processor_count, None)
    t_min, t_med = min(times), float(np.median(times))
    base = cpu_baseline(np.ascontiguousarray(hview[:32]), 16384, 10.0,
                        f"the first 32 planes of the same {shape[1]}x{shape[2]} volume")
    del host, hview, hu
    return {
        "workload": f"3D {shape[2]}x{shape[1]}x{shape[0]} uint16 14-bit two-phase field "
                    "sigma=6 (Gaussian random field at its 40th percentile, phases "
                    "N(3000,400) / N(11000,900)), 16384 bins",
        "value": nvox / t_res / 1e9, "unit": "Gvoxel/s", "ms_per_step": t_res * 1e3,
        "steps": steps, "dtype": "u16",
        "timing": "resident: median of CUDA events around ecc_compute_device on the device "
                  "image (input 27 GiB > L2)",
        "roofline": alu_roofline(nvox, alu_ops_per_voxel(14), kernel_s, alu_pk, nvox * 2.0,
                                 peak, peak_kind, "bit-sliced contribution+histogram"),
        "e2e": {"value": nvox / t_min / 1e9, "unit": "Gvoxel/s",
                "median": nvox / t_med / 1e9,
                "h2d_bytes_per_step": nvox * 2, "d2h_bytes_per_step": 16384 * 8,
                "how": "ecc_stream_begin / ecc_stream_push_slab of 64-plane slabs from pinned "
                       "host memory / ecc_stream_finish (4 GiB device ring), wall clock, best "
                       f"of {steps}",
                "h2d_gbs": nvox * 2 / t_min / 1e9,
                "frac_of_h2d_peak": nvox * 2 / t_min / 1e9 / h2d["gbs"],
                "rep_seconds": times},
        "cpu_baseline": base,
        "streamed_equals_resident": same, "generation_s": gen_s}


def workload_f32q(args):
    """A float32 Gaussian random field (sigma = 3 per axis; default the 4D
    128^4 image, --volume for others, e.g. 512,512,512) through the value
    transform into 16384 bins between its min and max (Sec. 3, "Other Ranges
    of Gray Values"), device-resident; the exact float pairs of the same image
    timed beside it."""
    import torch
    from paper_1705_02045_gb300 import ecc, synth
    shape = tuple(int(s) for s in args.volume.split(","))
    nvox = int(np.prod(shape))
    d = synth.grf_f32_torch(shape, 3.0, synth.SEED_BASE + 4).contiguous()
    torch.cuda.synchronize()
    lo, hi, bins = float(d.min()), float(d.max()), 16384
    h = ecc.ecc_create(device=0)
    curve = ecc.ecc_compute_quantized(h, d, lo, hi, bins)
    t, chi = ecc.ecc_compute(h, d)

    def best_of(fn):
        times = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            times.append(time.perf_counter() - t0)
        return min(times)

    tq = best_of(lambda: ecc.ecc_compute_quantized(h, d, lo, hi, bins))
    tx = best_of(lambda: ecc.ecc_compute(h, d))
    ecc.ecc_destroy(h)
    # the transform relation at the top of the range: everything has code <= bins-1
    assert curve[-1] == 1 and chi[-1] == 1
    print(json.dumps({
        "metric": METRIC, "workload": "f32q", "value": nvox / tq / 1e9,
        "unit": "Gvoxel/s", "n_gpus": 1, "steps": args.steps, "dtype": "f32->u16",
        "data": "synthetic",
        "config": {"workload": f"{len(shape)}D {shape} float32 Gaussian random field sigma=3, "
                               f"value transform into {bins} bins over [min, max], "
                               "device-resident, blocking call incl. curve read-back"},
        "seconds": tq, "ms_per_step": tq * 1e3,
        "exact_pairs": {"seconds": tx, "gvox_s": nvox / tx / 1e9, "pairs": int(len(t))},
        "speedup_vs_exact": tx / tq}), flush=True)


def workload_file(args):
    """Out-of-core: the 14-bit two-phase recipe (sigma = 6) written raw to a
    temporary file (default 256 x 3072 x 3072 uint16, 4.8 GB), then streamed
    from the file in 64-plane slabs (reader thread + pinned double buffer +
    device ring). The file was just written, so reads may come from the page
    cache; the line says how much of the file that could be. The curve is
    checked against the same planes pushed from pinned memory."""
    import shutil
    import tempfile
    import torch
    from paper_1705_02045_gb300 import ecc, synth
    shape = tuple(int(s) for s in args.volume.split(","))
    nvox = int(np.prod(shape))
    tmpdir = tempfile.mkdtemp(prefix="ecc_file_")
    try:
        free = shutil.disk_usage(tmpdir).free
        if free < nvox * 2 * 1.2:
            raise RuntimeError(f"not enough space in {tmpdir} for {nvox * 2} bytes")
        path = os.path.join(tmpdir, "vol.raw")
        host = torch.empty(shape, dtype=torch.int16, pin_memory=True)
        hview = host.numpy().view(np.uint16)
        with open(path, "wb") as f:
            for z0, slab in synth.two_phase_u16_slabs(shape, 6.0, synth.SEED_BASE + 2, 64):
                hview[z0:z0 + slab.shape[0]] = slab
                f.write(slab.tobytes())
        h = ecc.ecc_create(device=0, bins=16384, slab_depth=64, ring_bytes=4 << 30)
        times, curve_f = [], None
        for rep in range(args.steps + 1):
            t0 = time.perf_counter()
            curve_f = ecc.ecc_stream_file(h, path, shape, np.uint16)
            if rep:
                times.append(time.perf_counter() - t0)
        s = ecc.ecc_stream_begin(h, shape, np.uint16)
        hu = host.view(torch.uint16)
        for z0 in range(0, shape[0], 64):
            ecc.ecc_stream_push_slab(h, s, hu[z0:z0 + 64], z0)
        curve_p = ecc.ecc_stream_finish(h, s)
        ecc.ecc_destroy(h)
        same = bool(np.array_equal(curve_f, curve_p))
        assert same and curve_f[-1] == 1
        t = min(times)
        mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
        print(json.dumps({
            "metric": METRIC, "workload": "file", "value": nvox / t / 1e9, "unit": "Gvoxel/s",
            "n_gpus": 1, "steps": args.steps, "dtype": "u16", "data": "synthetic",
            "config": {"workload": f"3D {shape} uint16 14-bit two-phase field sigma=6, 16384 "
                                   "bins, raw file, 64-plane slabs, 4 GiB ring"},
            "seconds": t, "file_gbs": nvox * 2 / t / 1e9, "rep_seconds": times,
            "file_bytes": nvox * 2, "host_memory_bytes": mem,
            "page_cache_note": "file written just before; it fits in host memory, so reads "
                               "may be served from the page cache",
            "file_equals_pinned_stream": same}), flush=True)
    finally:
        shutil.rmtree(tmpdir, ignore_errors=True)


def config_plane512(steps: int, warmup: int):
    """2D 512 x 512 uint8, i.i.d. uniform 0..255, 256 bins: one small image
    per call, bound by launch latency. Device time of each call (events
    around it, L2 flushed between calls outside the events), the same call
    replayed from a CUDA graph, and end to end from pinned host memory."""
    import torch
    from paper_1705_02045_gb300 import ecc, synth
    shape = (512, 512)
    nvox = shape[0] * shape[1]
    img = synth.uniform_u8(shape, synth.SEED_BASE + 0)
    d = torch.from_numpy(img).cuda()
    c = torch.empty(256, dtype=torch.int64, device="cuda")
    h = ecc.ecc_create(device=0)
    st = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(warmup, 3)):
        ecc.ecc_compute_device(h, d, 256, c, stream=st)
    st.synchronize()
    ref = c.cpu().numpy().copy()
    assert ref[-1] == 1

    def timed(run):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for a, b in evs:
            with torch.cuda.stream(st):
                flush.zero_()
            a.record(st)
            run()
            b.record(st)
        st.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in evs]))

    launches0 = ecc.ecc_launch_count(h)
    direct_ms = timed(lambda: ecc.ecc_compute_device(h, d, 256, c, stream=st))
    launches = (ecc.ecc_launch_count(h) - launches0) // steps
    # the contribution kernel's own time from a separate, profiled pass
    ecc.ecc_set_profiling(h, True)
    ecc.ecc_profile_read(h)
    timed(lambda: ecc.ecc_compute_device(h, d, 256, c, stream=st))
    kms, n = ecc.ecc_profile_read(h)
    ecc.ecc_set_profiling(h, False)
    c.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        ecc.ecc_compute_device(h, d, 256, c, stream=st)
    graph_ms = timed(g.replay)
    assert np.array_equal(c.cpu().numpy(), ref)
    hp = torch.from_numpy(img).pin_memory()
    for _ in range(3):
        ecc.ecc_compute(h, hp)
    e2e = []
    for _ in range(steps):
        t0 = time.perf_counter()
        curve = ecc.ecc_compute(h, hp)
        e2e.append(time.perf_counter() - t0)
    assert np.array_equal(curve, ref)
    ecc.ecc_destroy(h)
    e2e_s = float(np.median(e2e))
    kernel_s = kms / max(n, 1) / 1e3
    peak, peak_kind = measured_peak_hbm()
    alg = nvox + 256 * 8
    return {
        "workload": "2D 512x512 uint8 i.i.d. uniform 0..255, 256 bins, one image per call, "
                    "device-resident",
        "value": nvox / (direct_ms * 1e-3) / 1e9, "unit": "Gvoxel/s",
        "ms_per_step": direct_ms, "steps": steps, "dtype": "u8",
        "timing": "median of CUDA events around each ecc_compute_device call; 256 MiB write "
                  "between calls, outside the events",
        "us_per_call": direct_ms * 1e3, "graph_us_per_call": graph_ms * 1e3,
        "graph_gvox_s": nvox / (graph_ms * 1e-3) / 1e9, "launches_per_call": int(launches),
        "roofline": {"bound": "hbm", "achieved": alg / kernel_s / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": alg / kernel_s / 1e9 / peak, "traffic": None,
                     "kernel": "bit-sliced contribution+histogram+fused scan",
                     "kernel_ms": kernel_s * 1e3, "peak_kind": peak_kind,
                     "note": "launch-latency bound: 256 KiB read by one launch of a few "
                             "microseconds"},
        "e2e": {"value": nvox / e2e_s / 1e9, "unit": "Gvoxel/s", "us_per_call": e2e_s * 1e6,
                "h2d_bytes_per_step": nvox, "d2h_bytes_per_step": 256 * 8},
        "cpu_baseline": cpu_baseline(img, 256, 3.0, "the same 512^2 image")}


def config_grf4d(steps: int, volume):
    """4D 128^4 float32 Gaussian random field (sigma = 3 per axis): (key,
    change) pairs, radix sort, reduce-by-key and scan into exact (threshold,
    chi) pairs. value: the blocking ecc_compute on the device-resident image
    (pairs copied to the host), median over the steps; e2e: the same from
    pinned host memory."""
    import torch
    from paper_1705_02045_gb300 import ecc, synth
    shape = tuple(int(s) for s in volume)
    nvox = int(np.prod(shape))
    d = synth.grf_f32_torch(shape, 3.0, synth.SEED_BASE + 4).contiguous()
    torch.cuda.synchronize()
    h = ecc.ecc_create(device=0)
    t, chi = ecc.ecc_compute(h, d)
    ecc.ecc_set_profiling(h, True)
    ecc.ecc_profile_read(h)
    times = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t, chi = ecc.ecc_compute(h, d)
        times.append(time.perf_counter() - t0)
    kms, n = ecc.ecc_profile_read(h)
    ecc.ecc_set_profiling(h, False)
    hp = d.cpu().pin_memory()
    ecc.ecc_compute(h, hp)
    e2e = []
    for _ in range(steps):
        t0 = time.perf_counter()
        t2, chi2 = ecc.ecc_compute(h, hp)
        e2e.append(time.perf_counter() - t0)
    ecc.ecc_destroy(h)
    assert chi[-1] == 1 and np.all(np.diff(t) > 0)
    assert np.array_equal(t, t2) and np.array_equal(chi, chi2)
    med, e2e_med = float(np.median(times)), float(np.median(e2e))
    kernel_s = kms / max(n, 1) / 1e3
    peak, peak_kind = measured_peak_hbm()
    alu_pk = alu_peak_tops(torch.cuda.get_device_properties(0).multi_processor_count, None)
    base = cpu_baseline(hp[:16].numpy().copy(), 0, 10.0,
                        f"the first 16 volumes of the same {shape} field")
    del d, hp
    torch.cuda.empty_cache()
    return {
        "workload": f"4D {'x'.join(map(str, shape))} float32 Gaussian random field sigma=3, "
                    "exact (threshold, chi) pairs, device-resident",
        "value": nvox / med / 1e9, "unit": "Gvoxel/s", "ms_per_step": med * 1e3,
        "steps": steps, "dtype": "f32", "pairs": int(len(t)),
        "timing": "median wall time of the blocking ecc_compute on the device image "
                  "(contribution kernel, radix sort, reduce-by-key, scan, pairs to the host); "
                  "input 1 GiB > L2",
        "roofline": alu_roofline(nvox, 40.0, kernel_s, alu_pk, nvox * 4.0, peak, peak_kind,
                                 "4D contribution kernel emitting (key, change) pairs"),
        "e2e": {"value": nvox / e2e_med / 1e9, "unit": "Gvoxel/s",
                "h2d_bytes_per_step": nvox * 4, "d2h_bytes_per_step": int(len(t)) * 12},
        "cpu_baseline": base}


def profile_case(args):
    """A few launches of the integer path on one image, nothing else: the
    small, self-ending case for ncu captures."""
    import torch
    from paper_1705_02045_gb300 import ecc, synth
    shape = tuple(int(s) for s in args.profile_shape.split(","))
    if args.profile_dtype == "u8":
        img, bins = synth.smooth_u8(shape, SIGMA, synth.SEED_BASE + 1), 256
    else:
        img, bins = synth.two_phase_u16(shape, 6.0, synth.SEED_BASE + 2), 16384
    h = ecc.ecc_create(device=0)
    d = torch.from_numpy(img).cuda()
    c = torch.empty(bins, dtype=torch.int64, device="cuda")
    for _ in range(args.profile_launches):
        ecc.ecc_compute_device(h, d, bins, c)
    torch.cuda.synchronize()
    assert ecc.ecc_device_status(h) == ecc.ECC_OK and int(c[-1]) == 1
    ecc.ecc_destroy(h)
    print("profile case ok", shape, args.profile_dtype)


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle, timed on this host, rank 0 only."""
    if rank != 0:
        return
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import oracle
    img = make_image()
    budget = 150.0
    n_steps = args.steps + args.warmup
    procs = max(1, os.cpu_count() or 1)
    t0 = time.perf_counter()
    oracle.vcec_int_zrange(img, BINS, 0, 1, "V")
    one = max(time.perf_counter() - t0, 1e-3)
    # each step: one task of k planes per host core, about budget / steps
    # seconds per step (at least one plane per task)
    per_step = max(0.05, budget / max(n_steps, 1))
    k = int(max(1, min(SHAPE[0] // procs or 1, per_step / one)))
    shm = shared_memory.SharedMemory(create=True, size=img.nbytes)
    try:
        np.ndarray(img.shape, dtype=img.dtype, buffer=shm.buf)[...] = img

        def tasks(step):
            base = step * procs * k
            return [(shm.name, img.shape, img.dtype.str, BINS, (base + i * k) % SHAPE[0],
                     (base + i * k) % SHAPE[0] + k) for i in range(procs)]

        with mp.get_context("spawn").Pool(procs) as pool:
            for i in range(args.warmup):
                pool.map(_oracle_planes, tasks(i), chunksize=1)
            t0 = time.perf_counter()
            planes = 0
            for i in range(args.steps):
                planes += sum(pool.map(_oracle_planes, tasks(i), chunksize=1))
            dt = time.perf_counter() - t0
    finally:
        shm.close()
        shm.unlink()
    vox = planes * SHAPE[1] * SHAPE[2]
    value = vox / dt / 1e9
    line = {"metric": METRIC, "value": value, "unit": "Gvoxel/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / max(args.steps, 1) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD + f"; each step = cells of {procs} x {k} plane(s)",
                       "parallelism": f"{procs} host processes"},
            "cpu_baseline": {"value": value, "unit": "Gvoxel/s", "cores": procs, "kind": "oracle",
                             "sample": f"{procs} processes x {k} planes of 512x512 per step"},
            "e2e": {"value": value, "unit": "Gvoxel/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--batch-images", type=int, default=4096,
                    help="images of the mixed request stream in the batched comparison")
    ap.add_argument("--serve-requests", type=int, default=4096,
                    help="requests of the served Poisson stream (0 = skip)")
    ap.add_argument("--no-configs", action="store_true",
                    help="headline only: skip the 2D, 14-bit volume and 4D float workloads")
    ap.add_argument("--config-steps", type=int, default=5,
                    help="repetitions of each workload in configs")
    ap.add_argument("--profile-launches", type=int, default=0,
                    help="only run this many ecc_compute_device launches (for ncu) and exit")
    ap.add_argument("--profile-shape", default="640,512,512")
    ap.add_argument("--profile-dtype", default="u8", choices=["u8", "u16"])
    ap.add_argument("--workload", default="resident512",
                    choices=["resident512", "stream", "f32_4d", "plane512", "f32q", "file"],
                    help="resident512: the full line (headline and every workload); the "
                         "others print one line each: stream (14-bit volume resident and from "
                         "pinned memory), file (the same recipe from a raw file), f32_4d "
                         "(exact float pairs), f32q (value transform), plane512 (2D 512^2)")
    ap.add_argument("--volume", default=None, help="shape for --workload stream / f32_4d")
    args = ap.parse_args()
    world, rank, local = _dist()
    if args.profile_launches > 0:
        profile_case(args)
        return
    if args.workload in ("plane512", "stream", "f32_4d"):
        if args.workload == "plane512":
            res = config_plane512(args.steps, args.warmup)
        elif args.workload == "stream":
            res = config_volume14(max(1, min(args.steps, 5)),
                                  (args.volume or "1536,3072,3072").split(","), h2d_peak())
        else:
            res = config_grf4d(max(1, min(args.steps, 20)),
                               (args.volume or "128,128,128,128").split(","))
        print(json.dumps({"metric": METRIC, "workload_key": args.workload, "n_gpus": 1,
                          "higher_is_better": True, "data": "synthetic", **res}), flush=True)
        return
    if args.workload != "resident512":
        args.steps = max(1, min(args.steps, 5))
    if args.workload == "file":
        args.volume = args.volume or "256,3072,3072"
        workload_file(args)
        return
    if args.workload == "f32q":
        args.volume = args.volume or "128,128,128,128"
        workload_f32q(args)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    from paper_1705_02045_gb300 import ecc

    if args.warmup < 3:
        args.warmup = 3
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ecc.load()
    h = ecc.ecc_create(device=local)

    img = make_image(1 + rank)
    nvox = img.size
    d_img = torch.from_numpy(img).cuda()
    d_curve = torch.empty(BINS, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()

    # correctness guard on this very input: top of the curve is 1 (box contractible)
    ecc.ecc_compute_device(h, d_img, BINS, d_curve, stream=stream)
    stream.synchronize()
    assert int(d_curve[-1].item()) == 1

    for _ in range(args.warmup):
        ecc.ecc_compute_device(h, d_img, BINS, d_curve, stream=stream)
    stream.synchronize()

    ecc.ecc_set_profiling(h, True)
    ecc.ecc_profile_read(h)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches0 = ecc.ecc_launch_count(h)
    _barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t_wall0 = time.perf_counter()
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                starts[i].record(stream)
            ecc.ecc_compute_device(h, d_img, BINS, d_curve, stream=stream)
            ends[i].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        if t_wall < 1.5:
            time.sleep(0.0)
    _barrier(world)
    launches = ecc.ecc_launch_count(h) - launches0
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps
    contrib_ms, n_rec = ecc.ecc_profile_read(h)
    contrib_ms /= max(n_rec, 1)
    ecc.ecc_set_profiling(h, False)
    value, step_ms_max = aggregate(nvox, step_ms, world)

    # roofline of the dominant kernel (the contribution kernel)
    peak, peak_kind = measured_peak_hbm()
    alg_bytes = nvox * 1 + BINS * 8
    achieved = alg_bytes / (contrib_ms * 1e-3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = json.load(open(tfile)).get("contrib_512cube_u8")
        except Exception:
            traffic = None

    # end to end through the public API with a pinned host image
    h_img = torch.from_numpy(img).pin_memory()
    for _ in range(2):
        ecc.ecc_compute(h, h_img)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        curve = ecc.ecc_compute(h, h_img)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    assert curve[-1] == 1
    e2e_s = _max_over_ranks(e2e_s, world)
    e2e_value = world * nvox / e2e_s / 1e9

    if rank == 0:
        cs = clocks.summary()
        num_sms = torch.cuda.get_device_properties(local).multi_processor_count
        alu_peak = alu_peak_tops(num_sms, cs.get("sm_max_mhz"))
        alu_achieved = nvox * alu_ops_per_voxel(8) / (contrib_ms * 1e-3) / 1e12
        line = {
            "metric": METRIC, "value": value, "unit": "Gvoxel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "images": world, "voxels_per_gpu": nvox,
                       "bins": BINS, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "256 MiB write between steps, outside the timed events"},
            "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak,
                         "unit": "Tops/s", "frac": alu_achieved / alu_peak, "traffic": traffic,
                         "kernel": "contribution+histogram", "kernel_ms": contrib_ms,
                         "ops_per_voxel": alu_ops_per_voxel(8),
                         "peak_kind": f"derived: {num_sms} SMs x {ALU_LANES_PER_SM_CLK} "
                                      "logic lanes/clock x max SM clock",
                         "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                                 "frac": achieved / peak, "peak_kind": peak_kind}},
            "e2e": {"value": e2e_value, "unit": "Gvoxel/s", "h2d_bytes_per_step": nvox,
                    "d2h_bytes_per_step": BINS * 8},
            "gpu_launches": int(launches),
            "clocks": cs,
        }
        if args.batch_images > 0 or args.serve_requests > 0:
            from paper_1705_02045_gb300 import synth
            n_req = max(args.batch_images, args.serve_requests)
            reqs = make_requests(n_req, synth.SEED_BASE + 3)
            hb = ecc.ecc_create(device=local)
            try:
                if args.batch_images > 0:
                    line["batched"] = bench_batched(hb, reqs[:args.batch_images], stream)
            finally:
                ecc.ecc_destroy(hb)
            if args.serve_requests > 0:
                sreqs = [(torch.from_numpy(a).pin_memory(), b) for a, b in reqs[:args.serve_requests]]
                # served curves are checked against the batched ones of the same images
                ref = getattr(bench_batched, "curves", None)
                def serve_pair(borrowed):
                    # saturated, then Poisson arrivals at 0.8x its throughput
                    hs = ecc.ecc_create(device=local)
                    try:
                        sat = bench_serving(hs, sreqs, 0.0, synth.SEED_BASE + 4, borrowed, ref)
                    finally:
                        ecc.ecc_destroy(hs)
                    rate = 0.8 * len(sreqs) / sat["wall_s"]
                    hs = ecc.ecc_create(device=local)
                    try:
                        pois = bench_serving(hs, sreqs, rate, synth.SEED_BASE + 5, borrowed, ref)
                    finally:
                        ecc.ecc_destroy(hs)
                    return {"poisson_0.8x": pois, "saturated": sat}

                line["serving"] = dict(serve_pair(False),
                                       borrowed=serve_pair(True),
                                       workload="mixed 2D/3D uint8 / 14-bit uint16 requests in "
                                                "pinned host memory, smoothed fields sigma=2 "
                                                "(synth.request_mix); borrowed: "
                                                "ecc_submit_borrowed; each measurement after "
                                                "one untimed pass of the same requests on "
                                                "the same handle")
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(img)
        if not args.no_configs:
            # the other configured workloads, each with its own value, roofline,
            # e2e and CPU baseline (the oracle on a bounded sample)
            del d_img, flush
            torch.cuda.empty_cache()
            line["h2d_peak"] = h2d_peak()
            cs = args.config_steps
            line["configs"] = {
                "plane512_u8": config_plane512(max(cs, 20), args.warmup),
                "volume14_u16": config_volume14(max(1, min(cs, 5)), (1536, 3072, 3072),
                                                line["h2d_peak"]),
                "grf4d_f32": config_grf4d(max(1, cs), (128, 128, 128, 128)),
            }
            # one byte per voxel crosses the host link
            line["e2e"]["frac_of_h2d_peak"] = e2e_value / world / line["h2d_peak"]["gbs"]
        print(json.dumps(line), flush=True)
    ecc.ecc_destroy(h)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
