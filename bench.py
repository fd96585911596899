"""Benchmark: pack + unpack of the six halo faces of a 512^3 float64 grid.

One step = pack the six send faces (a struct of six subarray types, one
kernel launch) into one contiguous 24 MiB buffer, then unpack that buffer
into the same six faces of a second 512^3 grid (one batched launch of six
per-face operations: the faces share edge cells, so together they are an
overlapping receive layout, while each face alone is not).  Metric:
algorithmic bytes (read + written user bytes, 2 * packed bytes per pack and
per unpack) per second.  L2 is flushed between timed steps (a 512 MiB write
and a 512 MiB read outside the timed events), since the touched bytes would
otherwise fit in the 126 MB L2.

After the timed steps the same line carries the rest of the metric under
"secondary": the large-block pack gate (fraction of the HBM roofline), the
10^4-op batch against per-call launches, and the serving loop's p50/p99
latency and its speedup over per-call launches (--no-secondary skips them).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dte|reference]

--impl reference times the CPU oracle (the plain typemap walker) on the same
workload (a bounded sample of steps) and prints the same JSON line with
"impl": "reference".  Under torchrun each rank runs the workload on its own
GPU (independent replicas, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N = 512
G = 2
ALG_FACTOR = 2  # read + write per moved byte
METRIC = "pack+unpack GB/s (algorithmic bytes, % of HBM roofline)"
WORKLOAD = "512^3 float64 grid, six halo faces (ghost 2): pack all six into one buffer, unpack into a second grid"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="dte", choices=["dte", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="keep the fixed kernel rule (no plan tuning)")
    p.add_argument("--no-secondary", action="store_true",
                   help="skip the rest of the metric (large-block gate, batch vs per-call, serving loop)")
    p.add_argument("--config", default="halo",
                   help="halo (headline, default) | vector | records | batch | largeblock | autograd | serve | "
                        "pipeline | faces | fastaxis | all")
    p.add_argument("--records-blocks", type=int, default=1 << 22)
    p.add_argument("--batch-ops", type=int, default=10000)
    p.add_argument("--serve-requests", type=int, default=20000)
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(src: str) -> str:
    """C/C++/CUDA source with comments removed and whitespace runs collapsed
    (string and character literals kept verbatim), so that the kernel-source
    hash changes with the code and not with its comments."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


# Sources the data-movement kernels are built from (the request loop's own
# file, server.cu, builds none of the kernels the traffic records describe).
KERNEL_SOURCES = ("bulk.cuh", "desc.h", "internal.h", "kernels.cu", "move.cuh", "typesys.cpp")


def csrc_hash():
    """Hash of the data-movement kernels' sources (code only), recorded
    beside committed ncu figures so that they are used only while those
    kernels are unchanged."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2402_12274_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(d, name), encoding="utf-8") as f:
            h.update(name.encode())
            h.update(_code_only(f.read()).encode())
    return h.hexdigest()[:16]


def traffic_from_profile(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except OSError:
        return None
    ent = rec.get(kernel)
    if not ent or ent.get("csrc_hash") != csrc_hash():
        return None
    return ent.get("dram_bytes_per_launch")


def sector_floor(faces, grid_bytes: int, packed_bytes: int):
    """DRAM bytes the six-face step cannot avoid at 32-byte sector
    granularity, from the faces' segment lists (every run here is a multiple
    of 16 bytes at a 16-byte boundary): pack reads every user sector a run
    touches (union over the faces, which share edge cells) and writes the
    packed bytes; unpack reads the packed bytes, writes every touched sector
    and first reads back (fills) each sector it writes only in part.
    Returns {"pack": bytes, "unpack": bytes, "touched_sectors", "partial_sectors"}."""
    import paper_2402_12274_gb300 as dte
    units = grid_bytes // 16
    diff = np.zeros(units + 1, np.int32)
    for f in faces:
        lst = np.array(dte.dte_type_iov(f.h, 0, f.num_segments), dtype=np.int64).reshape(-1, 2)
        np.add.at(diff, lst[:, 0] // 16, 1)
        np.add.at(diff, (lst[:, 0] + lst[:, 1]) // 16, -1)
    cov = (np.cumsum(diff[:-1]) > 0).reshape(-1, 2).sum(axis=1)
    touched = int(np.count_nonzero(cov))
    partial = int(np.count_nonzero(cov == 1))
    return {"pack": 32 * touched + packed_bytes, "unpack": packed_bytes + 32 * touched + 32 * partial,
            "touched_sectors": touched, "partial_sectors": partial}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.windows = []
        self.adjacent = False

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def open(self, adjacent: bool = False):
        self.adjacent = self.adjacent or adjacent
        self.windows.append([time.time(), None])

    def close(self):
        self.windows[-1][1] = time.time()

    @staticmethod
    def _ts(s):
        try:
            from datetime import datetime
            return datetime.strptime(s.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def _in_window(self, t):
        return t is not None and any(a <= t <= (b or 1e300) for a, b in self.windows)

    def count_in_window(self):
        time.sleep(0.1)  # let the reader catch up
        return sum(1 for ln in list(self.lines) if self._in_window(self._ts(ln.split(",")[0])))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in list(self.lines):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9 or not self._in_window(self._ts(parts[0])):
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        window = "adjacent soak of the same step" if self.adjacent else "timed region"
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0, "window": window}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm), "window": window}


class L2Flush:
    """Evict the step's data from L2 between timed steps: write a 512 MiB
    buffer (larger than the 126 MB L2), then read another 512 MiB so the lines
    left in L2 are clean -- the next timed kernel then pays neither for hits
    on its own data nor for writing back the flush's dirty lines."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
        self.r = torch.ones(128 << 20, dtype=torch.float32, device=dev)
        self.out = torch.empty((), dtype=torch.float32, device=dev)

    def zero_(self):
        import torch
        self.w.zero_()
        torch.sum(self.r, dim=0, out=self.out)


def max_over_ranks(seconds: float, world: int, dev=None) -> float:
    """The slowest rank's time (every rank gets it); a no-op on one rank.
    Ranks are independent replicas, so this is the only collective."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_throughput(bytes_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job GB/s: every rank moved bytes_per_rank in at most `seconds`."""
    return bytes_per_rank * world / seconds / 1e9


L2_NOTE = ("GPU arm: L2 flushed between timed steps outside the timed events (512 MiB write, then "
           "512 MiB read); CPU arm: no cache control")


def bench_config(packed_bytes: int, world: int) -> dict:
    """The workload description both arms print (identical dicts)."""
    return {"workload": WORKLOAD, "packed_bytes": int(packed_bytes),
            "alg_bytes_per_step": int(2 * ALG_FACTOR * packed_bytes), "l2": L2_NOTE,
            "parallelism": f"replicas x{world}"}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# CPU oracle leg (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_steps(seconds_budget: float, max_steps: int | None = None, warmup: int = 0):
    """Time the oracle on the same pack+unpack step after `warmup` untimed
    steps; stops after max_steps steps or once the budget is spent.
    Returns (GB/s, steps, secs)."""
    import oracle
    import inputs
    faces = [oracle.from_spec(f) for f in inputs.halo_face_specs(N, G)]
    send = oracle.from_spec(inputs.all_faces_struct(inputs.halo_face_specs(N, G)))
    grid = np.zeros(N ** 3, np.float64)
    grid[:] = inputs.normal_f64(N ** 3, 2)
    g2 = np.zeros_like(grid)
    size = send.size

    def one_step():
        pk = send.pack(grid.view(np.uint8), 1)
        pos = 0
        for f in faces:
            f.unpack(pk[pos:pos + f.size], 1, g2.view(np.uint8))
            pos += f.size

    for _ in range(warmup):
        one_step()
    steps, t0 = 0, time.perf_counter()
    while True:
        one_step()
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps and steps >= max_steps) or (seconds_budget and el >= seconds_budget):
            break
    alg = 2 * ALG_FACTOR * size * steps
    return alg / el / 1e9, steps, el, size


def run_reference(args):
    """The oracle timed on the host cores as the reference arm: W untimed
    steps, then exactly K timed steps, each one full pack+unpack of the
    headline workload (about 40 ms of single-thread CPU work per step)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    gbs, steps, el, size = oracle_steps(0.0, max_steps=max(1, args.steps), warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbs, 4), "unit": "GB/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": bench_config(size, world),
        "cpu_baseline": {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{steps} full pack+unpack steps after {args.warmup} untimed, single thread"},
        "e2e": {"value": round(gbs, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def run_dte(args):
    import torch
    import torch.distributed as dist

    import paper_2402_12274_gb300 as dte
    import inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    send = dte.Datatype.from_spec(inputs.all_faces_struct(inputs.halo_face_specs(N, G))).commit()
    faces = [dte.Datatype.from_spec(f).commit() for f in inputs.halo_face_specs(N, G)]
    size = send.size
    fsz = [f.size for f in faces]
    offs = np.concatenate([[0], np.cumsum(fsz)[:-1]]).tolist()
    gen = torch.Generator(device=dev)
    gen.manual_seed(2)
    grid = torch.randn(N ** 3, dtype=torch.float64, device=dev, generator=gen)
    grid2 = torch.zeros_like(grid)
    packed = torch.empty(size, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    flush = L2Flush(dev)

    # the six faces share edge cells, so they are unpacked as one batch of six
    # per-face operations (one launch); shared cells receive identical bytes
    batches = {}

    def unpack_all(dst):
        b = batches.get(dst)
        if b is None:
            b = batches[dst] = dte.Batch(dte.BATCH_UNPACK, [(f.h, 1, dst, packed.data_ptr() + o)
                                                              for f, o in zip(faces, offs)])
        b.enqueue(sh)

    def step():
        dte.dte_pack_enqueue(grid.data_ptr(), 1, send.h, packed.data_ptr(), size, 0, sh)
        unpack_all(grid2.data_ptr())

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            step()
            flush.zero_()
    stream.synchronize()

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.15)  # sampler running before the window opens
        clk.open()
        with torch.cuda.stream(stream):
            for i in range(K):
                flush.zero_()
                ev[i][0].record(stream)
                dte.dte_pack_enqueue(grid.data_ptr(), 1, send.h, packed.data_ptr(), size, 0, sh)
                ev[i][1].record(stream)
                unpack_all(grid2.data_ptr())
                ev[i][2].record(stream)
        stream.synchronize()
        clk.close()
        if clk.count_in_window() < 3:
            # window too short for nvidia-smi: sample an identical soak right after
            clk.open(adjacent=True)
            t_end = time.time() + 0.6
            with torch.cuda.stream(stream):
                while time.time() < t_end:
                    for _ in range(50):
                        flush.zero_()
                        step()
                    stream.synchronize()
            clk.close()
    torch.cuda.synchronize()
    t_pack = np.array([ev[i][0].elapsed_time(ev[i][1]) for i in range(K)]) * 1e-3
    t_unpack = np.array([ev[i][1].elapsed_time(ev[i][2]) for i in range(K)]) * 1e-3
    total = max_over_ranks(float((t_pack + t_unpack).sum()), world, dev)
    alg_step = 2 * ALG_FACTOR * size
    value = job_throughput(alg_step * K, world, total)

    # e2e: the same step through the C ABI on pinned host grids (the kernels
    # read and write host memory over NVLink-C2C; no staging copies)
    e2e = None
    if not args.no_e2e:
        h_grid = torch.empty(N ** 3, dtype=torch.float64, pin_memory=True)
        h_grid.copy_(grid.cpu())
        h_grid2 = torch.zeros(N ** 3, dtype=torch.float64, pin_memory=True)

        def step_host():
            dte.dte_pack_enqueue(h_grid.data_ptr(), 1, send.h, packed.data_ptr(), size, 0, sh)
            unpack_all(h_grid2.data_ptr())

        with torch.cuda.stream(stream):
            for _ in range(3):
                step_host()
        stream.synchronize()
        # timed like the device steps: the L2 flushed before every step,
        # outside the step's events, and the step times summed
        ke = max(5, min(K, 20))
        eev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(ke)]
        with torch.cuda.stream(stream):
            for i in range(ke):
                flush.zero_()
                eev[i][0].record(stream)
                step_host()
                eev[i][1].record(stream)
        stream.synchronize()
        te = max_over_ranks(sum(a.elapsed_time(b) for a, b in eev) * 1e-3, world, dev)
        e2e = {"value": round(job_throughput(alg_step * ke, world, te), 3), "unit": "GB/s",
               "h2d_bytes_per_step": size, "d2h_bytes_per_step": size,
               "mode": "pinned host grids accessed by the kernels (zero-copy over NVLink-C2C)",
               "l2": "flushed before every step, outside the step's events"}

    # correctness spot check (not timed): the second grid holds the faces
    g3, h3 = grid.view(N, N, N), grid2.view(N, N, N)
    ok = bool(torch.equal(h3[G:2 * G], g3[G:2 * G]) and torch.equal(h3[:, N - 2 * G:N - G], g3[:, N - 2 * G:N - G])
              and torch.equal(h3[:, :, G:2 * G], g3[:, :, G:2 * G]))

    peak, peak_kind = peaks()
    mp, mu = float(t_pack.mean()), float(t_unpack.mean())
    dom = "pack" if mp >= mu else "unpack"
    # one launch each: the struct pack and the six-op unpack batch move `size` bytes
    tdom = max(mp, mu)
    per_launch = size
    achieved = ALG_FACTOR * per_launch / tdom / 1e9
    kname = "dte::move_kernel<16, 1, 1, 0>" if dom == "pack" else "dte::batch_kernel<16, 0, 1, 0>"
    # the layout's own floor: DRAM bytes at 32-byte sector granularity (the
    # 16-byte runs of the fastest-axis faces cost a whole sector each, and an
    # unpack fills every sector it writes in part)
    floor = sector_floor(faces, N ** 3 * 8, size)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic_from_profile(kname),
            "kernel": kname, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "pack_ms": round(mp * 1e3, 4), "unpack_ms": round(mu * 1e3, 4),
            "alg_bytes_per_launch": ALG_FACTOR * per_launch,
            "floor_bytes": floor[dom], "frac_of_floor": round(floor[dom] / tdom / 1e9 / peak, 4),
            "floor_bytes_pack": floor["pack"], "floor_bytes_unpack": floor["unpack"],
            "frac_of_floor_pack": round(floor["pack"] / mp / 1e9 / peak, 4),
            "frac_of_floor_unpack": round(floor["unpack"] / mu / 1e9 / peak, 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        gbs, st, el, _ = oracle_steps(12.0)
        cpu = {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"{st} full pack+unpack steps of the same workload, {el:.1f} s, single thread"}

    # the rest of the metric, measured after the timed region: the large-block
    # pack gate, batched ops/s against per-call launches, and the serving
    # loop's latency and its speedup over per-call launches (one GPU only)
    secondary = None
    if rank == 0 and world == 1 and not args.no_secondary:
        secondary = {}
        if not args.no_tune:
            # kernel plans per shape for this workload, measured against the
            # fixed rule the timed steps above used: the six-face pack is one
            # single move, the unpack batch holds three shapes (faces with
            # 4 MiB, 8 KiB and 16-byte runs); the types go back to the rule
            from paper_2402_12274_gb300 import autotune
            pk_ops = [(send.h, 1, grid.data_ptr(), packed.data_ptr())]
            up_ops = [(f.h, 1, grid2.data_ptr(), packed.data_ptr() + o) for f, o in zip(faces, offs)]
            with torch.cuda.stream(stream):
                secondary["halo_plans"] = {
                    "pack": autotune.tune_plans(dte.BATCH_PACK, pk_ops, stream=stream, reps=60, flush=flush.zero_,
                                                single=True, use_cache=False),
                    "unpack_batch": autotune.tune_plans(dte.BATCH_UNPACK, up_ops, stream=stream, reps=60,
                                                        flush=flush.zero_, use_cache=False)}
            autotune.reset_plans(pk_ops + up_ops)
        del flush
        torch.cuda.empty_cache()
        for key, fn in (("largeblock_gate", lambda: largeblock_measure()),
                        ("batch", lambda: batch_measure(args.batch_ops, graphs=False)),
                        ("serving", lambda: serve_measure(args.serve_requests))):
            t0 = time.perf_counter()
            try:
                secondary[key] = fn()
            except Exception as exc:  # recorded, the headline line still prints
                secondary[key] = {"error": f"{type(exc).__name__}: {exc}"}
            secondary[key]["wall_s"] = round(time.perf_counter() - t0, 1)
            torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": K,
            "warmup": max(args.warmup, 3), "ms_per_step": round(1e3 * total / K, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": bench_config(size, world),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * K,
            "clocks": clk.summary(), "check": "ok" if ok else "MISMATCH",
            "secondary": secondary,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Secondary workloads (one JSON line each; not the headline)
# ---------------------------------------------------------------------------
def _mean_s(stream, fn, reps, flush=None):
    import torch
    ev = []
    with torch.cuda.stream(stream):
        for _ in range(3):
            fn()
        for _ in range(reps):
            if flush is not None:
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ev.append((a, b))
    stream.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev])) * 1e-3


def _line(name, metric, value, unit, extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic", "config": {"workload": name}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_config_vector(args):
    """vector(1024,4,16) float32, count 64 (1 MiB packed out of a 4 MB span),
    rotating over 64 buffer pairs (256 MB > L2) so every launch reads HBM.
    A 1 MiB op is short enough that the host's enqueue cost shows, so three
    figures are reported: one call at a time through the Python binding
    (host + GPU), back-to-back enqueues on one stream (GPU time per op while
    the host keeps up), and the same ops replayed from a captured CUDA graph.
    Plus the full 65,536-segment list on the device."""
    import ctypes
    import torch
    import paper_2402_12274_gb300 as dte
    import inputs
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream()
    sh = s.cuda_stream
    t = dte.Datatype.from_spec(inputs.strided_vector_spec()).commit()
    count, span = 64, 63 * t.extent + t.true_extent
    R = 64
    srcs = [torch.from_numpy(inputs.uniform_f32(span // 4, 1 + i)).to(dev) for i in range(R)]
    pks = [torch.empty(count * t.size, dtype=torch.uint8, device=dev) for _ in range(R)]
    iov = torch.empty((count * 1024, 2), dtype=torch.int64, device=dev)
    it = [0]
    pos = ctypes.c_int64(0)

    def pack(stream=sh):
        i = it[0] = (it[0] + 1) % R
        pos.value = 0
        dte.lib.dte_pack_enqueue(srcs[i].data_ptr(), count, t.h, pks[i].data_ptr(), pks[i].numel(), ctypes.byref(pos),
                                 stream)

    def unpack(stream=sh):
        i = it[0] = (it[0] + 1) % R
        pos.value = 0
        dte.lib.dte_unpack_enqueue(pks[i].data_ptr(), pks[i].numel(), ctypes.byref(pos), srcs[i].data_ptr(), count,
                                   t.h, stream)

    def iovq():
        dte.dte_type_iov_async(t.h, count, 0, iov.data_ptr(), count * 1024, 0, 0, sh)

    tp, tu, ti = _mean_s(s, pack, 400), _mean_s(s, unpack, 400), _mean_s(s, iovq, 400)

    def back_to_back(fn, n=400):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            # hold the GPU (~50 ms) while the host queues all n calls (~15 us each)
            torch.cuda._sleep(100_000_000)
            e0.record(s)
            for _ in range(n):
                fn()
            e1.record(s)
        s.synchronize()
        return e0.elapsed_time(e1) * 1e-3 / n

    bp, bu = back_to_back(pack), back_to_back(unpack)

    def graph_of(fn):
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream()
        with torch.cuda.graph(g, stream=gs):
            for _ in range(R):
                fn(gs.cuda_stream)
        return g

    gp, gu = graph_of(pack), graph_of(unpack)
    tgp, tgu = _mean_s(s, gp.replay, 20) / R, _mean_s(s, gu.replay, 20) / R
    peak, _ = peaks()
    z = count * t.size
    _line("vector(1024,4,16) float32 x64 (1 MiB packed), 64 rotating buffers", "pack+unpack GB/s",
          round(4 * z / (bp + bu) / 1e9, 1), "GB/s",
          {"timing": "back-to-back enqueues on one stream (GPU time per op)",
           "back_to_back": {"pack_us": round(bp * 1e6, 2), "unpack_us": round(bu * 1e6, 2)},
           "graph_replay": {"pack_us": round(tgp * 1e6, 2), "unpack_us": round(tgu * 1e6, 2),
                            "GBs": round(4 * z / (tgp + tgu) / 1e9, 1)},
           "one_call_at_a_time": {"pack_us": round(tp * 1e6, 2), "unpack_us": round(tu * 1e6, 2),
                                  "GBs": round(4 * z / (tp + tu) / 1e9, 1)},
           "iov_segments_per_s": round(count * 1024 / ti), "iov_us": round(ti * 1e6, 2),
           "hbm_peak_GBs": peak})


def run_config_records(args):
    """struct{int32[3],float64[5]} resized to 64 B inside an indexed type of
    2^22 geometric blocks: pack/unpack GB/s, device iov chunk lookups from
    random byte offsets (4096 segments each), the full sequential segment
    list on the device, host query latency."""
    import torch
    import paper_2402_12274_gb300 as dte
    import inputs
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream()
    nb = args.records_blocks
    rng = np.random.default_rng(3)
    t = dte.Datatype.from_spec(inputs.record_indexed_spec(rng, nb)).commit()
    span = t.true_lb + t.true_extent
    src = torch.empty(span, dtype=torch.uint8, device=dev)
    src.random_(0, 256)
    pk = torch.empty(t.size, dtype=torch.uint8, device=dev)
    tp = _mean_s(s, lambda: dte.dte_pack_enqueue(src.data_ptr(), 1, t.h, pk.data_ptr(), pk.numel(), 0, s.cuda_stream), 10)
    tu = _mean_s(s, lambda: dte.dte_unpack_enqueue(pk.data_ptr(), pk.numel(), 0, src.data_ptr(), 1, t.h, s.cuda_stream), 10)
    nq, m = 4096, 4096
    offs = torch.from_numpy(rng.integers(0, t.size, nq).astype(np.int64)).to(dev)
    iov = torch.empty((nq * m, 2), dtype=torch.int64, device=dev)
    first = torch.empty(nq, dtype=torch.int64, device=dev)
    act = torch.empty(nq, dtype=torch.int64, device=dev)
    tq = _mean_s(s, lambda: dte.dte_type_iov_at_bytes_async(t.h, nq, offs.data_ptr(), m, iov.data_ptr(), first.data_ptr(),
                                                           act.data_ptr(), 0, s.cuda_stream), 10)
    # the full sequential segment list (16 B written per segment)
    nseg = t.num_segments
    full = torch.empty((nseg, 2), dtype=torch.int64, device=dev)
    tl = _mean_s(s, lambda: dte.dte_type_iov_async(t.h, 1, 0, full.data_ptr(), nseg, 0, 0, s.cuda_stream), 5)
    del full
    # host queries (the paper's synchronous API): iov_len(B) then iov(k, 4096)
    import ctypes
    buf = (dte.dte_iov * m)()
    k, nbytes, got = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    lat = []
    for b in rng.integers(0, t.size, 2000):
        t0 = time.perf_counter()
        dte.lib.dte_type_iov_len(t.h, int(b), ctypes.byref(k), ctypes.byref(nbytes))
        dte.lib.dte_type_iov(t.h, k.value, buf, m, ctypes.byref(got))
        lat.append(time.perf_counter() - t0)
    peak, _ = peaks()
    _line(f"record layout, {nb} indexed blocks ({t.size} B packed)", "pack+unpack GB/s",
          round(4 * t.size / (tp + tu) / 1e9, 1), "GB/s",
          {"pack_GBs": round(2 * t.size / tp / 1e9, 1), "unpack_GBs": round(2 * t.size / tu / 1e9, 1),
           "descriptor_bytes": t.descriptor_bytes, "iov_device_queries_per_s": round(nq / tq),
           "iov_device_batch_us": round(tq * 1e6, 1), "iov_full_list_segments": nseg,
           "iov_full_list_ms": round(tl * 1e3, 3), "iov_full_list_GBs_written": round(16 * nseg / tl / 1e9, 1),
           "iov_host_query_p50_us": round(float(np.percentile(lat, 50)) * 1e6, 1),
           "iov_host_query_p99_us": round(float(np.percentile(lat, 99)) * 1e6, 1), "hbm_peak_GBs": peak})


def batch_measure(nops: int, graphs: bool = True):
    """10^4 independent packs (vector/indexed/subarray of float32 or bf16,
    64 B - 4 MiB, seed 4): per-call launches vs one autotuned batch, each
    optionally also replayed from a captured CUDA graph.  Inputs total several
    GB (no L2 flush needed)."""
    import torch
    import paper_2402_12274_gb300 as dte
    from paper_2402_12274_gb300 import autotune
    import inputs
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream()
    rng = np.random.default_rng(4)
    specs = inputs.batch_specs(rng, nops)
    types = [dte.Datatype.from_spec(sp).commit() for sp, _ in specs]
    spans = [t.true_lb + t.true_extent for t in types]
    sizes = [t.size for t in types]
    up = lambda v: (v + 255) // 256 * 256  # noqa: E731
    so = np.concatenate([[0], np.cumsum([up(v) for v in spans])])
    po = np.concatenate([[0], np.cumsum([up(v) for v in sizes])])
    src = torch.empty(int(so[-1]), dtype=torch.uint8, device=dev)
    src.random_(0, 256)
    pk = torch.zeros(int(po[-1]), dtype=torch.uint8, device=dev)
    ops = [(t.h, 1, src.data_ptr() + int(a), pk.data_ptr() + int(b)) for t, a, b in zip(types, so, po)]
    total = int(sum(sizes))
    sh = s.cuda_stream

    def per_call():
        for t, a, b, z in zip(types, so, po, sizes):
            dte.dte_pack_enqueue(src.data_ptr() + int(a), 1, t.h, pk.data_ptr() + int(b), z, 0, sh)

    # the fixed kernel rule, then plans picked per shape group, in one run
    auto = dte.Batch(dte.BATCH_PACK, ops)
    t_auto = _mean_s(s, lambda: auto.enqueue(s), 10)
    auto.free()
    plans = autotune.tune_plans(dte.BATCH_PACK, ops, stream=s, reps=3, use_cache=False)
    batch = dte.Batch(dte.BATCH_PACK, ops)
    t_plans = _mean_s(s, lambda: batch.enqueue(s), 10)
    shapes = [(16, z) for z in sizes]
    best, _, table = autotune.tune(batch, dte.BATCH_PACK, shapes, stream=s, reps=3, use_cache=False)
    t_batch = _mean_s(s, lambda: batch.enqueue(s), 10)
    pk_b = pk.clone()
    pk.zero_()
    t_call = _mean_s(s, per_call, 3)
    same = bool(torch.equal(pk, pk_b))
    del pk_b
    out = {"ops": nops, "packed_bytes": total, "ops_per_s": round(nops / t_batch),
           "batch_GBs": round(2 * total / t_batch / 1e9, 1), "batch_ms": round(t_batch * 1e3, 3),
           "per_call_ops_per_s": round(nops / t_call), "per_call_ms": round(t_call * 1e3, 3),
           "speedup_batch_vs_per_call": round(t_call / t_batch, 2),
           "fixed_rule_batch_ms": round(t_auto * 1e3, 3), "tuned_plans_batch_ms": round(t_plans * 1e3, 3),
           "plan_groups_changed": {k: v for k, v in plans.items()
                                   if not k.startswith("_") and v["pick"] not in ("auto", v["auto"])},
           "plan_groups": sum(not k.startswith("_") for k in plans), "plan_totals_ms": plans.get("_total_ms"),
           "autotuned_launch": {"blocks_per_sm": best[0], "span_tiles": best[1]},
           "autotune_table_ms": {f"{b}x{sp}": round(v * 1e3, 3) for (b, sp), v in (table or {}).items()},
           "bit_identical_batch_vs_per_call": same}
    if graphs:
        def graph_of(fn):
            g = torch.cuda.CUDAGraph()
            gs = torch.cuda.Stream()
            with torch.cuda.graph(g, stream=gs):
                fn(gs)
            return g

        g_batch = graph_of(lambda gs: batch.enqueue(gs))
        g_call = graph_of(lambda gs: [dte.dte_pack_enqueue(src.data_ptr() + int(a), 1, t.h, pk.data_ptr() + int(b),
                                                           z, 0, gs.cuda_stream)
                                      for t, a, b, z in zip(types, so, po, sizes)])
        t_gb = _mean_s(s, g_batch.replay, 10)
        t_gc = _mean_s(s, g_call.replay, 3)
        out.update({"graph_batch_ms": round(t_gb * 1e3, 3), "graph_per_call_ms": round(t_gc * 1e3, 3),
                    "speedup_graph_batch_vs_graph_per_call": round(t_gc / t_gb, 2)})
    batch.free()
    return out


def run_config_batch(args):
    r = batch_measure(args.batch_ops)
    peak, _ = peaks()
    _line(f"{args.batch_ops} independent packs, 64 B-4 MiB (vector/indexed/subarray, f32/bf16), "
          f"{r['packed_bytes']} B packed", "batched pack ops/s", r["ops_per_s"], "ops/s", dict(hbm_peak_GBs=peak, **r))


def largeblock_measure(runs=(1024, 4096, 16384, 65536, 262144, 1 << 20), reps: int = 30):
    """Large-block pack/unpack: hvector of runs of 1 KiB - 1 MiB with gaps of
    half a run, 256 MiB packed (the HBM-roofline gate), L2 flushed between
    reps, with torch's own device copy of 256 MiB beside it."""
    import torch
    import paper_2402_12274_gb300 as dte
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream()
    fl = L2Flush(dev)
    dst = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    src = torch.empty((256 << 20) * 3 // 2 + (1 << 20), dtype=torch.uint8, device=dev)
    res = {}
    for L in runs:
        n = (256 << 20) // L
        t = dte.Datatype.hvector(n, 1, L + L // 2, dte.Datatype.contiguous(L // 8, dte.FLOAT64)).commit()
        tp = _mean_s(s, lambda: dte.dte_pack_enqueue(src.data_ptr(), 1, t.h, dst.data_ptr(), dst.numel(), 0,
                                                     s.cuda_stream), reps, fl)
        tu = _mean_s(s, lambda: dte.dte_unpack_enqueue(dst.data_ptr(), dst.numel(), 0, src.data_ptr(), 1, t.h,
                                                       s.cuda_stream), reps, fl)
        res[str(L)] = {"pack_GBs": round(2 * t.size / tp / 1e9, 1), "unpack_GBs": round(2 * t.size / tu / 1e9, 1)}
    tc = _mean_s(s, lambda: dst.copy_(src[: 256 << 20]), reps, fl)
    peak, kind = peaks()
    wp = min(v["pack_GBs"] for v in res.values())
    wu = min(v["unpack_GBs"] for v in res.values())
    del fl, dst, src
    return {"min_pack_GBs": wp, "min_unpack_GBs": wu, "pack_frac_of_peak": round(wp / peak, 4),
            "unpack_frac_of_peak": round(wu / peak, 4), "gate": 0.75,
            "gate_met": bool(wp / peak >= 0.75), "peak": peak, "peak_source": kind, "runs": res,
            "torch_copy_GBs": round(2 * (256 << 20) / tc / 1e9, 1),
            "l2": "flushed between reps (write + read 512 MiB)"}


def run_config_largeblock(args):
    r = largeblock_measure()
    _line("large-block hvector sweep, runs 1 KiB-1 MiB, 256 MiB packed", "large-block pack GB/s (min over runs)",
          r["min_pack_GBs"], "GB/s", r)


def run_config_autograd(args):
    """Differentiable pack of six halo faces of a 256^3 float32 field as
    element-granular indexed types with 10% repeated entries: forward pack
    and adjoint (deterministic segmented sum) times."""
    import torch
    import paper_2402_12274_gb300 as dte
    import inputs
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream()
    rng = np.random.default_rng(5)
    n = 256
    t = dte.Datatype.from_spec(inputs.all_faces_struct(inputs.halo_indexed_specs(rng, n, 2, 0.10))).commit()
    x = torch.randn(n ** 3, dtype=torch.float32, device=dev)
    y = torch.empty(t.size // 4, dtype=torch.float32, device=dev)
    gx = torch.zeros_like(x)
    fl = L2Flush(dev)
    tf = _mean_s(s, lambda: dte.dte_pack_enqueue(x.data_ptr(), 1, t.h, y.data_ptr(), t.size, 0, s.cuda_stream), 50, fl)
    tb = _mean_s(s, lambda: dte.dte_pack_adjoint_f32_enqueue(y.data_ptr(), 1, t.h, gx.data_ptr(), s.cuda_stream), 50, fl)
    _line("six halo faces of 256^3 float32, indexed entries, 10% repeated", "forward+backward us",
          round((tf + tb) * 1e6, 1), "us", {"higher_is_better": False, "forward_us": round(tf * 1e6, 1),
                                            "backward_us": round(tb * 1e6, 1), "entries": t.size // 4})


def serve_measure(nreq: int, rhos=(0.5, 0.8, 0.95), seed: int = 5, ctas_per_sm: int = 4, span_tiles: int = 4):
    """Request loop under Poisson arrivals: pack/unpack requests (50/50) of
    layouts from the batch generator with sizes log-uniform 1 KiB - 64 MiB,
    admission cap 8 GiB.  The service rate mu is measured first (all requests
    submitted at once); then arrivals at rho*mu for each rho, latency = host
    arrival time to observed completion.  Beside it, the same requests as
    per-call enqueues on one stream (dte_pack_enqueue / dte_unpack_enqueue,
    wall time from the first enqueue to the stream's completion) and as two
    plain batches (one pack, one unpack)."""
    import torch
    import paper_2402_12274_gb300 as dte
    import inputs
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(seed)
    pool = []
    for spec, _ in inputs.batch_specs(rng, 160, lo=1 << 10, hi=64 << 20):
        t = dte.Datatype.from_spec(spec).commit()
        span = t.true_lb + t.true_extent
        u = torch.empty(span, dtype=torch.uint8, device=dev)
        u.random_(0, 256)
        p = torch.empty(t.size, dtype=torch.uint8, device=dev)
        p.random_(0, 256)
        pool.append((t, u, p))
    torch.cuda.synchronize()
    picks = rng.integers(0, len(pool), nreq)
    kinds = rng.integers(0, 2, nreq)
    nbytes = np.array([2 * pool[i][0].size for i in picks], dtype=np.float64)
    srv = dte.dte_server_create(ring_slots=1024, max_inflight_bytes=8 << 30, ctas_per_sm=ctas_per_sm,
                                span_tiles=span_tiles)

    def submit(i):
        t, u, p = pool[picks[i]]
        return dte.dte_server_submit(srv, int(kinds[i]), t.h, 1, u.data_ptr(), p.data_ptr())

    # warm up and measure the service rate (everything offered at once)
    for i in range(min(50, nreq)):
        dte.dte_server_wait(srv, submit(i), 60_000_000)
    t0 = time.perf_counter()
    tks = [submit(i) for i in range(nreq)]
    t_sub = time.perf_counter() - t0
    for tk in tks:
        dte.dte_server_wait(srv, tk, 600_000_000)
    t_all = time.perf_counter() - t0
    mu = nreq / t_all
    res = {}
    for rho in rhos:
        gaps = rng.exponential(1.0 / (rho * mu), nreq)
        arrive = np.cumsum(gaps)
        lat = np.zeros(nreq)
        outstanding = []
        start = time.perf_counter()
        i = 0
        while i < nreq or outstanding:
            now = time.perf_counter() - start
            while i < nreq and arrive[i] <= now:
                outstanding.append((submit(i), i, start + arrive[i]))
                i += 1
            dte.dte_server_progress(srv)
            keep = []
            for tk, j, ta in outstanding:
                if dte.dte_server_test(srv, tk):
                    lat[j] = time.perf_counter() - ta
                else:
                    keep.append((tk, j, ta))
            outstanding = keep
        wall = time.perf_counter() - start
        res[str(rho)] = {"p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                         "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                         "throughput_GBs": round(float(nbytes.sum()) / wall / 1e9, 1),
                         "offered_req_per_s": round(rho * mu, 1)}
    dte.dte_server_free(srv)
    # the same requests launched one by one on one stream
    s = torch.cuda.Stream()
    sh = s.cuda_stream

    def per_call():
        for i in range(nreq):
            t, u, p = pool[picks[i]]
            if kinds[i] == dte.BATCH_PACK:
                dte.dte_pack_enqueue(u.data_ptr(), 1, t.h, p.data_ptr(), t.size, 0, sh)
            else:
                dte.dte_unpack_enqueue(p.data_ptr(), t.size, 0, u.data_ptr(), 1, t.h, sh)

    per_call()
    s.synchronize()
    t0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    per_call()
    e1.record(s)
    s.synchronize()
    t_call = time.perf_counter() - t0
    t_call_gpu = e0.elapsed_time(e1) * 1e-3
    # and as two plain batches
    ops = {k: [(pool[picks[i]][0].h, 1, pool[picks[i]][1].data_ptr(), pool[picks[i]][2].data_ptr())
               for i in range(nreq) if kinds[i] == k] for k in (dte.BATCH_PACK, dte.BATCH_UNPACK)}
    bs = [dte.Batch(k, v) for k, v in ops.items() if v]
    t_b = _mean_s(s, lambda: [b.enqueue(s) for b in bs], 5)
    for b in bs:
        b.free()
    total = float(nbytes.sum())
    return {"service_rate_req_per_s": round(mu, 1), "host_submit_us_per_request": round(t_sub / nreq * 1e6, 2),
            "service_GBs": round(total / t_all / 1e9, 1), "by_load": res,
            "per_call": {"wall_ms": round(t_call * 1e3, 2), "gpu_ms": round(t_call_gpu * 1e3, 2),
                         "GBs": round(total / t_call / 1e9, 1)},
            "speedup_served_vs_per_call": round(t_call / t_all, 2),
            "two_batches": {"ms": round(t_b * 1e3, 2), "GBs": round(total / t_b / 1e9, 1)},
            "requests": nreq, "mean_request_bytes_moved": round(float(nbytes.mean()))}


def run_config_serve(args):
    r = serve_measure(args.serve_requests)
    _line(f"request loop, {args.serve_requests} Poisson-arriving pack/unpack requests of 1 KiB-64 MiB, 8 GiB cap",
          "p99 latency at rho=0.8 (ms)", r["by_load"]["0.8"]["p99_ms"], "ms", dict(higher_is_better=False, **r))


def run_config_pipeline(args):
    """Windowed send-to-self pipeline (pack -> device copy -> unpack per
    window, one stream): a periodic halo exchange of the 512^3 float64 grid
    (each of the six 4 MiB send faces into the opposite ghost face) and a
    256 MiB large-block hvector message, at several staging sizes."""
    import torch
    import paper_2402_12274_gb300 as dte
    import inputs
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream()
    fl = L2Flush(dev)
    n = 512
    a = torch.empty(n ** 3, dtype=torch.float64, device=dev)
    b = torch.empty(n ** 3, dtype=torch.float64, device=dev)
    send = [dte.Datatype.from_spec(x).commit() for x in inputs.halo_face_specs(n, 2)]
    recv = [dte.Datatype.from_spec(x).commit() for x in inputs.halo_recv_face_specs(n, 2)]
    msg = sum(t.size for t in send)
    halo = {}
    for st in (256 << 10, 1 << 20, 4 << 20, 16 << 20):
        g = torch.empty(st, dtype=torch.uint8, device=dev)

        def step():
            for f in range(6):
                dte.dte_sendrecv_enqueue(a.data_ptr(), 1, send[f].h, b.data_ptr(), 1, recv[f ^ 1].h,
                                         g.data_ptr(), st, s.cuda_stream)
        ts = _mean_s(s, step, 50, fl)
        halo[f"staging_{st >> 10}KiB"] = {"us": round(ts * 1e6, 1), "message_GBs": round(msg / ts / 1e9, 1),
                                          "hbm_GBs": round(6 * msg / ts / 1e9, 1)}
    big = {}
    L = 65536
    t = dte.Datatype.hvector((256 << 20) // L, 1, L + L // 2, dte.Datatype.contiguous(L // 8, dte.FLOAT64)).commit()
    src = torch.empty((256 << 20) * 3 // 2 + (1 << 20), dtype=torch.uint8, device=dev)
    dst = torch.empty_like(src)
    for st in (8 << 20, 64 << 20, 512 << 20):
        g = torch.empty(st, dtype=torch.uint8, device=dev)
        ts = _mean_s(s, lambda: dte.dte_sendrecv_enqueue(src.data_ptr(), 1, t.h, dst.data_ptr(), 1, t.h,
                                                         g.data_ptr(), st, s.cuda_stream), 20, fl)
        big[f"staging_{st >> 20}MiB"] = {"ms": round(ts * 1e3, 3), "message_GBs": round(t.size / ts / 1e9, 1),
                                         "hbm_GBs": round(6 * t.size / ts / 1e9, 1)}
    peak, kind = peaks()
    best = max(v["hbm_GBs"] for v in big.values())
    _line("send-to-self pipeline: 512^3 f64 periodic halo faces; 256 MiB hvector(64 KiB runs)",
          "pipeline HBM GB/s (large-block, best staging)", best, "GB/s",
          {"frac_of_peak": round(best / peak, 4), "peak": peak, "peak_source": kind,
           "halo_faces": halo, "large_block": big, "halo_message_bytes": msg,
           "bytes_model": "6 x message (pack r+w, copy r+w, unpack r+w)",
           "l2": "flushed between reps (write + read 512 MiB)"})


def run_config_faces(args):
    """Breakdown of the headline halo step: each of the six faces of the
    512^3 float64 grid packed and unpacked alone, the same face moved by a
    torch strided copy, and the unpack batch split into the faces with long
    runs and the two faces normal to the fastest axis (16-byte runs)."""
    import torch
    import paper_2402_12274_gb300 as dte
    import inputs
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream()
    fl = L2Flush(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2)
    grid = torch.randn(N ** 3, dtype=torch.float64, device=dev, generator=gen)
    grid2 = torch.zeros_like(grid)
    specs = inputs.halo_face_specs(N, G)
    faces = [dte.Datatype.from_spec(f).commit() for f in specs]
    g3, h3 = grid.view(N, N, N), grid2.view(N, N, N)
    R = 100
    res = {}
    for i, (f, sp) in enumerate(zip(faces, specs)):
        pk = torch.empty(f.size, dtype=torch.uint8, device=dev)
        sl = tuple(slice(int(a), int(a + b)) for a, b in zip(sp[3], sp[2]))
        pv = pk.view(torch.float64).view(tuple(int(x) for x in sp[2]))
        tp = _mean_s(s, lambda: dte.dte_pack_enqueue(grid.data_ptr(), 1, f.h, pk.data_ptr(), f.size, 0,
                                                     s.cuda_stream), R, fl)
        tu = _mean_s(s, lambda: dte.dte_unpack_enqueue(pk.data_ptr(), f.size, 0, grid2.data_ptr(), 1, f.h,
                                                       s.cuda_stream), R, fl)
        ttp = _mean_s(s, lambda: pv.copy_(g3[sl]), R, fl)
        ttu = _mean_s(s, lambda: h3[sl].copy_(pv), R, fl)
        res[f"face{i}_axis{i // 2}"] = {"pack_us": round(tp * 1e6, 2), "unpack_us": round(tu * 1e6, 2),
                                        "torch_copy_in_us": round(ttp * 1e6, 2),
                                        "torch_copy_out_us": round(ttu * 1e6, 2)}
    offs = np.concatenate([[0], np.cumsum([f.size for f in faces])[:-1]]).tolist()
    packed = torch.empty(sum(f.size for f in faces), dtype=torch.uint8, device=dev)
    send = dte.Datatype.from_spec(inputs.all_faces_struct(specs)).commit()
    t_pack = _mean_s(s, lambda: dte.dte_pack_enqueue(grid.data_ptr(), 1, send.h, packed.data_ptr(), send.size, 0,
                                                     s.cuda_stream), R, fl)
    parts = {}
    for name, idx in (("all_six", range(6)), ("axes_0_1", [0, 1, 2, 3]), ("axis_2", [4, 5])):
        b = dte.Batch(dte.BATCH_UNPACK, [(faces[j].h, 1, grid2.data_ptr(), packed.data_ptr() + offs[j]) for j in idx])
        parts[name] = round(_mean_s(s, lambda: b.enqueue(s.cuda_stream), R, fl) * 1e6, 2)
    a = torch.empty(24 << 20, dtype=torch.uint8, device=dev)
    b2 = torch.empty_like(a)
    t_copy = _mean_s(s, lambda: b2.copy_(a), R, fl)
    _line("512^3 float64 halo faces, one at a time (axis 2 = fastest; its faces have 16-byte runs)",
          "six-face struct pack us", round(t_pack * 1e6, 2), "us",
          {"higher_is_better": False, "faces": res, "unpack_batch_us": parts,
           "torch_copy_24MiB_us": round(t_copy * 1e6, 2),
           "note": "means of 100 CUDA-event timings (8.192 us event resolution), L2 flushed before each"})


def run_config_fastaxis(args):
    """The two halo faces normal to the fastest axis of the 512^3 float64
    grid (2 x 262,144 runs of 16 bytes at a 4 KiB stride): their struct pack
    (one move_kernel launch) and their unpack as a two-op batch (one
    batch_kernel launch), eight of each, L2 flushed before every launch; the
    sector floor of each beside the times."""
    import torch
    import paper_2402_12274_gb300 as dte
    import inputs
    dev = torch.device("cuda", 0)
    s = torch.cuda.Stream()
    fl = L2Flush(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2)
    grid = torch.randn(N ** 3, dtype=torch.float64, device=dev, generator=gen)
    grid2 = torch.zeros_like(grid)
    specs = inputs.halo_face_specs(N, G)[4:6]
    faces = [dte.Datatype.from_spec(f).commit() for f in specs]
    send = dte.Datatype.from_spec(inputs.all_faces_struct(specs)).commit()
    packed = torch.empty(send.size, dtype=torch.uint8, device=dev)
    b2 = dte.Batch(dte.BATCH_UNPACK, [(faces[0].h, 1, grid2.data_ptr(), packed.data_ptr()),
                                      (faces[1].h, 1, grid2.data_ptr(), packed.data_ptr() + faces[0].size)])
    ev = []
    with torch.cuda.stream(s):
        for _ in range(8):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            fl.zero_()
            e[0].record(s)
            dte.dte_pack_enqueue(grid.data_ptr(), 1, send.h, packed.data_ptr(), send.size, 0, s.cuda_stream)
            e[1].record(s)
            fl.zero_()
            e[2].record(s)
            b2.enqueue(s.cuda_stream)
            e[3].record(s)
            ev.append(e)
    s.synchronize()
    tp = float(np.mean([e[0].elapsed_time(e[1]) for e in ev[3:]])) * 1e-3
    tu = float(np.mean([e[2].elapsed_time(e[3]) for e in ev[3:]])) * 1e-3
    floor = sector_floor(faces, N ** 3 * 8, send.size)
    peak, _ = peaks()
    _line("512^3 float64 halo faces normal to the fastest axis (16-byte runs at a 4 KiB stride)",
          "two-face pack+unpack us", round((tp + tu) * 1e6, 2), "us",
          {"higher_is_better": False, "pack_us": round(tp * 1e6, 2), "unpack_us": round(tu * 1e6, 2),
           "floor_bytes": {"pack": floor["pack"], "unpack": floor["unpack"]},
           "frac_of_floor": {"pack": round(floor["pack"] / tp / 1e9 / peak, 4),
                             "unpack": round(floor["unpack"] / tu / 1e9 / peak, 4)}})


CONFIGS = {"vector": run_config_vector, "records": run_config_records, "batch": run_config_batch,
           "largeblock": run_config_largeblock, "autograd": run_config_autograd, "serve": run_config_serve,
           "pipeline": run_config_pipeline, "faces": run_config_faces, "fastaxis": run_config_fastaxis}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config != "halo":
        import torch
        torch.cuda.set_device(0)
        for name in (CONFIGS if args.config == "all" else args.config.split(",")):
            CONFIGS[name](args)
    else:
        run_dte(args)


if __name__ == "__main__":
    main()
