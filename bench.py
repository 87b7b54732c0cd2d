"""Benchmark: GSamples/s written to HBM by the generate kernels, with the
roofline of the dominant kernel, an end-to-end figure through the host-
delivery call, the oracle on the host cores, and clocks seen meanwhile.

Workload (full device): MWC, xor128 and KISS at 2^22 streams x 1024 outputs
per stream per call, uint32 and FP32, state carried on the device from call
to call.  One step = one call of each (kind, format) pair: 6 launches,
6 x 2^32 samples, 96 GiB written.  Each call's 16 GiB output is far larger
than L2, so no flush is needed between calls.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "GSamples/s (uint32/FP32 to HBM) and % of HBM-write/INT32 roofline; batched vs plain"
UNIT = "GSamples/s"
KINDS = (0, 1, 2)
FMTS = (0, 1)
KNAME = {0: "mwc", 1: "xor128", 2: "kiss"}
FNAME = {0: "u32", 1: "f32"}
STATE_WORDS = {0: 2, 1: 4, 2: 4}
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n-streams", type=int, default=1 << 22)
    p.add_argument("--n-per-stream", type=int, default=1024)
    p.add_argument("--seed", type=int, default=42)
    p.add_argument("--e2e-steps", type=int, default=5)
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the other workloads (batched, serving, other configs)")
    p.add_argument("--workload", default="full",
                   choices=["full", "batched", "serving", "inline", "paper", "battery"])
    p.add_argument("--rate", type=float, default=20_000.0, help="serving: arrivals/s")
    p.add_argument("--duration", type=float, default=10.0, help="serving: seconds")
    p.add_argument("--verify-every", type=int, default=100, help="serving: check every k-th")
    p.add_argument("--serve-chunk-rows", type=int, default=1024,
                   help="serving: most rows per client per tick")
    p.add_argument("--tick-gib", type=float, default=8.0,
                   help="serving: target output per tick, shared by busy clients")
    p.add_argument("--sat-tick-gib", type=float, default=32.0,
                   help="serving, saturating run: target output per tick (throughput)")
    p.add_argument("--budget-gib", type=float, default=40.0,
                   help="serving: HBM budget (state plus outputs)")
    p.add_argument("--saturating-only", action="store_true",
                   help="serving: only the saturating run (no real-time run, no check pass)")
    p.add_argument("--instances", type=int, default=10_000)
    p.add_argument("--wave-gib", type=float, default=24.0)
    p.add_argument("--tune", action="store_true", help="autotune launch shapes first")
    p.add_argument("--lanes", type=int, default=2,
                   help="batched: groups of instances whose waves overlap")
    p.add_argument("--no-verify", action="store_true", help="batched: skip the check pass")
    p.add_argument("--chunk-rows", type=int, default=1024,
                   help="batched: rows per piece (0 = whole instances)")
    return p.parse_args()


def alg_bytes(kind: int, n: int, steps: int) -> int:
    """Bytes one launch must move: the outputs, the state read and written
    back, and the multipliers read (MWC, KISS)."""
    w = STATE_WORDS[kind]
    return 4 * n * steps + 2 * 4 * w * n + (4 * n if kind != 1 else 0)


def peaks():
    f = ROOT / "MEASURED_PEAKS.json"
    if f.exists():
        d = json.loads(f.read_text())
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("include/gbrng_device.cuh", "paper_1101_1846_gb300/csrc/gen_body.cuh",
                  "paper_1101_1846_gb300/csrc/gen_kernels.cuh",
                  "paper_1101_1846_gb300/csrc/generate.cu", "paper_1101_1846_gb300/csrc/gbrng.cuh")


def _code_only(text: str) -> str:
    """Source text without // comments, trailing blanks and empty lines, so
    that editing a comment does not look like a change of the kernels."""
    lines = []
    for line in text.splitlines():
        line = line.split("//", 1)[0].rstrip()
        if line:
            lines.append(line)
    return "\n".join(lines)


def kernel_source_hash(read=None) -> str:
    """Hash of the code (comments aside) of the files the generate kernels
    are compiled from."""
    read = read or (lambda name: (ROOT / name).read_text())
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(_code_only(read(name)).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    f = ROOT / "profiles" / "dram_traffic.json"
    if not f.exists():
        return None
    d = json.loads(f.read_text())
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    rec = d.get("kernels", {}).get(kernel, {})
    if rec.get("workload") != workload:
        return None
    return rec.get("dram_bytes_per_launch")


def recorded_pipes(kernel: str):
    """Per-pipe utilisation (% of peak) of a generate kernel from the
    committed ncu record, if it was taken on the current kernel source."""
    f = ROOT / "profiles" / "int_pipes.json"
    if not f.exists():
        return None
    d = json.loads(f.read_text())
    if d.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return d.get("kernels", {}).get(kernel)


# ----------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "50"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        busy = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_selector(torch) -> str | None:
    try:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        u = str(getattr(props, "uuid", "") or "")
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return None


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo; on Arm the
    implementer and part codes when no name is given)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        info = Path("/proc/cpuinfo").read_text()
    except OSError:
        return "unknown"
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = (x.strip() for x in line.split(":", 1))
            fields.setdefault(k, v)
    if "model name" in fields:
        return fields["model name"]
    return f"implementer {fields.get('CPU implementer', '?')} part {fields.get('CPU part', '?')}"


def gpu_pci_dir(torch, dev: int) -> Path | None:
    p = torch.cuda.get_device_properties(dev)
    d = Path(f"/sys/bus/pci/devices/{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:"
             f"{p.pci_device_id:02x}.0")
    return d if d.exists() else None


def _cpulist(text: str) -> set[int]:
    cpus = set()
    for part in text.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def gpu_local_cpus(torch, dev: int) -> tuple[int | None, set[int]]:
    """The GPU's NUMA node and the CPUs near it (from sysfs), intersected
    with the CPUs this process may run on."""
    d = gpu_pci_dir(torch, dev)
    node, cpus = None, set()
    if d is not None:
        try:
            node = int((d / "numa_node").read_text())
            cpus = _cpulist((d / "local_cpulist").read_text())
        except (OSError, ValueError):
            pass
    if node is not None and node >= 0 and not cpus:
        try:
            cpus = _cpulist(Path(f"/sys/devices/system/node/node{node}/cpulist").read_text())
        except OSError:
            pass
    return node, cpus & os.sched_getaffinity(0)


def numa_pages(addr: int) -> dict[str, int]:
    """Pages per NUMA node of the mapping that holds `addr`
    (/proc/self/numa_maps)."""
    best, fields = -1, ""
    try:
        for line in Path("/proc/self/numa_maps").read_text().splitlines():
            start, rest = line.split(" ", 1)
            a = int(start, 16)
            if best < a <= addr:
                best, fields = a, rest
    except (OSError, ValueError):
        return {}
    out = {}
    for tok in fields.split():
        if tok.startswith("N") and "=" in tok:
            k, v = tok.split("=", 1)
            if k[1:].isdigit():
                out[k] = int(v)
    return out


def pinned_near_gpu(torch, shape, dev: int):
    """A pinned host tensor allocated while this thread runs on the CPUs
    near the GPU, so that first touch places its pages on the GPU's own
    node; returns the tensor and where its pages are."""
    node, cpus = gpu_local_cpus(torch, dev)
    old = os.sched_getaffinity(0)
    placed = False
    try:
        if cpus and cpus != old:
            os.sched_setaffinity(0, cpus)
            placed = True
        # cudaHostAlloc pins (and so first-touches) every page in this thread
        host = torch.empty(shape, dtype=torch.int32, pin_memory=True)
    finally:
        if placed:
            os.sched_setaffinity(0, old)
    info = {"gpu_numa_node": node, "near_cpus": len(cpus), "allocated_on_near_cpus": placed,
            "buffer_pages_by_node": numa_pages(host.data_ptr())}
    return host, info


# ---------------------------------------------------------------- oracle
def _oracle_worker(args):
    kind, fmt, m, steps, seed, a = args
    import numpy as np

    import oracle
    st = oracle.seed_streams(kind, a if kind != 1 else None, seed, np.arange(m))
    t0 = time.perf_counter()
    oracle.generate(kind, a if kind != 1 else None, st, steps, fmt)
    return m * steps, time.perf_counter() - t0


def cpu_baseline(steps_per_stream: int, streams_per_job: int = 1 << 13, seed: int = 42):
    """The oracle as it stands, one single-threaded process per host core,
    each on its own slice (streams_per_job streams x steps_per_stream) of
    every (kind, format) pair of the workload.  Returns GSamples/s over the
    wall time of the parallel region."""
    import numpy as np

    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    a = oracle.multipliers(streams_per_job, 32)
    jobs = [(k, f, streams_per_job, steps_per_stream, seed + r * streams_per_job, a)
            for r in range(cores) for k in KINDS for f in FMTS]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_worker, [(0, 0, 64, 4, 1, a[:64])] * cores)  # warm the workers
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t0
    samples = sum(r[0] for r in res)
    cpu_s = sum(r[1] for r in res)
    return {"value": samples / wall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x 6 (kind, fmt) slices of {streams_per_job} streams "
                      f"x {steps_per_stream} outputs ({samples / 1e6:.0f} M samples, "
                      f"{cpu_s:.1f} CPU-s, {wall:.1f} s wall)",
            "samples": samples, "wall_s": wall, "np_version": np.__version__}


def cpu_single_thread(samples_per_pair: int = 1 << 26, seed: int = 42):
    """The oracle on one host core: a slice of samples_per_pair samples
    (2^16 streams x 1024 outputs) of every (kind, format) pair, as the
    paper's single-thread CPU rows (Table IV).  Runs in a spawned process so
    that the parent's CUDA context is not shared."""
    steps = 1024
    m = samples_per_pair // steps
    ctx = mp.get_context("spawn")
    import oracle
    oracle.build()
    a = oracle.multipliers(m, 32)
    with ctx.Pool(1) as pool:
        res = pool.map(_oracle_worker, [(k, f, m, steps, seed, a) for k in KINDS for f in FMTS],
                       chunksize=1)
    pairs = {f"{KNAME[k]}_{FNAME[f]}": r[0] / r[1] / 1e9
             for (k, f), r in zip([(k, f) for k in KINDS for f in FMTS], res)}
    return {"unit": UNIT, "cores": 1, "sample": f"{m} streams x {steps} outputs per "
            "(kind, fmt) pair", "gsamples_s": pairs,
            "paper_q6600_single_thread_gsamples_s": {"mwc": 0.3, "xorshift": 0.1, "kiss": 0.2}}


# ------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps_per_stream = min(args.n_per_stream, 256)
    vals = []
    cb = None
    for _ in range(args.warmup):
        cpu_baseline(steps_per_stream, 1 << 11)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cb = cpu_baseline(steps_per_stream, 1 << 11)
        vals.append(cb["samples"] / cb["wall_s"])
    total = time.perf_counter() - t0
    value = statistics.median(vals) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"full_2^22x{args.n_per_stream}",
                   "note": "each step a bounded slice of the same workload on the host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"],
                         "kind": "oracle", "sample": cb["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ ours
def run_ours(args):
    import ctypes

    import torch
    import torch.distributed as dist

    from paper_1101_1846_gb300 import capi, replicas
    from paper_1101_1846_gb300.generator import Generator

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    capi.lib()
    n, steps = args.n_streams, args.n_per_stream
    workload = f"full_2^{n.bit_length() - 1}x{steps}" if n & (n - 1) == 0 else f"{n}x{steps}"

    def barrier():
        if world > 1:
            dist.barrier()

    # weak scaling: rank r owns global streams r*n .. (r+1)*n - 1 of one
    # generator per kind (replicas.shard_spec)
    gens = {}
    for k in KINDS:
        s_begin, seed_k = replicas.shard_spec(k, rank, world, n, args.seed)
        gens[k] = Generator(k, n, seed_k, s_begin=s_begin)
    out = torch.empty((steps, n), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    pairs = [(k, f) for k in KINDS for f in FMTS]

    def one_step(events=None):
        for k, f in pairs:
            if events is not None:
                events[(k, f)][0].append(torch.cuda.Event(enable_timing=True))
                events[(k, f)][0][-1].record(stream)
            gens[k].generate(steps, f, out=out, stream=stream)
            if events is not None:
                events[(k, f)][1].append(torch.cuda.Event(enable_timing=True))
                events[(k, f)][1][-1].record(stream)

    for _ in range(max(args.warmup, 0)):
        one_step()
    torch.cuda.synchronize()

    clocks = Clocks(gpu_selector(torch))
    clocks.start()
    time.sleep(0.3)
    events = {p: ([], []) for p in pairs}
    barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        one_step(events)
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    clock_info = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    ms_max = replicas.max_over_ranks(ms, device="cuda")
    samples = world * args.steps * len(pairs) * n * steps
    value = replicas.job_rate(args.steps * len(pairs) * n * steps, world, ms_max * 1e-3) / 1e9

    per_kernel = {}
    for (k, f), (s_ev, e_ev) in events.items():
        d = [a.elapsed_time(b) for a, b in zip(s_ev, e_ev)]
        avg = sum(d) / len(d)
        b = alg_bytes(k, n, steps)
        per_kernel[f"{KNAME[k]}_{FNAME[f]}"] = {
            "ms": avg, "gsamples_s": n * steps / (avg * 1e-3) / 1e9,
            "gbs": b / (avg * 1e-3) / 1e9, "total_ms": sum(d)}
    dom = max(per_kernel, key=lambda x: per_kernel[x]["total_ms"])
    peak, peak_src = peaks()
    dk = KINDS[[KNAME[k] for k in KINDS].index(dom.split("_")[0])]
    achieved = alg_bytes(dk, n, steps) / (per_kernel[dom]["ms"] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": recorded_traffic(dom, workload),
                "kernel": dom, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs, "
                "copy read+write)" if peak_src == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": alg_bytes(dk, n, steps),
                "nominal_gbs": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS}
    # the integer pipes of every writeback kernel, against the probed peaks
    probes = run_int_probes((clock_info or {}).get("sm_mhz") or 2070.0, device_sms())
    for (k, f) in pairs:
        pk = per_kernel[f"{KNAME[k]}_{FNAME[f]}"]
        pk["int"] = int_roofline(k, f, pk["gsamples_s"] * 1e9, probes)
        rec = recorded_pipes(f"{KNAME[k]}_{FNAME[f]}")
        if rec:
            pk["int"]["ncu_pipes_pct"] = rec
    roofline["int"] = per_kernel[dom]["int"]
    roofline["int_probes"] = probes

    # write-only bandwidth probe over the same buffer (context for the roofline):
    # 32 CTAs of 256 threads per SM, streaming stores (7.2 TB/s on GB300,
    # against 6.5 with 8 CTAs per SM, all resident)
    nbytes = out.numel() * 4
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    capi.check(capi.lib().gbrng_probe_write(ctypes.c_void_p(out.data_ptr()), nbytes, sms * 32,
                                            256, 1, 1, ctypes.c_void_p(stream.cuda_stream)))
    pe0.record(stream)
    capi.check(capi.lib().gbrng_probe_write(ctypes.c_void_p(out.data_ptr()), nbytes, sms * 32,
                                            256, 1, 3, ctypes.c_void_p(stream.cuda_stream)))
    pe1.record(stream)
    torch.cuda.synchronize()
    write_only_gbs = 3 * nbytes / (pe0.elapsed_time(pe1) * 1e-3) / 1e9

    # end to end: the host-delivery call, D2H copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        del out
        torch.cuda.empty_cache()
        host, placement = pinned_near_gpu(torch, (steps, n), local)
        # warm-up: one untimed step of every pair (staging buffers, and the first
        # passes over a freshly pinned buffer, which reach host memory slowly)
        for k, f in pairs:
            gens[k].generate_host(steps, f, out=host)
        torch.cuda.synchronize()
        # the link itself: plain device-to-host copies into the same pinned
        # buffer, (a) 1 GiB at its start, best of three, and (b) the whole
        # buffer in 256 MiB pieces from one device buffer, the bytes and
        # pattern of one host-delivery call
        m = min(1 << 28, host.numel())
        src = torch.empty(m, dtype=torch.int32, device="cuda")
        flat = host.view(-1)
        link = []
        for _ in range(4):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            flat[:m].copy_(src, non_blocking=True)
            b.record(stream)
            b.synchronize()
            link.append(a.elapsed_time(b))
        link_gbs = 4 * m / (min(link[1:]) * 1e-3) / 1e9
        piece = min(1 << 26, flat.numel())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for off in range(0, flat.numel(), piece):
            k = min(piece, flat.numel() - off)
            flat[off:off + k].copy_(src[:k], non_blocking=True)
        b.record(stream)
        b.synchronize()
        link_full_gbs = 4 * flat.numel() / (a.elapsed_time(b) * 1e-3) / 1e9
        del src
        barrier()
        per_pair = {p: 0.0 for p in pairs}
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            for k, f in pairs:
                tp = time.perf_counter()
                gens[k].generate_host(steps, f, out=host)  # synchronous
                per_pair[(k, f)] += time.perf_counter() - tp
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        # the link again, after the timed region (the host's memory is shared)
        src = torch.empty(piece, dtype=torch.int32, device="cuda")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for off in range(0, flat.numel(), piece):
            k = min(piece, flat.numel() - off)
            flat[off:off + k].copy_(src[:k], non_blocking=True)
        b.record(stream)
        b.synchronize()
        link_after_gbs = 4 * flat.numel() / (a.elapsed_time(b) * 1e-3) / 1e9
        del src
        dt = replicas.max_over_ranks(dt, device="cuda")
        e2e_samples = world * args.e2e_steps * len(pairs) * n * steps
        e2e = {"value": e2e_samples / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": 0,
               "d2h_bytes_per_step": len(pairs) * n * steps * 4,
               "steps": args.e2e_steps,
               "api": "rng_generate_host into pinned host memory",
               "d2h_gbs": len(pairs) * n * steps * 4 * args.e2e_steps / dt / 1e9,
               "plain_copy_d2h_gbs": link_gbs, "plain_copy_whole_buffer_d2h_gbs": link_full_gbs,
               "plain_copy_whole_buffer_after_d2h_gbs": link_after_gbs,
               "per_pair_d2h_gbs": {f"{KNAME[k]}_{FNAME[f]}":
                                    round(4 * n * steps * args.e2e_steps / t / 1e9, 1)
                                    for (k, f), t in per_pair.items()},
               "host_buffer": placement}
        e2e["of_plain_copy"] = e2e["d2h_gbs"] / link_gbs
        e2e["of_plain_copy_whole_buffer"] = e2e["d2h_gbs"] / link_full_gbs

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        del gens
        torch.cuda.empty_cache()
        extras = run_extras(args, (clock_info or {}).get("sm_mhz") or 2070.0)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(steps, 1 << 15)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        cpu["cpu_model"] = cpu_model()
        cpu["single_thread"] = cpu_single_thread()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": workload, "kinds": ["mwc", "xor128", "kiss"],
                       "fmts": ["u32", "f32"], "n_streams": n, "n_per_stream": steps,
                       "launches_per_step": len(pairs), "state": "carried across calls",
                       "l2": "16 GiB output per launch >> 129 MB L2; no flush"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": args.steps * len(pairs), "clocks": clock_info,
            "per_kernel": per_kernel, "write_only_probe_gbs": write_only_gbs,
        }
        line.update(extras)
        # the batched and saturating serving rates against this run's
        # single-instance full-device rate
        if "batched" in line:
            line["batched"]["over_plain_full_device"] = line["batched"]["value"] / value
        sat = line.get("serving", {}).get("saturating")
        if sat:
            sat["over_plain_full_device"] = sat["gsamples_s"] / value
        # a compact summary of the other workloads inside the roofline entry,
        # each rate as a fraction of the copy peak (4 bytes per sample plus
        # the state, as the roofline counts them)
        summary = {}
        for name, r in line.get("other_configs", {}).items():
            kname, _, rest = name.partition("_")
            k = {v: i for i, v in KNAME.items()}[kname]
            nn, ss = (1 << 20, 1024) if "2^20" in rest else (4096, 4096)
            gbs = alg_bytes(k, nn, ss) / (r["ms"] * 1e-3) / 1e9
            summary[name] = {"gsamples_s": round(r["gsamples_s"], 1),
                             "frac": round(gbs / peak, 3)}
            if nn == 4096:  # 16.8 M samples per call: a latency, not a roofline point
                summary[name]["us_per_call"] = round(r["ms"] * 1e3, 1)
                summary[name]["note"] = "latency-bound (few streams, split into jumped segments)"
        if "batched" in line:
            summary["batched_10000"] = {
                "gsamples_s": round(line["batched"]["value"], 1),
                "over_plain_full_device": round(line["batched"]["over_plain_full_device"], 3)}
            if "roofline" in line["batched"]:
                summary["batched_10000"]["frac"] = round(line["batched"]["roofline"]["frac"], 3)
        if sat:
            summary["serving_saturating"] = {
                "gsamples_s": round(sat["gsamples_s"], 1),
                "over_plain_full_device": round(sat["over_plain_full_device"], 3)}
        if summary:
            line["roofline"]["configs"] = summary
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------- batched
def run_batched(args):
    """10,000 mixed instances (workloads.batched_instances).  Instances are
    cut into pieces of at most --chunk-rows rows (the state carries from
    piece to piece, so the pieces give exactly the rows of one call), and
    the pieces are packed into waves of at most --wave-gib of output
    (scheduler.laned_waves: --lanes groups of instances, each with waves of
    its own).  Every wave is one plan (one persistent kernel) captured in a
    CUDA graph; a lane's waves run in order on its own stream, and the lanes
    overlap.  The same instances then run as plain per-instance
    launches (timed), and a separate untimed pass checks every piece of
    every wave bit for bit against plain calls."""
    import torch

    from paper_1101_1846_gb300 import autotune, capi, laned, scheduler, workloads
    from paper_1101_1846_gb300.generator import BatchItem, Generator, Plan

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    capi.lib()
    inst = workloads.batched_instances(args.instances, 1234)
    budget = int(args.wave_gib * (1 << 30))
    lanes = max(1, args.lanes)
    laned_pairs = scheduler.laned_waves([i.n_streams for i in inst],
                                        [i.n_per_stream for i in inst], budget,
                                        args.chunk_rows, lanes)
    waves = [w for _, w in laned_pairs]
    main = torch.cuda.current_stream()
    # A lane's waves continue the same instances, so they run in order on the
    # lane's stream and reuse the lane's buffer; lanes share no instance and
    # overlap.  The check pass below needs two buffers.
    R = max(2, lanes)
    longest = max(4 * i.n_streams * i.n_per_stream for i in inst)  # plain calls write whole
    cap = max(budget, longest) // 4 + 4 * max(len(w) for w in waves)
    bufs = [torch.empty(cap, dtype=torch.int32, device="cuda") for _ in range(R)]
    n_streams = [i.n_streams for i in inst]
    fmts = [i.fmt for i in inst]

    def make_gens():
        return [Generator(i.kind, i.n_streams, i.seed) for i in inst]

    def items_for(gens, wave, outs):
        return [BatchItem(gens[p.inst], p.rows, o, inst[p.inst].fmt) for p, o in zip(wave, outs)]

    t0 = time.perf_counter()
    gb = make_gens()
    create_s = time.perf_counter() - t0

    shape, tune_ms = (0, 0), None
    if args.tune:
        tg = make_gens()
        shape, tune_ms = autotune.tune_plan(items_for(tg, waves[0],
                                                      laned.carve(bufs[0], waves[0], n_streams)))
        for g in tg:
            g.close()

    # plans and graphs for every wave, built before the timed region
    run = laned.LanedGraphs(laned_pairs, gb, fmts, lambda k, lane, w: bufs[lane],
                            threads=shape[0], ctas_per_sm=shape[1])
    tiles = run.tiles

    samples = sum(i.n_streams * i.n_per_stream for i in inst)
    # bytes the waves must move: every piece writes its rows and reads and
    # writes back its streams' state (and reads their multipliers)
    moved = sum(alg_bytes(inst[p.inst].kind, inst[p.inst].n_streams, p.rows)
                for w in waves for p in w)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    run.replay()
    e1.record(main)
    torch.cuda.synchronize()
    b_ms = e0.elapsed_time(e1)
    run.close()

    # plain per-instance launches (one call per instance, one stream)
    gp = make_gens()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(main)
    for i, ins in enumerate(inst):
        gp[i].generate(ins.n_per_stream, ins.fmt, out=bufs[i % R], stream=main)
    p1.record(main)
    torch.cuda.synchronize()
    p_ms = p0.elapsed_time(p1)
    states_equal = all(torch.equal(a.get_state(), b.get_state()) for a, b in
                       zip(gb[::41], gp[::41]))
    for g in gb + gp:
        g.close()

    # untimed check: every piece of every wave against plain calls
    mismatched, checked = 0, 0
    if not args.no_verify:
        vb, vp = make_gens(), make_gens()
        for w in waves:
            ob, op = laned.carve(bufs[0], w, n_streams), laned.carve(bufs[1], w, n_streams)
            plan = Plan(items_for(vb, w, ob), threads=shape[0], ctas_per_sm=shape[1])
            plan.launch(main)
            for p, o in zip(w, op):
                vp[p.inst].generate(p.rows, inst[p.inst].fmt, out=o, stream=main)
            torch.cuda.synchronize()
            for x, y in zip(ob, op):
                checked += 1
                if not torch.equal(x, y):
                    mismatched += 1
            plan.close()
        states_equal = states_equal and all(
            torch.equal(a.get_state(), b.get_state()) for a, b in zip(vb, vp))
        for g in vb + vp:
            g.close()

    line = {
        "metric": METRIC, "workload": f"batched_{args.instances}", "impl": "ours",
        "value": samples / (b_ms * 1e-3) / 1e9, "unit": UNIT,
        "plain_per_instance_value": samples / (p_ms * 1e-3) / 1e9,
        "batched_over_plain_per_instance": p_ms / b_ms, "samples": samples,
        "bytes": 4 * samples, "waves": len(waves), "pieces": sum(len(w) for w in waves),
        "lanes": lanes, "tiles": tiles, "chunk_rows": args.chunk_rows,
        "batched_ms": b_ms, "plain_ms": p_ms, "plain_launches": len(inst),
        "gpu_launches": len(waves), "plan_shape": list(shape), "tune_ms":
            {f"{t}x{c}": v for (t, c), v in tune_ms.items()} if tune_ms else None,
        "bit_identical": (mismatched == 0 and states_equal) if not args.no_verify else None,
        "pieces_checked": checked, "mismatched_pieces": mismatched, "create_s": create_s,
        "realigned_instances": sum(1 for i in inst if i.n_streams % 4),
        "roofline": {"bound": "hbm", "algorithmic_bytes": moved,
                     "state_bytes_over_output": moved / (4 * samples) - 1,
                     "achieved": moved / (b_ms * 1e-3) / 1e9, "peak": peaks()[0],
                     "frac": moved / (b_ms * 1e-3) / 1e9 / peaks()[0], "unit": "GB/s"},
        "config": {"workload": "batched", "instances": args.instances, "seed": 1234,
                   "wave_bytes": budget, "graph": "one CUDA graph per wave",
                   "order": f"{lanes} lanes: a lane's waves in order on its own stream "
                            "and buffer, lanes overlapping"},
    }
    return line


# --------------------------------------------------------------- serving
def _probe_sequences(clients, streams, seed_of, rows, golden):
    """Oracle outputs (uint32 and float32 bits) of a few streams per client,
    rows 0 .. rows-1: the streams are golden-file indices, whose multipliers
    the oracle wrote there."""
    import numpy as np

    import oracle
    idx = [s for s in golden["sample_index"] if s < streams]
    probes = [idx[0], idx[1], idx[255 % len(idx)], idx[-1]]
    a_of = dict(zip(golden["sample_index"], golden["sample_a"]))
    seqs = {}
    for c in clients:
        for s in probes:
            a = np.array([a_of[s]], dtype=np.uint32)
            st = oracle.seed_streams(2, a, seed_of(c), np.array([s]))[0]
            u, _ = oracle.stream(2, int(a[0]), st, rows[c], 0)
            f, _ = oracle.stream(2, int(a[0]), st, rows[c], 1)
            seqs[(c, s)] = (u, f.view(np.uint32))
    return probes, seqs


def run_serving(args):
    """Poisson arrivals at --rate requests/s for --duration s over 256
    clients (65536-stream KISS generators resident on the device), sizes
    log-uniform on [1 KiB, 256 MiB] (workloads.request_log), admission under
    a 40 GB budget; real time, then the same requests all at once
    (saturating).  Every --verify-every-th request is checked against the
    oracle on four probe streams of its client."""
    import numpy as np
    import torch

    from paper_1101_1846_gb300 import capi, workloads
    from paper_1101_1846_gb300.serving import Server, replay

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    capi.lib()
    n_clients, streams = 256, 65536
    log = workloads.request_log(args.rate, args.duration, n_clients, 1024, 256 << 20, seed=5)
    golden = json.loads((ROOT / "tests" / "golden" / "multipliers_b32.json").read_text())
    chunk_rows = args.serve_chunk_rows
    server = Server(capi.RNG_KISS, n_clients, streams, seed_base=args.seed,
                    budget_bytes=int(args.budget_gib * (1 << 30)), chunk_rows=chunk_rows,
                    tick_bytes=int(args.tick_gib * (1 << 30)))
    totals = {}
    for r in log:
        totals[r.client] = totals.get(r.client, 0) + r.n_samples
    rows = {c: t // streams + 2 for c, t in totals.items()}
    checked, bad = [0], [0]
    probes, seqs = (None, None)
    if args.verify_every > 0 and not args.no_verify:
        probes, seqs = _probe_sequences(sorted(totals), streams, server.client_seed, rows,
                                        golden)
    active = []  # the engine being checked

    def on_done(rid, req):
        if probes is None or rid % args.verify_every:
            return
        srv = active[0]
        info = srv.result(rid)
        start, N = info["start"], info["n"]
        out = srv.copy(rid, out=torch.empty(N, dtype=torch.int32, pin_memory=True))
        out = out.numpy().view(np.uint32)
        for s in probes:
            col = (s - start) % streams
            if col >= N:
                continue
            cnt = (N - 1 - col) // streams + 1
            got = out[col::streams]
            assert len(got) == cnt
            row0 = (start + col) // streams
            u, f = seqs[(info["client"], s)]
            exp = (u if info["fmt"] == 0 else f)[row0:row0 + cnt]
            checked[0] += 1
            if not np.array_equal(got, exp):
                bad[0] += 1

    if args.saturating_only:
        server.close()
        probes = None
        live = None
    else:
        live = replay(server, log, realtime=True).summary()
        server.close()
    # saturating run: the same requests, all submitted at once, with the
    # engine's tick sized for throughput (after a short warm-up engine)
    sat_tick = int(args.sat_tick_gib * (1 << 30))
    warm = Server(capi.RNG_KISS, n_clients, streams, seed_base=args.seed,
                  budget_bytes=int(args.budget_gib * (1 << 30)), chunk_rows=chunk_rows, tick_bytes=sat_tick)
    replay(warm, log[:2000], realtime=False)
    warm.close()
    server2 = Server(capi.RNG_KISS, n_clients, streams, seed_base=args.seed,
                     budget_bytes=int(args.budget_gib * (1 << 30)), chunk_rows=chunk_rows, tick_bytes=sat_tick)
    sat = replay(server2, log, realtime=False).summary()
    sat["tick_bytes"] = sat_tick
    server2.close()
    # untimed check: the same requests again, probing every k-th result
    if probes is not None:
        server3 = Server(capi.RNG_KISS, n_clients, streams, seed_base=args.seed,
                         budget_bytes=int(args.budget_gib * (1 << 30)), chunk_rows=chunk_rows,
                    tick_bytes=int(args.tick_gib * (1 << 30)))
        active.append(server3)
        replay(server3, log, realtime=False, on_done=on_done)
        server3.close()
    if live is None:
        return {"metric": METRIC, "workload": "serving_saturating", "impl": "ours",
                "value": sat["gsamples_s"], "unit": UNIT, "saturating": sat,
                "config": {"clients": n_clients, "streams_per_client": streams,
                           "duration_s": args.duration, "budget_bytes":
                           int(args.budget_gib * (1 << 30)), "tick_bytes": sat_tick}}
    line = {
        "metric": METRIC, "workload": "serving", "impl": "ours",
        "value": live["gsamples_s"], "unit": UNIT,
        "p50_ms": live["p50_ms"], "p99_ms": live["p99_ms"], "mean_ms": live["mean_ms"],
        "requests": live["requests"], "samples": live["samples"], "wall_s": live["wall_s"],
        "offered_gsamples_s": sum(r.n_samples for r in log) / args.duration / 1e9,
        "saturating": sat, "probe_checks": checked[0], "probe_mismatches": bad[0],
        "bit_exact_probes": (bad[0] == 0) if checked[0] else None,
        "max_arena_used_bytes": live["max_arena_used"], "ticks": live["ticks"],
        "config": {"workload": "serving", "clients": n_clients, "streams_per_client": streams,
                   "kind": "kiss", "rate_hz": args.rate, "duration_s": args.duration,
                   "sizes": "log-uniform [1 KiB, 256 MiB]",
                   "budget_bytes": int(args.budget_gib * (1 << 30)),
                   "chunk_rows": chunk_rows, "tick_bytes": int(args.tick_gib * (1 << 30)),
                   "seed_base": args.seed},
    }
    return line


L2_FLUSH_BYTES = 512 << 20  # four times the 129 MB L2


def _flush_l2(_buf=[]):
    """Writes a buffer larger than L2 so that the next timed call starts
    with none of its output lines resident."""
    import torch
    if not _buf:
        _buf.append(torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda"))
    _buf[0].fill_(0)


def _plain_rate(kind, n, steps, fmt, seed, reps=11):
    """Median CUDA-event time of one rng_generate call (the L2 is flushed
    before each timed call whose output is smaller than four L2s)."""
    import torch

    from paper_1101_1846_gb300.generator import Generator
    g = Generator(kind, n, seed)
    out = torch.empty((steps, n), dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    flush = 4 * n * steps < L2_FLUSH_BYTES
    g.generate(steps, fmt, out=out)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush:
            _flush_l2()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        g.generate(steps, fmt, out=out)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    g.close()
    ms = sorted(ts)[len(ts) // 2]
    return {"ms": ms, "gsamples_s": n * steps / (ms * 1e-3) / 1e9, "l2_flushed": flush}


# Integer operations per sample in the paper's counting (Eq. 9's n_ops: every
# 32-bit shift, logical op, add or multiply-add counts one): MWC32 = the
# two halves of the 32 x 32 + 32 -> 64 multiply-add; xor128 = 3 shifts +
# 4 xors; KISS = MWC 2 + xorshift32 6 + LCG 1 + 2 adds.  The sum consumer
# adds 2 (a 64-bit add as add-with-carry).
GEN_OPS = {0: 2, 1: 7, 2: 11}
SUM_OPS = 2
LANES_PER_SM_CLK = 128  # 4 schedulers x 32 lanes issue per clock

# The integer work of one output by operation class of the probes
# (gbrng_probe_int): mwc_step = one 32 x 32 + 32 -> 64 multiply-add (two
# instructions), lcg_mad = one 32-bit multiply-add, shift_xor = one shift and
# one xor, add = one 32-bit add or a lone logic op.  xor128: t = x ^ (x << 11),
# w ^ (w >> 19), ^ (t >> 8) are three shift-xors and ^ t a lone xor; KISS: the
# MWC step, the LCG, xorshift32's three shift-xors and the two adds of the
# sum.  FP32 output adds the shift of u >> 8 (the convert and the multiply run
# on the floating-point pipes).
OP_MIX = {0: {"mwc_step": 1}, 1: {"shift_xor": 3, "add": 1},
          2: {"mwc_step": 1, "lcg_mad": 1, "shift_xor": 3, "add": 2}}
F32_EXTRA = {"add": 1}


def device_sms() -> int:
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def alu_peak_tops(mhz: float, sms: int) -> float:
    """Issue-limited integer rate: SMs x 4 schedulers x 32 lanes per clock,
    at the given SM clock."""
    return sms * LANES_PER_SM_CLK * mhz * 1e6 / 1e12


def int_roofline(kind: int, fmt: int, samples_per_s: float, probes: dict) -> dict:
    """How much of the probed integer throughput a writeback kernel's
    arithmetic uses: per operation class, samples/s x operations per sample
    / the probe's operations/s for that class (the measured peak of the
    pipe that runs it); `bound` is the class nearest its peak and `serial`
    the sum over classes (the fraction if every class shared one pipe)."""
    mix = dict(OP_MIX[kind])
    if fmt == 1:
        for c, v in F32_EXTRA.items():
            mix[c] = mix.get(c, 0) + v
    fr = {c: samples_per_s * v / probes[c]["ops_per_s"] for c, v in mix.items()}
    bound = max(fr, key=fr.get)
    return {"bound": bound, "frac": fr[bound], "serial": sum(fr.values()),
            "classes": fr, "ops_per_sample": mix,
            "peak_source": "gbrng_probe_int on this device, this run"}


def _reduce_rate(kind, n, steps, op, seed, reps=5):
    import torch

    from paper_1101_1846_gb300.generator import Generator
    g = Generator(kind, n, seed)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    g.generate_reduce(steps, op, out=out)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        g.generate_reduce(steps, op, out=out)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    g.close()
    ms = sorted(ts)[len(ts) // 2]
    return {"ms": ms, "gsamples_s": n * steps / (ms * 1e-3) / 1e9}


def _jump_ms(kind, n, k, seed, reps=5):
    import torch

    from paper_1101_1846_gb300.generator import Generator
    g = Generator(kind, n, seed)
    s = torch.cuda.current_stream()
    g.jump(k)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        g.jump(k)
        b.record(s)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    g.close()
    return sorted(ts)[len(ts) // 2]


def run_int_probes(clock_mhz: float, sms: int):
    """Integer-pipe probes (gbrng_probe_int): 8 independent chains per
    thread of one operation, 1216 CTAs x 256 threads.  Returns, per op, the
    operations per second and the lane-instructions per SM per clock."""
    import ctypes

    import torch

    from paper_1101_1846_gb300 import capi
    blocks, threads, iters = sms * 8, 256, 1 << 13
    sink = torch.empty(blocks * threads, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    names = {0: ("mwc_step", 2), 1: ("lcg_mad", 1), 2: ("shift_xor", 2), 3: ("add", 1)}
    res = {}
    for op, (name, instr) in names.items():
        def launch():
            capi.check(capi.lib().gbrng_probe_int(op, ctypes.c_void_p(sink.data_ptr()), blocks,
                                                  threads, iters, ctypes.c_void_p(s.cuda_stream)))
        launch()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        launch()
        b.record(s)
        b.synchronize()
        sec = a.elapsed_time(b) * 1e-3
        ops = blocks * threads * iters * 8 / sec
        res[name] = {"ops_per_s": ops, "instr_per_op": instr,
                     "lane_instr_per_sm_clk": ops * instr / (sms * clock_mhz * 1e6)}
    return res


def run_inline(clock_mhz: float):
    """The generators with the numbers used in registers (no output array):
    per kind, the sum consumer and the quarter-disc count at 2^22 streams x
    1024 outputs, with the integer-ALU roofline of the sum consumer; and
    rng_jump over 2^22 streams."""
    import ctypes

    from paper_1101_1846_gb300 import capi
    n, steps = 1 << 22, 1024
    sms = device_sms()
    peak = alu_peak_tops(clock_mhz, sms)
    res = {"workload": f"2^22 streams x {steps} outputs, no output array",
           "alu_peak_tops": peak,
           "alu_peak_basis": f"{sms} SMs x 128 lanes/clk x {clock_mhz} MHz", "kinds": {}}
    for kind in KINDS:
        r = _reduce_rate(kind, n, steps, capi.RNG_SUM_U32, 11)
        d = _reduce_rate(kind, n, steps, capi.RNG_DISC, 11)
        ops = GEN_OPS[kind] + SUM_OPS
        tops = ops * n * steps / (r["ms"] * 1e-3) / 1e12
        res["kinds"][KNAME[kind]] = {
            "sum_u32": r, "disc": d,
            "roofline": {"bound": "alu", "achieved": tops, "peak": peak, "unit": "Tops/s",
                         "frac": tops / peak, "ops_per_sample": ops},
            "jump_2^22_streams_by_2^40+1_ms": _jump_ms(kind, n, (1 << 40) + 1, 5)}
    probes = run_int_probes(clock_mhz, sms)
    res["int_probes"] = probes
    # the same rates against the probed peak of each operation class (the
    # sum consumer's 64-bit add is two adds), as for the writeback kernels
    for kind in KINDS:
        kk = res["kinds"][KNAME[kind]]
        r = int_roofline(kind, 0, kk["sum_u32"]["gsamples_s"] * 1e9, probes)
        extra = 2 * kk["sum_u32"]["gsamples_s"] * 1e9 / probes["add"]["ops_per_s"]
        r["classes"]["add"] = r["classes"].get("add", 0.0) + extra
        r["ops_per_sample"]["add"] = r["ops_per_sample"].get("add", 0) + 2
        r["bound"] = max(r["classes"], key=r["classes"].get)
        r["frac"] = r["classes"][r["bound"]]
        r["serial"] = sum(r["classes"].values())
        kk["int_probe_roofline"] = r
    mwc = res["kinds"]["mwc"]["sum_u32"]["gsamples_s"] * 1e9
    res["kinds"]["mwc"]["of_probed_mwc_step_rate"] = mwc / probes["mwc_step"]["ops_per_s"]
    # few streams: the 4096 x 4096 MWC call with and without splitting
    v = ctypes.c_int()
    capi.check(capi.lib().gbrng_get_split(0, ctypes.byref(v)))
    res["mwc_u32_4096x4096_split"] = _plain_rate(0, 4096, 4096, 0, 42)
    capi.check(capi.lib().gbrng_set_split(0, 0))
    try:
        res["mwc_u32_4096x4096_unsplit"] = _plain_rate(0, 4096, 4096, 0, 42)
    finally:
        capi.check(capi.lib().gbrng_set_split(0, v.value))
    return res


# The paper's rates on a GTX280 (GSamples/s, uint32; Tables I-III), for
# context only: another card, another year.
PAPER_GTX280 = {"mwc16x2": {"with_writeback": 18.0, "without_writeback": 37.5},
                "xorshift8": {"with_writeback": 12.5, "without_writeback": 14.5},
                "kiss_xor": {"with_writeback": 9.2, "without_writeback": 19.1}}


def run_paper_variants():
    """The paper's own generators: writeback (uint32 to HBM) and inline (sum
    consumer) rates.  The two MWC-pair kinds have at most 76,636 streams (the
    pairs of 392 multipliers), so they run 76,636 x 16,384 per call, cut into
    jumped segments; XORSHIFT8 runs 2^22 x 1024 like the target kinds."""
    from paper_1101_1846_gb300 import capi
    res = {}
    for kind, name, n, steps in ((3, "mwc16x2", capi.RNG_MAX_STREAMS_MWC16, 16384),
                                 (4, "xorshift8", 1 << 22, 1024),
                                 (5, "kiss_xor", capi.RNG_MAX_STREAMS_MWC16, 16384)):
        w = _plain_rate(kind, n, steps, 0, 21)
        r = _reduce_rate(kind, n, steps, capi.RNG_SUM_U32, 21)
        res[name] = {"workload": f"{n} streams x {steps} outputs",
                     "with_writeback": {**w, "tb_s": 4 * n * steps / (w["ms"] * 1e-3) / 1e12},
                     "without_writeback_sum": r,
                     "paper_gtx280_gsamples_s": PAPER_GTX280[name]}
    return res


def run_battery():
    """The battery's p-values for every kind over 2^20 streams x 1024
    uint32 outputs (the pair kinds: 76,636 x 16,384), and the time of the
    counting call."""
    import torch

    from paper_1101_1846_gb300 import battery, capi
    from paper_1101_1846_gb300.generator import Generator
    names = {0: "mwc", 1: "xor128", 2: "kiss", 3: "mwc16x2", 4: "xorshift8", 5: "kiss_xor"}
    res = {}
    for kind, name in names.items():
        n, rows = ((capi.RNG_MAX_STREAMS_MWC16, 16384) if kind in (3, 5) else (1 << 20, 1024))
        g = Generator(kind, n, 99)
        u = g.generate(rows)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = battery.counts(u, n, rows)
        dt = time.perf_counter() - t0
        st = battery.statistics(c)
        res[name] = {"outputs": n * rows, "count_ms": dt * 1e3, "passed": battery.passed(st),
                     **{k: round(v["p"], 6) for k, v in st.items()},
                     "birthday_samples": st["birthday"]["samples"]}
        del u
        g.close()
        torch.cuda.empty_cache()
    return res


def run_extras(args, clock_mhz: float = 2070.0):
    """The other workloads, summarised for the same JSON line: the 2^20 x 1024
    xor128/KISS calls, the 4096 x 4096 MWC call (few streams: split into
    jumped segments), the inline consumers, the batched 10,000-instance
    workload and the serving loop."""
    extras = {"other_configs": {}}
    for kind, kn in ((1, "xor128"), (2, "kiss")):
        for fmt, fn in ((0, "u32"), (1, "f32")):
            extras["other_configs"][f"{kn}_{fn}_2^20x1024"] = _plain_rate(kind, 1 << 20, 1024,
                                                                          fmt, 7)
    extras["other_configs"]["mwc_u32_4096x4096"] = _plain_rate(0, 4096, 4096, 0, 42)
    extras["inline"] = run_inline(clock_mhz)
    extras["paper_variants"] = run_paper_variants()
    extras["battery"] = run_battery()
    keep = ("value", "plain_per_instance_value", "bit_identical", "pieces_checked",
            "mismatched_pieces", "waves", "pieces", "tiles", "chunk_rows", "plan_shape",
            "batched_ms", "gpu_launches", "roofline")
    b = run_batched(args)  # the library's default plan shape (--tune to sweep shapes)
    extras["batched"] = {k: b[k] for k in keep if k in b}
    s = run_serving(args)
    extras["serving"] = {k: s[k] for k in ("value", "p50_ms", "p99_ms", "mean_ms", "requests",
                                           "offered_gsamples_s", "saturating", "probe_checks",
                                           "probe_mismatches", "bit_exact_probes", "config")}
    return extras


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        print(json.dumps(run_batched(args)))
    elif args.workload == "serving":
        print(json.dumps(run_serving(args)))
    elif args.workload == "inline":
        print(json.dumps(run_inline(2070.0)))
    elif args.workload == "paper":
        print(json.dumps(run_paper_variants()))
    elif args.workload == "battery":
        print(json.dumps(run_battery()))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
