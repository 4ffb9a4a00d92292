#!/usr/bin/env python3
"""Benchmark of the GB300 particle position compressor (arXiv 2404.02826 hot path).

One step = compress + decompress of one synthetic snapshot through the C ABI
(value range, quantization, k-d partition, bit boxes, packing, then unpack and
dequantize).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

value      uncompressed bytes (n * 3 * sizeof(T)) through one round trip per
           second, inputs already resident in HBM; whole job over all ranks
e2e        the same metric through the host-buffer entry points: positions
           copied in from pinned memory, the stream copied out, copied back in
           and the positions copied out, every step
roofline   the kernel with the largest traced time: algorithmic bytes per
           launch / mean launch time (CUDA events on the launching stream, in a
           second pass of the same steps: tracing is off in the timed region),
           against the measured HBM copy bandwidth
cpu_baseline  the oracle (single thread) on a bounded sample of the workload

With N > 1 (torchrun), every rank compresses its own snapshot (replicas, no
collective on the data path); time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: generator, n, dtype, eb mode, eb
    "cosmology-2^27-f32-rel1e-4": ("cosmology", 1 << 27, "f32", "rel", 1e-4),
    "cosmology-2^27-f32-rel1e-3": ("cosmology", 1 << 27, "f32", "rel", 1e-3),
    "uniform-2^20-f32-rel1e-3": ("uniform", 1 << 20, "f32", "rel", 1e-3),
    "fluid-2^24-f64-abs1e-4": ("fluid", 1 << 24, "f64", "abs", 1e-4),
    "cosmology-2^24-f32-rel1e-4": ("cosmology", 1 << 24, "f32", "rel", 1e-4),
    "cosmology-2^25-f32-rel1e-4": ("cosmology", 1 << 25, "f32", "rel", 1e-4),
}
DEFAULT_WORKLOAD = "cosmology-2^27-f32-rel1e-4"
CPU_SAMPLE = 1 << 23        # particles of the oracle's timed sample (cpu_baseline): about 13 s on one core
REF_SAMPLE = 1 << 20        # particles per step of the reference arm
METRIC = "compress+decompress round-trip throughput (uncompressed bytes)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch-256", "serve-2000", "leaf-sweep"], default=DEFAULT_WORKLOAD)
    ap.add_argument("--leaf-size", type=int, default=4096)
    ap.add_argument("--autotune", action="store_true",
                    help="leaf size chosen by the autotuner (then --leaf-size is the largest candidate, "
                         "0 = PC_MAX_LEAF_SIZE)")
    ap.add_argument("--reduce", action="store_true",
                    help="compress with the bit-box reduction (Sec. 4.1, Alg. 1) in place of plain leaves")
    ap.add_argument("--reorder", action="store_true",
                    help="reorder sequences by sum m_d and particles by R-index (Sec. 4.2) before packing")
    ap.add_argument("--widest", action="store_true",
                    help="split every k-d node on the axis of its widest cell (else depth mod 3)")
    ap.add_argument("--lossless", action="store_true",
                    help="after the timed steps, compress the stream once more on the host with zlib (DEFLATE: "
                         "LZ77 + Huffman, standing in for Huffman + ZSTD) and report that ratio separately")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the untimed extras of the default run: the other workloads' one-line results, "
                         "the batch-256 and serve-2000 summaries")
    return ap.parse_args()


def generate(gen, n, dtype, seed):
    import numpy as np

    import synth

    dt = np.float32 if dtype == "f32" else np.float64
    return synth.by_name(gen, n, seed=seed, dtype=dt)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while it runs."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "20"]
        if gpu_id:
            cmd.insert(1, f"--id={gpu_id}")
        self.rows = []
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [r for t, r in self.rows if t0 <= t <= t1 + 0.05 and len(r) >= 9]
        window = "timed"
        if not rows:  # region shorter than the sampling period: take the samples around it
            rows = [r for t, r in self.rows if t0 - 1.0 <= t <= t1 + 1.0 and len(r) >= 9]
            window = "around-timed"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no-samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "window": window,
                "power_w_max": max(pw) if pw else None}


def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    """Largest value over the ranks (the timed region of the slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(world: int, bytes_per_rank_step: int, steps: int, max_ms: float) -> float:
    """Whole-job throughput: every rank's bytes over the slowest rank's time."""
    return world * bytes_per_rank_step * steps / (max_ms / 1e3) / 1e9


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, workload: str, n: int):
    """DRAM bytes per launch of `kernel` from a committed ncu capture, scaled to
    n particles; None when the capture is missing or the kernel source changed."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            rec = json.load(f)[kernel]
        if rec["source_hash"] != source_hash(rec["sources"]):
            return None
        return rec["dram_bytes_per_particle"] * n
    except Exception:
        return None


def algorithmic_bytes(kernel, n, esz, cb, stream_bytes, with_idx=False, launches=1):
    """Bytes a launch must move at minimum (per-kernel figures, stated in the design notes).
    The reduction's take kernel runs once per round: over all rounds it must read
    every particle's codes once and write its sequence and rank once."""
    idx = 4 if with_idx else 0
    if kernel == "k_rd_take":
        return (3 * cb + 8) * n / max(launches, 1)
    if kernel == "k_ro_sort":  # reads and writes every particle's codes (and index) once
        return 2 * (3 * cb + idx) * n
    return {
        "k_range": 3 * esz * n,
        "k_quantize": 3 * esz * n + 3 * cb * n + idx * n,
        "k_hist": cb * n,
        "k_median": cb * n,
        "k_count": cb * n,
        "k_scatter": 2 * (3 * cb + idx) * n,
        "k_leafbox": 3 * cb * n,
        "k_leafpack": 3 * cb * n + stream_bytes,
        "k_decode": stream_bytes + 3 * esz * n,
        # the deep levels, bit boxes and packing on chip: every particle's codes read once, the stream written
        "k_subtree": 3 * cb * n + idx * n + stream_bytes,
        # the leaf-size search's on-chip pass: every particle's codes read once (the arrangement it
        # writes back when the search goes deeper is not counted)
        "k_subtree_cost": 3 * cb * n + idx * n,
    }.get(kernel)


def oracle_round_trip(pos, mode, eb, leaf_size, reduce=False, reorder=False, parallel=False, widest=False):
    import oracle

    m = oracle.REL if mode == "rel" else oracle.ABS
    if reduce:
        stream, _, _ = oracle.compress_reduced(pos, m, eb, leaf_size=leaf_size, want_perm=False, parallel=parallel,
                                               widest=widest)
    else:
        stream, _ = oracle.compress(pos, m, eb, leaf_size=leaf_size, want_perm=False, parallel=parallel,
                                    widest=widest)
    if reorder:
        stream, _, _ = oracle.reorder(stream)
    oracle.decompress(stream, parallel=parallel)
    return len(stream)


def oracle_round_trip_parallel(pos, mode, eb, leaf_size, reduce=False, reorder=False, widest=False):
    return oracle_round_trip(pos, mode, eb, leaf_size, reduce, reorder, parallel=True, widest=widest)


def cpu_baseline(spec, leaf_size, n_sample=CPU_SAMPLE, reduce=False, reorder=False, widest=False):
    gen, n, dtype, mode, eb = spec
    pos = generate(gen, n_sample, dtype, seed=0)
    t0 = time.perf_counter()
    oracle_round_trip(pos, mode, eb, leaf_size, reduce, reorder, widest=widest)
    dt = time.perf_counter() - t0
    out = {"value": round(pos.nbytes / dt / 1e9, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
           "sample": f"{n_sample} particles of the {gen} generator ({dtype}, {mode} eb {eb}), one compress + "
                     f"decompress in {dt:.2f} s"}
    # the same oracle source built with OpenMP, on every host core, on a 4x larger sample
    import oracle

    oracle.build(parallel=True)
    big = generate(gen, (1 if reduce else 4) * n_sample, dtype, seed=0)
    oracle_round_trip_parallel(big[: 1 << 16], mode, eb, leaf_size, reduce, reorder, widest)  # thread pool start-up
    t0 = time.perf_counter()
    oracle_round_trip_parallel(big, mode, eb, leaf_size, reduce, reorder, widest)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out["parallel"] = {"value": round(big.nbytes / dt / 1e9, 6), "unit": "GB/s", "cores": cores,
                       "kind": "oracle, OpenMP build of the same source",
                       "sample": f"{big.shape[0]} particles, one compress + decompress in {dt:.2f} s"}
    if reduce:
        out["sample"] += " (bit-box reduction)"
    if reorder:
        out["sample"] += " (reordered)"
    if widest:
        out["sample"] += " (widest-cell split axis)"
    return out


def run_reference(args, spec):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    gen, n, dtype, mode, eb = spec
    import oracle

    oracle.build()
    samples = [generate(gen, REF_SAMPLE, dtype, seed=s) for s in range(2)]
    for i in range(args.warmup):
        oracle_round_trip(samples[i % 2], mode, eb, args.leaf_size, args.reduce, args.reorder, widest=args.widest)
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        oracle_round_trip(samples[i % 2], mode, eb, args.leaf_size, args.reduce, args.reorder, widest=args.widest)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    units = samples[0].nbytes * args.steps
    value = units / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": args.workload, "sample_particles_per_step": REF_SAMPLE, "leaf_size": args.leaf_size,
                   "box_reduction": bool(args.reduce), "reorder": bool(args.reorder),
                   "widest_axis": bool(args.widest),
                   "note": "the oracle (plain single-threaded C, double precision) on host cores"},
        "cpu_baseline": {"value": round(value, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"{REF_SAMPLE} particles of the {gen} generator per step"},
        "e2e": {"value": round(value, 6), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, spec):
    import numpy as np
    import torch

    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as pcbuild

    gen, n, dtype, mode, eb = spec
    world, rank, local = dist_setup(args)
    if rank == 0:
        pcbuild.build()
    barrier(world)
    pc.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    st = torch.cuda.current_stream()
    pos_h = generate(gen, n, dtype, seed=rank)
    pdt = pc.PC_F32 if dtype == "f32" else pc.PC_F64
    emode = pc.PC_EB_REL if mode == "rel" else pc.PC_EB_ABS
    esz = 4 if dtype == "f32" else 8
    pos = torch.from_numpy(pos_h).to(dev)
    cfg = pc.config(args.leaf_size, autotune=args.autotune, reduce=args.reduce, reorder=args.reorder,
                    widest=args.widest)
    comp = pc.Compressor(n, pdt, leaf_size=cfg, device=dev)
    dec = torch.empty_like(pos)

    def step():
        size = comp.compress(pos, emode, eb)
        comp.decompress(comp.out, dec, size)
        return size

    size = 0
    for _ in range(max(args.warmup, 3)):
        size = step()
    torch.cuda.synchronize()
    info = pc.pc_stream_info(comp.out[:96].cpu().numpy().tobytes())
    lo = pos.amin(0).double().cpu().numpy()
    hi = pos.amax(0).double().cpu().numpy()
    qmax = int(np.rint((hi - lo) / info.s).max())
    cb = 2 if qmax < 65536 else 4

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    time.sleep(0.3)

    def timed_steps():
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
               torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(world)
        torch.cuda.synchronize()
        w0 = time.time()
        sz = 0
        for i in range(args.steps):
            ev[i][0].record(st)
            sz = comp.compress(pos, emode, eb)
            ev[i][1].record(st)
            comp.decompress(comp.out, dec, sz)
            ev[i][2].record(st)
        torch.cuda.synchronize()
        barrier(world)
        return ev, w0, time.time(), sz

    # the timed region: kernel tracing off (its two event records per launch cost ~5 % of a step)
    ev, t_wall0, t_wall1, size = timed_steps()
    time.sleep(0.1)
    sampler.stop()
    clocks = sampler.summary(t_wall0, t_wall1)
    total_ms = max_over_ranks(ev[0][0].elapsed_time(ev[-1][2]), world)
    comp_ms = max_over_ranks(sum(e[0].elapsed_time(e[1]) for e in ev), world)
    dec_ms = max_over_ranks(sum(e[1].elapsed_time(e[2]) for e in ev), world)
    nbytes = 3 * esz * n
    value = whole_job_gbs(world, nbytes, args.steps, total_ms)
    # the same steps once more with every launch bracketed by events on its stream:
    # per-kernel times for the roofline
    pc.pc_trace_reset()
    pc.pc_trace_enable(True)
    timed_steps()
    pc.pc_trace_enable(False)

    table = pc.trace_table()
    launches = int(sum(v[0] for v in table.values()))
    kernels = {k: {"launches": v[0], "ms": round(v[1], 4)} for k, v in sorted(table.items(), key=lambda kv: -kv[1][1])}
    top = max(table, key=lambda k: table[k][1])
    per_launch_ms = table[top][1] / table[top][0]
    alg = algorithmic_bytes(top, n, esz, cb, size, launches=table[top][0])
    peak, peak_kind = peaks()
    roofline = None
    if alg is not None:
        achieved = alg / (per_launch_ms / 1e3) / 1e9
        roofline = {"kernel": top, "bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                    "timing": "CUDA events around each launch, same steps traced after the timed region",
                    "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                    "traffic": measured_traffic(top, args.workload, n),
                    "algorithmic_bytes_per_launch": alg, "mean_launch_ms": round(per_launch_ms, 4)}
    # whole-step algorithmic bytes (input read + stream written + stream read + output written)
    step_alg = 2 * (nbytes + size)
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        e2e = measure_e2e(pc, pos_h, pdt, emode, eb, args, world, cfg)
    # reconstruction quality (Sec. 5.1), from one more untimed round trip with the permutation
    quality = None
    if rank == 0:
        qc = pc.Compressor(n, pdt, leaf_size=cfg, with_perm=True, device=dev)
        qsize = qc.compress(pos, emode, eb)
        qdec = torch.empty_like(pos)
        qc.decompress(qc.out, qdec, qsize)
        qinfo = pc.pc_stream_info(qc.out[:96].cpu().numpy().tobytes())
        err = (pos[qc.perm[:n].long()].double() - qdec.double()).abs()
        dmax = float((pos.double().amax(0) - pos.double().amin(0)).max())
        nrmse = float(torch.sqrt(torch.mean((err / dmax) ** 2))) if dmax > 0 else 0.0
        quality = {"max_err_over_eps": round(float(err.max()) / qinfo.eps, 6),
                   "violations": int((err > qinfo.eps).sum()), "nrmse": nrmse,
                   "psnr_db": round(-20.0 * float(np.log10(nrmse)), 3) if nrmse > 0 else None,
                   "eps": qinfo.eps, "timed": False}
        del qc, qdec, err
    lossless = None
    if rank == 0 and args.lossless:
        import zlib

        data = comp.out[:size].cpu().numpy().tobytes()
        t0 = time.perf_counter()
        z = len(zlib.compress(data, 6))
        lossless = {"codec": "zlib level 6 on the host (DEFLATE: LZ77 + Huffman)", "stream_bytes": int(size),
                    "coded_bytes": z, "ratio_over_stream": round(size / z, 4),
                    "compression_ratio_after": round(nbytes / z, 4), "seconds": round(time.perf_counter() - t0, 2),
                    "timed": False}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec, info.leaf_size if args.autotune else args.leaf_size,
                           CPU_SAMPLE // 4 if args.reduce else CPU_SAMPLE, args.reduce,
                           args.reorder, args.widest)

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras and args.workload == DEFAULT_WORKLOAD:
        del comp, dec
        torch.cuda.empty_cache()
        try:
            extras = run_extras(pc, dev, pos, args)
        except Exception as e:  # noqa: BLE001 (figures beside the line, never its failure)
            extras = {"extras_error": f"{type(e).__name__}: {e}"[:300]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload, "generator": gen, "particles": n, "eb_mode": mode, "eb": eb,
                       "leaf_size": info.leaf_size if args.autotune else args.leaf_size,
                       "autotuned_leaf_size": bool(args.autotune), "box_reduction": bool(args.reduce),
                       "reorder": bool(args.reorder), "widest_axis": bool(args.widest),
                       "parallelism": f"replicas x{world}" if world > 1 else "single",
                       "l2": "inputs larger than L2 (no flush)", "code_bytes": cb},
            "compress_gbs": round(whole_job_gbs(world, nbytes, args.steps, comp_ms), 3),
            "decompress_gbs": round(whole_job_gbs(world, nbytes, args.steps, dec_ms), 3),
            "particles_per_s": round(world * n * args.steps / (total_ms / 1e3), 1),
            "compression_ratio": round(nbytes / size, 4), "bits_per_particle": round(8 * size / n, 4),
            "step_hbm_frac_algorithmic": round(step_alg / (total_ms / args.steps / 1e3) / 1e9 / peak, 4),
            # each direction's algorithmic bytes (positions read + stream written; stream read +
            # positions written) over its own time, against the measured HBM copy bandwidth
            "compress_hbm_frac_algorithmic": round((nbytes + size) / (comp_ms / args.steps / 1e3) / 1e9 / peak, 4),
            "decompress_hbm_frac_algorithmic": round((nbytes + size) / (dec_ms / args.steps / 1e3) / 1e9 / peak, 4),
            "roofline": roofline, "kernels": kernels, "gpu_launches": launches, "clocks": clocks,
            "quality": quality, "e2e": e2e, "cpu_baseline": cpu,
        }
        if lossless:
            line["lossless"] = lossless
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def measure_e2e(pc, pos_h, pdt, emode, eb, args, world, cfg):
    """Round trips through the host-buffer entry points, copies inside the timing."""
    import torch

    n = pos_h.shape[0]
    dev = torch.cuda.current_device()
    hp = torch.from_numpy(pos_h).pin_memory()
    bound = pc.pc_compress_bound(n, pdt, cfg)
    hstream = torch.empty(bound, dtype=torch.uint8).pin_memory()
    hdec = torch.empty_like(hp).pin_memory()
    ws_c = torch.empty(pc.pc_compress_host_workspace_size(n, pdt, cfg), dtype=torch.uint8, device=dev)
    ws_d = torch.empty(pc.pc_decompress_host_workspace_size(n, pdt, bound), dtype=torch.uint8, device=dev)
    for _ in range(3):  # warm-up: the first transfers from freshly pinned pages run slower
        size = pc.pc_compress_host(hp, emode, eb, hstream, ws_c, cfg)
        pc.pc_decompress_host(hstream, size, hdec, ws_d)
    times = []
    for _ in range(args.e2e_steps):
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        size = pc.pc_compress_host(hp, emode, eb, hstream, ws_c, cfg)
        pc.pc_decompress_host(hstream, size, hdec, ws_d)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t = max_over_ranks(sum(times), world)
    value = world * hp.numel() * hp.element_size() * args.e2e_steps / t / 1e9
    out = {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": int(hp.nbytes + size),
           "d2h_bytes_per_step": int(size + hp.nbytes), "steps": args.e2e_steps,
           "api": "pc_compress_host + pc_decompress_host (pinned host buffers)"}
    # The same round trips from two host threads, each with its own stream and buffers: one
    # pipeline's copies run beside the other's kernels and its copies in the other direction.
    # A separate figure; `value` above is one round trip after another.
    try:
        out["two_pipelines"] = two_pipelines(pc, hp, emode, eb, cfg, ws_c, ws_d, hstream, hdec, args.e2e_steps,
                                             world)
    except Exception as e:  # noqa: BLE001 (a figure beside the line, never its failure)
        out["two_pipelines"] = {"unavailable": str(e)[:200]}
    del ws_c, ws_d
    return out


def two_pipelines(pc, hp, emode, eb, cfg, ws_c, ws_d, hstream, hdec, steps, world):
    """Round trips through the host-buffer entry points on two host threads at once."""
    import threading
    import torch

    dev = torch.cuda.current_device()
    sets = [(ws_c, ws_d, hstream, hdec, torch.cuda.Stream(dev)),
            (torch.empty_like(ws_c), torch.empty_like(ws_d), torch.empty_like(hstream).pin_memory(),
             torch.empty_like(hdec).pin_memory(), torch.cuda.Stream(dev))]
    errors = []

    def run(k, n_steps):
        wc, wd, hs, hd, st = sets[k]
        try:
            torch.cuda.set_device(dev)
            for _ in range(n_steps):
                size = pc.pc_compress_host(hp, emode, eb, hs, wc, cfg, stream=st)
                pc.pc_decompress_host(hs, size, hd, wd, stream=st)
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    def both(n_steps):
        th = [threading.Thread(target=run, args=(k, n_steps)) for k in range(2)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        if errors:
            raise errors[0]

    both(2)  # warm-up: the second set's freshly pinned pages
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    both(steps)
    torch.cuda.synchronize()
    t = max_over_ranks(time.perf_counter() - t0, world)
    value = world * 2 * steps * hp.numel() * hp.element_size() / t / 1e9
    return {"value": round(value, 3), "unit": "GB/s", "steps_per_pipeline": steps,
            "api": "pc_compress_host + pc_decompress_host on two host threads, one stream each"}


def direction_times(pc, pos, pdt, emode, eb, steps, warmup=3):
    """Compress and decompress GB/s (uncompressed bytes) and the compression ratio of one
    snapshot resident on the device, CUDA events on the current stream."""
    import torch

    n = pos.shape[0]
    comp = pc.Compressor(n, pdt, device=pos.device)
    dec = torch.empty_like(pos)
    st = torch.cuda.current_stream()
    size = 0
    for _ in range(warmup):
        size = comp.compress(pos, emode, eb)
        comp.decompress(comp.out, dec, size)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for e in ev:
        e[0].record(st)
        size = comp.compress(pos, emode, eb)
        e[1].record(st)
        comp.decompress(comp.out, dec, size)
        e[2].record(st)
    torch.cuda.synchronize()
    c_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
    d_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / steps
    nbytes = pos.numel() * pos.element_size()
    peak, _ = peaks()
    del comp, dec
    return {"compress_gbs": round(nbytes / c_ms / 1e6, 3), "decompress_gbs": round(nbytes / d_ms / 1e6, 3),
            "round_trip_gbs": round(nbytes / (c_ms + d_ms) / 1e6, 3), "compression_ratio": round(nbytes / size, 4),
            "compress_hbm_frac_algorithmic": round((nbytes + size) / c_ms / 1e6 / peak, 4),
            "decompress_hbm_frac_algorithmic": round((nbytes + size) / d_ms / 1e6 / peak, 4), "steps": steps}


def run_extras(pc, dev, pos, args):
    """Untimed extras of the default run (they do not enter `value`): the other bound of the
    cosmology workload on the same snapshot, the fluid workload, and compact batch-256 and
    serve-2000 summaries (the full lines come from --workload batch-256 / serve-2000)."""
    import torch

    out = {"workloads": {}}
    out["workloads"]["cosmology-2^27-f32-rel1e-3"] = direction_times(pc, pos, pc.PC_F32, pc.PC_EB_REL, 1e-3, 5)
    gen, n, dtype, mode, eb = WORKLOADS["fluid-2^24-f64-abs1e-4"]
    fl = torch.from_numpy(generate(gen, n, dtype, seed=0)).to(dev)
    out["workloads"]["fluid-2^24-f64-abs1e-4"] = direction_times(pc, fl, pc.PC_F64, pc.PC_EB_ABS, eb, 5)
    del fl
    torch.cuda.empty_cache()
    b = batch_measure(pc, dev, 1, 0, steps=2, warmup=1)
    out["batch"] = {"workload": BATCH_WORKLOAD, "snapshots": b["snapshots"], "particles": b["particles"],
                    "lanes": b["lanes"], "batched_round_trip_gbs": b["batched"]["round_trip_gbs"],
                    "one_call_per_snapshot_round_trip_gbs": b["one_call_per_snapshot"]["round_trip_gbs"],
                    "speedup_round_trip": b["speedup_round_trip"], "identical_sizes": b["identical_sizes"],
                    "compression_ratio": b["compression_ratio"], "tuning": BATCH_TUNING,
                    "tuned_knobs": b["tuned_knobs"], "steps": 2}
    torch.cuda.empty_cache()
    v = serve_measure(pc, dev, 1, 0)
    out["serve"] = {"workload": SERVE_WORKLOAD, "requests": v["requests"], "lanes": v["lanes"],
                    "p50_ms": v["served"]["p50_ms"], "p99_ms": v["served"]["p99_ms"],
                    "one_lane_p50_ms": v["one_lane"]["p50_ms"], "one_lane_p99_ms": v["one_lane"]["p99_ms"],
                    "saturated_gbs": v["saturated"]["lanes"]["gbs"],
                    "saturated_one_lane_gbs": v["saturated"]["one_lane"]["gbs"]}
    torch.cuda.empty_cache()
    return out


BATCH_WORKLOAD = "batch-256"
# leaf size and launch knobs autotuned: the one-call-per-snapshot arm runs first, so its warm-up
# tunes every class of the mix (one call at a time), and both arms then run the tuned knobs
BATCH_CFG = lambda pc: pc.config(0, autotune=True, tune_knobs=True)  # noqa: E731
BATCH_TUNING = "leaf size 64..12000 and launch knobs (threads per node 512..8192, packing tile 256..4096) per class"
SERVE_WORKLOAD = "serve-2000"
SWEEP_WORKLOAD = "leaf-sweep"


def run_sweep(args):
    """Stream size and parts against the leaf size on the default workload's data
    (one descent of the tree per error bound); prints one JSON line."""
    import torch

    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as pcbuild

    pcbuild.build()
    pc.load()
    gen, n, dtype, mode, eb0 = WORKLOADS[DEFAULT_WORKLOAD]
    pos = torch.from_numpy(generate(gen, n, dtype, seed=0)).cuda()
    out = {}
    for eb in (1e-3, 1e-4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pts = pc.pc_leaf_size_sweep(pos, pc.PC_EB_REL, eb, r_min=64, r_max=pc.PC_MAX_LEAF_SIZE)
        dt = time.perf_counter() - t0
        out[str(eb)] = {"points": pts, "seconds": round(dt, 3)}
    print(json.dumps({"metric": "stream bytes against leaf size", "workload": DEFAULT_WORKLOAD, "particles": n,
                      "sweeps": out}), flush=True)


def _pools(dev, size, gens, dtypes):
    """Device copies of one synthetic snapshot per generator and dtype; requests take slices of them."""
    import numpy as np
    import torch

    out = {}
    for g in gens:
        for dt in dtypes:
            out[(g, dt)] = torch.from_numpy(generate(g, size, dt, seed=0)).to(dev)
    return out


def knob_summary(pc):
    """What the launch-knob autotuner chose: the tuned classes and how often each value was picked."""
    classes = pc.autotune_export()
    count = lambda key: {str(v): sum(1 for c in classes if c[key] == v) for v in sorted({c[key] for c in classes})}
    return {"classes": len(classes), "warp_node_max": count("warp_node_max"), "warp_leaf_max": count("warp_leaf_max")}


def batch_measure(pc, dev, world, rank, steps, warmup):
    """Many snapshots of uneven size, dtype and bound: one pc_compress_batch (and
    pc_decompress_batch) call against one plain call per snapshot."""
    import numpy as np
    import torch

    rng = np.random.default_rng(rank)
    pool_n = 1 << 24
    pools = _pools(dev, pool_n, ("cosmology", "fluid"), ("f32", "f64"))
    jobs = []
    for _ in range(256):
        n = int(round(10 ** rng.uniform(4, 7)))
        g = "cosmology" if rng.random() < 0.5 else "fluid"
        dt = "f32" if rng.random() < 0.5 else "f64"
        eb = float(rng.choice([1e-2, 1e-3, 1e-4]))
        off = int(rng.integers(0, pool_n - n + 1))
        jobs.append((pools[(g, dt)][off: off + n], pc.PC_EB_REL, eb, BATCH_CFG(pc)))
    dtype_of = lambda t: pc.PC_F32 if t.dtype == torch.float32 else pc.PC_F64
    outs = [torch.empty(pc.pc_compress_bound(p.shape[0], dtype_of(p), leaf), dtype=torch.uint8, device=dev)
            for p, _, _, leaf in jobs]
    lanes = 16  # measured on the batch-256 mix: 111.5 GB/s round trip against 105.2 with 8 and 109.0 with 12
    ws = torch.empty(pc.pc_compress_batch_workspace_size([(p.shape[0], dtype_of(p), leaf) for p, _, _, leaf in jobs],
                                                         lanes), dtype=torch.uint8, device=dev)
    decs = [torch.empty_like(p) for p, _, _, _ in jobs]
    nbytes = sum(p.numel() * p.element_size() for p, _, _, _ in jobs)
    particles = sum(p.shape[0] for p, _, _, _ in jobs)

    def batched():
        sizes, st = pc.pc_compress_batch(jobs, outs, workspace=ws, lanes=lanes)
        assert all(x == pc.PC_OK for x in st)
        t1 = time.perf_counter()
        st = pc.pc_decompress_batch(outs, sizes, decs, lanes=lanes)
        assert all(x == pc.PC_OK for x in st)
        return sizes, t1

    big = max(jobs, key=lambda j: j[0].shape[0])[0]
    seq = pc.Compressor(big.shape[0], pc.PC_F64, leaf_size=BATCH_CFG(pc), device=dev)

    def sequential():
        sizes = []
        for (p, m, eb, leaf), o in zip(jobs, outs):
            sizes.append(pc.pc_compress(p, m, eb, o, seq.ws, leaf))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for o, sz, d in zip(outs, sizes, decs):
            pc.pc_decompress(o, d, seq.dws, sz)
        return sizes, t1

    results = {}
    for name, fn in (("sequential", sequential), ("batched", batched)):
        for _ in range(max(warmup, 1)):
            fn()
        tc = td = 0.0
        for _ in range(steps):
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sizes, t1 = fn()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            tc += t1 - t0
            td += t2 - t1
        tc = max_over_ranks(tc, world)
        td = max_over_ranks(td, world)
        results[name] = {"compress_gbs": round(whole_job_gbs(world, nbytes, steps, 1e3 * tc), 3),
                         "decompress_gbs": round(whole_job_gbs(world, nbytes, steps, 1e3 * td), 3),
                         "round_trip_gbs": round(whole_job_gbs(world, nbytes, steps, 1e3 * (tc + td)), 3),
                         "ms_per_batch": round(1e3 * (tc + td) / steps, 3)}
        results[name + "_sizes"] = sizes
    b, q = results["batched"], results["sequential"]
    out = {"snapshots": len(jobs), "particles": particles, "lanes": lanes, "batched": b, "one_call_per_snapshot": q,
           "tuned_knobs": knob_summary(pc),
           "speedup_round_trip": round(b["round_trip_gbs"] / q["round_trip_gbs"], 3),
           # the batched streams are the plain calls' streams
           "identical_sizes": bool(results["batched_sizes"] == results["sequential_sizes"]),
           "compression_ratio": round(nbytes / sum(results["batched_sizes"]), 4)}
    del pools, jobs, outs, ws, decs, seq
    return out


def run_batch(args):
    import torch

    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as pcbuild

    world, rank, local = dist_setup(args)
    if rank == 0:
        pcbuild.build()
    barrier(world)
    pc.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    r = batch_measure(pc, dev, world, rank, args.steps, args.warmup)
    if rank == 0:
        b = r["batched"]
        line = {
            "metric": "batched compress+decompress throughput (uncompressed bytes)", "value": b["round_trip_gbs"],
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 1),
            "ms_per_step": b["ms_per_batch"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "snapshots": r["snapshots"], "particles": r["particles"],
                       "sizes": "round(10^U(4,7))", "generators": "cosmology or fluid slices, p = 1/2",
                       "eb": "rel, one of 1e-2 1e-3 1e-4", "tuning": BATCH_TUNING, "lanes": r["lanes"],
                       "parallelism": f"replicas x{world}" if world > 1 else "single"},
            "batched": b, "one_call_per_snapshot": r["one_call_per_snapshot"],
            "speedup_round_trip": r["speedup_round_trip"], "identical_sizes": r["identical_sizes"],
            "compression_ratio": r["compression_ratio"], "tuned_knobs": r["tuned_knobs"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def serve_measure(pc, dev, world, rank, lanes_list=(8, 1)):
    """Poisson arrivals of compress (70 %) and decompress (30 %) requests through
    the library's serving loop; latency from submission to completion.  The
    same trace also runs saturated (every request submitted at once), where the
    overlap of several lanes shows as throughput."""
    import numpy as np
    import torch

    rng = np.random.default_rng(rank)
    pool_n = 50_000_000
    pool = torch.from_numpy(generate("cosmology", pool_n, "f32", seed=0)).to(dev)
    count, rate = 2000, 200.0
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    kinds = rng.random(count) < 0.7
    sizes = np.round(10 ** rng.uniform(5, np.log10(5e7), count)).astype(np.int64)
    ebs = rng.choice([1e-3, 1e-4], count)
    offs = [int(rng.integers(0, pool_n - n + 1)) for n in sizes]
    arena = torch.empty(40 << 30, dtype=torch.uint8, device=dev)
    report = {}
    runs = [(lanes, 1.0) for lanes in lanes_list] + [(lanes, 0.0) for lanes in lanes_list]
    for lanes, stretch in runs:
        srv = pc.Server(arena, lanes=lanes)
        kept = []  # completed compress outputs kept for decompress requests: (completion, n)
        busy = {}  # tag -> kept entry a decompress request reads
        lat, done_bytes, t_first, t_last = [], 0, None, None
        submitted = completed = 0
        t0 = pc.Server.now() + 0.2
        while completed < count:
            now = pc.Server.now()
            while submitted < count and t0 + stretch * arrivals[submitted] <= now:
                i = submitted
                if kinds[i] or not kept:
                    n = int(sizes[i])
                    srv.submit_compress(pool[offs[i]: offs[i] + n], pc.PC_EB_REL, float(ebs[i]), tag=i)
                else:
                    k = kept[int(rng.integers(0, len(kept)))]
                    busy[i] = k
                    k[2] += 1
                    srv.submit_decompress(srv.output(k[0]), k[0].output_bytes, k[1], pc.PC_F32, tag=i)
                submitted += 1
            cs = srv.poll(wait=False)
            for c in cs:
                assert c.status == pc.PC_OK, (c.tag, c.status)
                completed += 1
                lat.append(c.t_done - c.t_submit)
                t_first = c.t_submit if t_first is None else min(t_first, c.t_submit)
                t_last = c.t_done if t_last is None else max(t_last, c.t_done)
                if c.kind == pc.PC_REQ_COMPRESS:
                    done_bytes += int(sizes[c.tag]) * 12
                    kept.append([c, int(sizes[c.tag]), 0])
                    while len(kept) > 16 and kept[0][2] == 0:
                        srv.release(kept.pop(0)[0])
                else:
                    k = busy.pop(c.tag)
                    done_bytes += k[1] * 12
                    k[2] -= 1
                    srv.release(c)
            if not cs:
                time.sleep(0.0002)
        for k in kept:
            srv.release(k[0])
        srv.close()
        lat_ms = np.array(lat) * 1e3
        report[(lanes, stretch)] = {"p50_ms": round(float(np.percentile(lat_ms, 50)), 3),
                         "p99_ms": round(float(np.percentile(lat_ms, 99)), 3),
                         "mean_ms": round(float(lat_ms.mean()), 3),
                         "gbs": round(done_bytes / (t_last - t_first) / 1e9, 3)}
    del arena, pool
    return {"requests": count, "lanes": lanes_list[0], "served": report[(lanes_list[0], 1.0)],
            "one_lane": report[(lanes_list[-1], 1.0)],
            "saturated": {"lanes": report[(lanes_list[0], 0.0)], "one_lane": report[(lanes_list[-1], 0.0)],
                          "note": "all requests submitted at once"}}


def run_serve(args):
    import torch

    import paper_2404_02826_gb300 as pc
    from paper_2404_02826_gb300 import build as pcbuild

    world, rank, local = dist_setup(args)
    if rank == 0:
        pcbuild.build()
    barrier(world)
    pc.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    r = serve_measure(pc, dev, world, rank)
    if rank == 0:
        best = r["served"]
        line = {
            "metric": "served compress/decompress latency p99 (arrival to completion)", "value": best["p99_ms"],
            "unit": "ms", "n_gpus": world, "steps": r["requests"], "warmup": 0, "ms_per_step": best["mean_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": SERVE_WORKLOAD, "requests": r["requests"], "arrivals": "Poisson, 200 per s",
                       "mix": "70 % compress, 30 % decompress of a completed stream",
                       "sizes": "round(10^U(5, log10 5e7)) particles, slices of one cosmology snapshot",
                       "eb": "rel 1e-3 or 1e-4", "arena_bytes": 40 << 30, "lanes": r["lanes"]},
            "served": best, "one_lane": r["one_lane"], "saturated": r["saturated"],
            "p50_ms": best["p50_ms"], "p99_ms": best["p99_ms"], "throughput_gbs": best["gbs"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def main():
    args = parse()
    if args.workload == BATCH_WORKLOAD:
        run_batch(args)
        return
    if args.workload == SERVE_WORKLOAD:
        run_serve(args)
        return
    if args.workload == SWEEP_WORKLOAD:
        run_sweep(args)
        return
    spec = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, spec)
    else:
        run_ours(args, spec)


if __name__ == "__main__":
    main()
