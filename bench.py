#!/usr/bin/env python
"""Throughput benchmark of the GB300 compressor.

Headline workload (default): two 512^3 float32 fields, a positive log-normal
density exp(1.5 G), G with power spectrum k^-2, and a signed velocity-like
Gaussian random field with spectrum k^-4; eb_rel = 1e-4; 8x8x8 blocks; a
perceptron over the 13-point causal stencil with hidden widths 32/32, trained
on the device from 2^20 sampled stencils per field, evaluated in its
fixed-point (bf16 tensor-core) form, with the Lorenzo predictor as per-block
fallback.  Both fields together (1.07 GB) are larger than L2.

One step = pc_compress of both fields + pc_decompress of both containers (the
whole hot path: statistics, constants, transform, prediction, selection,
quantization, histogram, codebook, packing, and the inverse path).

Secondary workloads (reported inside the same JSON line unless
--no-secondary): 100x500x500 float32 at eb_rel 1e-3 with the FP32 and the
fixed-point 7-point 16/16 perceptron; 256x384x384 float64 at eb_rel 1e-5
(fixed-point 16/16 perceptron, float64 transform); 64^3 float32 at eb_rel 1e-2
with the FP32 perceptron trained by the oracle.

All fields are seeded synthetic Gaussian random fields standing in for the
paper's SEG-Y seismic volumes.  Prints one JSON line (rank 0).
`--impl reference` times the CPU oracle (the reference arm: no reference code
exists beyond the paper) on bounded samples of the same workload.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "compress/decompress GB/s and bits/value at eb_rel, % of HBM roofline, vs FP32 plain"
BLOCK = (8, 8, 8)

# name -> workload description
WORKLOADS = {
    "density_velocity_512": dict(desc="two 512^3 float32 fields: positive log-normal density exp(1.5 G), G ~ k^-2, "
                                      "and a signed velocity-like GRF ~ k^-4", eb=1e-4, k=13, h1=32, h2=32,
                                 samples=1 << 20, form="bf16", dtype="f32", train="device"),
    "grf100x500x500_f32": dict(desc="100x500x500 float32 signed log-normal GRF, k^-11/3, 2% zeros", eb=1e-3, k=7,
                               h1=16, h2=16, samples=None, form="fp32", dtype="f32", train="device"),
    "grf256x384x384_f64": dict(desc="256x384x384 float64 GRF k^-3, magnitudes 1e-8..1e8, mixed sign, 1% zeros",
                               eb=1e-5, k=7, h1=16, h2=16, samples=None, form="bf16", dtype="f64", train="device"),
    "grf64_f32": dict(desc="64^3 float32 signed log-normal GRF, k^-3, 5% zeros", eb=1e-2, k=7, h1=16, h2=16,
                      samples=None, form="fp32", dtype="f32", train="oracle"),
}
HEADLINE = "density_velocity_512"
THR10 = int(0.1 * 2 ** 32)  # 10% of points drawn for training (Section IV.C)


def make_fields(name: str, device):
    """The workload's fields as device tensors (seeded)."""
    import torch
    from paper_2309_09778_gb300 import gen
    if name == "density_velocity_512":
        return list(gen.density_velocity_pair((512, 512, 512), device))
    if name == "grf100x500x500_f32":
        return [torch.from_numpy(gen.signed_lognormal((100, 500, 500), 11.0 / 3.0, 0, 2.0, 0.02)).to(device)]
    if name == "grf256x384x384_f64":
        return [gen.wide_range_device((256, 384, 384), 3.0, 0, device, 8.0, 0.01)]
    if name == "grf64_f32":
        return [torch.from_numpy(gen.signed_lognormal((64, 64, 64), 3.0, 0, 2.0, 0.05)).to(device)]
    raise KeyError(name)


def thr_for(shape, samples):
    """Sampling threshold (of 2^32) for an expected count of `samples` non-anchor points, else 10%."""
    if not samples:
        return THR10
    n = int(np.prod(shape))
    nb = int(np.prod([-(-s // b) for s, b in zip(shape, BLOCK)]))
    return min(int(round(samples / (n - nb) * 2 ** 32)), 2 ** 32 - 1)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms (read only)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (the cpu_baseline leg and the reference arm).  Workers are
# spawned, never forked, so that no child inherits a CUDA context.
# ---------------------------------------------------------------------------
def oracle_worker(args):
    sub, eb, k, h1, h2, s_in, w, q = args
    from oracle import oracle as O
    O.build()
    t0 = time.perf_counter()
    st, blob = O.compress(sub, eb, block=BLOCK, weights=w, stencil=k, h1=h1, h2=h2, s_in=s_in, qnet=q)
    st2, y = O.decompress(blob)
    dt = time.perf_counter() - t0
    if st != 0 or st2 != 0:
        raise RuntimeError(f"oracle status {st}/{st2}")
    return sub.nbytes, dt, len(blob)


def report_worker(args):
    """One field sample: the oracle's prediction report, or its container size with one predictor form."""
    kind, sub, eb, k, h1, h2, s_in, w, q = args
    from oracle import oracle as O
    O.build()
    if kind == "report":
        return kind, O.pred_report(sub, eb, w, s_in, block=BLOCK, k=k, h1=h1, h2=h2, qnet=q)
    st, blob = O.compress(sub, eb, block=BLOCK, weights=w, stencil=k, h1=h1, h2=h2, s_in=s_in,
                          qnet=q if kind == "bf16" else None, fp64=kind == "fp64")
    if st != 0:
        raise RuntimeError(f"oracle status {st}")
    return kind, 8.0 * len(blob) / sub.size


def fp64_report(fields_host, spec, infos, cores, pts):
    """Prediction error and compression ratio of the FP32 and fixed-point forms against the same trained
    weights evaluated in FP64 (the reporting predictor), by the oracle on one sub-volume per field."""
    eb, k, h1, h2 = spec["eb"], spec["k"], spec["h1"], spec["h2"]
    tasks, idx = [], []
    for fi, (x, inf) in enumerate(zip(fields_host, infos)):
        if inf["w"] is None:
            continue
        sub = slabs([x], pts, 1)[0]
        for kind in ("report", "fp64", "fp32", "bf16"):
            if kind == "bf16" and inf["q"] is None:
                continue
            tasks.append((kind, sub, eb, k, h1, h2, inf["s_in"], inf["w"], inf["q"]))
            idx.append(fi)
    if not tasks:
        return None
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(min(cores, len(tasks))) as pool:
        res = pool.map(report_worker, tasks)
    out = {}
    for fi, (kind, v) in zip(idx, res):
        d = out.setdefault(fi, {"bits_per_value": {}})
        if kind == "report":
            d.update(v)
        else:
            d["bits_per_value"][kind] = v
    for d in out.values():
        b = d["bits_per_value"]
        d["size_vs_fp64"] = {f: b[f] / b["fp64"] - 1.0 for f in ("fp32", "bf16") if f in b and "fp64" in b}
    shp = slabs([fields_host[0]], pts, 1)[0].shape
    return {"sample": f"one {shp[0]}x{shp[1]}x{shp[2]} corner sub-volume per field, the device-trained weights",
            "seconds": time.perf_counter() - t0, "fields": [out[i] for i in sorted(out)]}


def slabs(fields_host, pts_per_slab, count):
    """`count` distinct corner-aligned sub-volumes of about pts_per_slab points, drawn round-robin from the fields."""
    out = []
    for i in range(count):
        x = fields_host[i % len(fields_host)]
        Z, Y, X = x.shape
        sy, sx = min(Y, 128), min(X, 128)
        dz = max(8, min(Z, (pts_per_slab // (sy * sx)) // 8 * 8))
        j = i // len(fields_host)
        z0 = (j * dz) % max(1, Z - dz + 1)
        out.append(np.ascontiguousarray(x[z0: z0 + dz, :sy, :sx]))
    return out


def oracle_rate(fields_host, spec, pred, cores: int, pts_per_slab: int, rounds: int = 1):
    """Oracle compress + decompress on `cores` slabs at once (one process per core), `rounds` times.
    Returns (GB/s of input, per-round seconds, description)."""
    eb, k, h1, h2 = spec["eb"], spec["k"], spec["h1"], spec["h2"]
    s_in, w, q = pred
    subs = slabs(fields_host, pts_per_slab, cores * rounds)
    work = [(s, eb, k, h1, h2, s_in, w, q) for s in subs]
    ctx = mp.get_context("spawn")
    t_round = []
    nbytes = 0
    with ctx.Pool(cores) as pool:
        # warm the workers (library load, page-in) on tiny sub-volumes
        tiny = [(np.ascontiguousarray(subs[0][:8, :16, :16]),) + w[1:] for w in work[:cores]]
        pool.map(oracle_worker, tiny)
        for r in range(rounds):
            t0 = time.perf_counter()
            res = pool.map(oracle_worker, work[r * cores:(r + 1) * cores])
            t_round.append(time.perf_counter() - t0)
            nbytes += sum(b for b, _, _ in res)
    shp = subs[0].shape
    desc = (f"{cores} process(es) x 1 sub-volume {shp[0]}x{shp[1]}x{shp[2]} of the workload fields per round, "
            f"{rounds} round(s), compress + decompress with the device-chosen predictor")
    return nbytes / sum(t_round) / 1e9, t_round, desc


# ---------------------------------------------------------------------------
# Device side.
# ---------------------------------------------------------------------------
def sha_of(*paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# DRAM bytes (read + write) per launch of a kernel, from an ncu capture of the
# kernel on the named workload and form; each entry carries the hash of the
# sources it was captured from and is dropped (traffic null) once they change.
TRAFFIC = {
    # (workload, stage, form): (bytes per launch, sha of the sources, profile summary)
    # captured on 256 x 256 x 512 (one quarter of a 512^3 field, same recipe and network shape) and scaled by
    # the points processed: 69.1 MB read + 74.9 MB written there
    ("density_velocity_512", "recon", "bf16"): (4 * (69058304 + 74940928), "75ff1fa4048c60e2",
                                                "profiles/k_recon_c3_wmma.md"),
    # 134.8 MB read + 38.2 MB written on the same quarter-size case
    ("density_velocity_512", "compress", "bf16"): (4 * (134845440 + 38154496), "5558dd42ecd8e777",
                                                   "profiles/k_compress_c3_tcgen05.md"),
    # captured on 128 x 384 x 384 (one half of the float64 field, same recipe): 151.8 MB read + 23.0 MB written
    ("grf256x384x384_f64", "compress", "bf16"): (2 * (151760128 + 22973952), "5558dd42ecd8e777",
                                                 "profiles/k_compress_c5_f64.md"),
}
STAGE_SOURCES = {
    "compress": ("paper_2309_09778_gb300/csrc/pc_compress.cu", "paper_2309_09778_gb300/csrc/pc_tcnet.cuh",
                 "paper_2309_09778_gb300/csrc/pc_tc.cuh", "paper_2309_09778_gb300/csrc/pc_qmlp.cuh",
                 "paper_2309_09778_gb300/csrc/pc_device.cuh", "paper_2309_09778_gb300/csrc/pc_kernels.cuh"),
    "recon": ("paper_2309_09778_gb300/csrc/pc_decompress.cu", "paper_2309_09778_gb300/csrc/pc_tcnet.cuh",
              "paper_2309_09778_gb300/csrc/pc_qmlp.cuh", "paper_2309_09778_gb300/csrc/pc_device.cuh",
              "paper_2309_09778_gb300/csrc/pc_kernels.cuh"),
}
# kernels behind each profiled stage (the codebook stage launches k_codebook and k_cb_assign; the decoder's
# scan stage k_dec_chunksum, k_dec_chunkscan and k_dec_blockoff)
KERNELS_PER_STAGE = {"codebook": 2, "dec_scan": 3}


def traffic_for(workload, stage, form):
    e = TRAFFIC.get((workload, stage, form))
    if not e or stage not in STAGE_SOURCES:
        return None
    return e[0] if sha_of(*STAGE_SOURCES[stage]) == e[1] else None


def net_flops(k, h1, h2, form):
    """Algorithmic flops of one forward pass: 2 per multiply-add; the fixed-point form multiplies
    every weight by two 8-bit limbs of its input."""
    macs = k * h1 + (h1 * h2 + h2 if h2 else h1)
    return 2 * macs * (2 if form == "bf16" else 1)


def block_census(blob: bytes, shape):
    """Per block: perceptron flag and the points that are neither anchor nor balance point."""
    import struct
    _, off_bb, off_bn, _, _ = struct.unpack_from("<5Q", blob, 176)
    nb = [-(-s // b) for s, b in zip(shape, BLOCK)]
    nblocks = nb[0] * nb[1] * nb[2]
    flags = np.frombuffer(blob, "<u4", nblocks, off_bb) >> 31
    nout = np.frombuffer(blob, "<u2", nblocks, off_bn).astype(np.int64)
    ext = [np.minimum(b, s - np.arange(n) * b) for s, b, n in zip(shape, BLOCK, nb)]
    pts = (ext[0][:, None, None] * ext[1][None, :, None] * ext[2][None, None, :]).reshape(-1)
    return flags.astype(bool), pts - nout


def train_predictors(torch, pc, fields, spec, dev):
    """Training phase per field (Section IV.C): on the device (or by the oracle), then the fixed-point
    form of the chosen network.  Returns one dict per field."""
    out = []
    k, h1, h2, eb = spec["k"], spec["h1"], spec["h2"], spec["eb"]
    lrs, lams = pc.default_grid()
    for d in fields:
        shape = tuple(d.shape)
        dt = pc.PC_F32 if d.dtype == torch.float32 else pc.PC_F64
        thr32 = thr_for(shape, spec["samples"])
        tp = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2))
        ws = torch.empty(pc.pc_train_workspace_size(shape, dt, tp, thr32, lrs.size), dtype=torch.uint8, device=dev)
        info = {"thr32": thr32, "samples_expected": thr32 / 2 ** 32 * (d.numel() - d.numel() // 512)}
        if spec["train"] == "oracle":
            from oracle import oracle as O
            x = d.cpu().numpy()
            t0 = time.perf_counter()
            chosen, W, s_in, costs = O.train(x, eb, block=BLOCK, k=k, h1=h1, h2=h2, seed=0, thr32=thr32)
            info["train_s"] = time.perf_counter() - t0
            info["trained_by"] = "oracle"
        else:
            pc.pc_train(d, tp, 0, thr32, lrs, lams, ws)  # warm-up (module load, first launches)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            W, s_in, chosen, costs = pc.pc_train(d, tp, 0, thr32, lrs, lams, ws)
            torch.cuda.synchronize()
            info["train_s"] = time.perf_counter() - t0
            info["trained_by"] = "device"
        info.update(chosen=int(chosen), s_in=int(s_in), val_costs=[int(c) for c in costs])
        w = W[chosen] if chosen >= 0 else None
        info["w"] = w
        info["q"] = None
        info["quant_s"] = None
        if w is not None:
            p32 = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2), s_in=s_in,
                                 weights=w)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info["q"] = pc.pc_quantize(d, p32, 0, thr32, ws)
            torch.cuda.synchronize()
            info["quant_s"] = time.perf_counter() - t0
        del ws
        out.append(info)
    return out


def params_for(pc, spec, info, form, codebook=None):
    eb, k, h1, h2 = spec["eb"], spec["k"], spec["h1"], spec["h2"]
    cb = dict(codebook=codebook)
    if info["w"] is None or form == "lorenzo":
        return pc.make_params(eb, BLOCK, **cb), "lorenzo"
    if form == "bf16":
        return pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_BF16, stencil=k, hidden=(h1, h2), s_in=info["s_in"],
                              qnet=info["q"], **cb), f"mlp_bf16_fixed_point_s{k}_{h1}x{h2}"
    return pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2), s_in=info["s_in"],
                          weights=info["w"], **cb), f"mlp_fp32_s{k}_{h1}x{h2}"


class Runner:
    """Buffers for compressing every field and decompressing every container of one workload."""

    def __init__(self, torch, pc, fields, params, dev):
        self.torch, self.pc, self.fields, self.params = torch, pc, fields, params
        self.dt = [pc.PC_F32 if d.dtype == torch.float32 else pc.PC_F64 for d in fields]
        self.out = [torch.empty(pc.pc_compress_bound(tuple(d.shape), t, p), dtype=torch.uint8, device=dev)
                    for d, t, p in zip(fields, self.dt, params)]
        self.wsc = [torch.empty(pc.pc_compress_workspace_size(tuple(d.shape), t, p), dtype=torch.uint8, device=dev)
                    for d, t, p in zip(fields, self.dt, params)]
        self.y = [torch.empty_like(d) for d in fields]
        self.size = [self.compress(i) for i in range(len(fields))]
        self.wsd = []
        for o in self.out:
            _, _, wsb = pc.pc_header_info(o[:256].cpu().numpy().tobytes())
            self.wsd.append(torch.empty(max(wsb, 1), dtype=torch.uint8, device=dev))

    def compress(self, i, stream=None):
        return self.pc.pc_compress(self.fields[i], self.params[i], self.out[i], self.wsc[i], stream)

    def decompress(self, i, stream=None):
        self.pc.pc_decompress(self.out[i], self.size[i], self.y[i], self.wsd[i], stream)

    def step(self, stream, ev):
        torch = self.torch
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        for i in range(len(self.fields)):
            self.size[i] = self.compress(i, stream)
        e[1].record(stream)
        for i in range(len(self.fields)):
            self.decompress(i, stream)
        e[2].record(stream)
        ev.append(e)

    def bound_held(self, eb):
        ok = True
        for d, y in zip(self.fields, self.y):
            ok &= bool(((y.double() - d.double()).abs() <= eb * d.double().abs()).all().item())
        return ok

    def free(self):
        self.out = self.wsc = self.y = self.wsd = None


def rank_max(torch, dist, values, device):
    """Replicas (one per GPU, the same step each): the job's times are the slowest rank's."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(world, bytes_per_rank, ms_per_step):
    """Whole-job throughput in GB/s: every rank's bytes over the slowest rank's step time."""
    return world * bytes_per_rank / (ms_per_step * 1e6)


def measure(torch, pc, fields, spec, params, steps, warmup, stream, flush, dist=None):
    """Warm-up, bound check, then `steps` timed steps (CUDA events on the launching stream, L2 flushed
    between steps).  Returns (result dict, runner)."""
    r = Runner(torch, pc, fields, params, fields[0].device)
    for _ in range(warmup):
        flush.zero_()
        r.step(stream, [])
    torch.cuda.synchronize()
    ok = r.bound_held(spec["eb"])
    pc.pc_profile_enable(True)
    pc.pc_profile_read()
    ev = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        flush.zero_()
        r.step(stream, ev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t0
    prof = pc.pc_profile_read()
    pc.pc_profile_enable(False)
    tc = sum(a.elapsed_time(b) for a, b, _ in ev) / len(ev)
    td = sum(b.elapsed_time(c) for _, b, c in ev) / len(ev)
    if dist:
        tc, td = rank_max(torch, dist, [tc, td], fields[0].device)
    nbytes = sum(d.numel() * d.element_size() for d in fields)
    npts = sum(d.numel() for d in fields)
    out_bytes = sum(r.size)
    stages = {k: (v[0] / steps, v[1] / steps) for k, v in prof.items() if v[1] > 0}
    res = {"compress_ms": tc, "decompress_ms": td, "ms_per_step": tc + td, "input_bytes": nbytes, "points": npts,
           "compressed_bytes": out_bytes, "bits_per_value": 8.0 * out_bytes / npts, "bound_held": ok,
           "compress_gbs": nbytes / (tc * 1e6), "decompress_gbs": nbytes / (td * 1e6),
           "stages_ms_per_step": {k: v[0] for k, v in stages.items()},
           "launches_per_step": sum(v[1] * KERNELS_PER_STAGE.get(k, 1) for k, v in stages.items()),
           "stage_launches_per_step": {k: v[1] for k, v in stages.items()}, "wall_s_timed": wall}
    return res, r


def hbm_fractions(res, peak):
    """Whole-step HBM roofline: compress must read the field twice (the global extrema come before any
    transform) and write the container; decompress reads the container and writes the field."""
    n, out, tc, td = res["input_bytes"], res["compressed_bytes"], res["compress_ms"], res["decompress_ms"]
    c = (2 * n + out) / (tc * 1e6)
    c1 = (n + out) / (tc * 1e6)
    d = (out + n) / (td * 1e6)
    return {"peak_gbs": peak["hbm_gbs"], "peak_source": peak["source"],
            "compress": {"algorithmic_bytes": 2 * n + out, "achieved_gbs": c, "frac": c / peak["hbm_gbs"],
                         "single_read_frac": c1 / peak["hbm_gbs"]},
            "decompress": {"algorithmic_bytes": out + n, "achieved_gbs": d, "frac": d / peak["hbm_gbs"]}}


# FP64 flops of the float64 transform per point (Eq. 6, 7 and the bound check), 2 per fused multiply-add:
# log2 (m - 1, m + 1, the quotient, s^2, 10 fma, two products, the exponent's sum) = 27; the code's product
# and its inverse's product = 2; exp2 (t - n, times ln 2, 13 fma, three power-of-two scalings) = 31; the error
# and its bound = 2.  The inverse transform of a coded point is its product and exp2: 32.
F64_FLOPS_TRANSFORM = 62
F64_FLOPS_INVERSE = 32
# the FP64 rate of the part (nominal; no measured figure exists for it)
F64_PEAK_TFLOPS = 1.25


def stage_roofline(workload, stage, ms, res, spec, form, nn_pts, nsm, sm_mhz, peak, coded_pts=0):
    """The dominant stage against its bounding roof, from its algorithmic work per launch."""
    n_pts = res["points"]
    ts = res["input_bytes"] // n_pts
    nf = len(spec.get("_fields", [])) or 1
    if ts == 8 and stage in ("compress", "recon"):
        # the float64 transform on the narrow FP64 pipe binds these stages; coded points are those that are
        # neither a block's anchor nor a stored balance point
        flops = (F64_FLOPS_TRANSFORM * n_pts if stage == "compress" else F64_FLOPS_INVERSE * coded_pts) / nf
        a = flops / (ms * 1e-3) / 1e12
        return {"kernel": stage, "bound": "alu", "achieved": a, "peak": F64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": a / F64_PEAK_TFLOPS, "traffic": traffic_for(workload, stage, form),
                "peak_source": "nominal FP64 rate of the part (1.25 TFLOP/s dense); no measured FP64 peak",
                "algorithmic_flops_per_launch": flops, "avg_launch_ms": ms}
    if stage in ("compress", "recon") and form in ("fp32", "bf16"):
        pts = nn_pts if stage == "recon" else n_pts
        flops = net_flops(spec["k"], spec["h1"], spec["h2"], form) * pts / nf
        a = flops / (ms * 1e-3) / 1e12
        if form == "fp32":
            pk = nsm * 128 * 2 * sm_mhz * 1e6 / 1e12
            src = f"derived: {nsm} SMs x 128 FP32 lanes x 2 flop x {sm_mhz:.0f} MHz"
            bound = "alu"
        else:
            pk = peak["bf16_tflops_sustained"]
            src = f"{peak['source']} bf16 dense, sustained"
            bound = "tensor"
        return {"kernel": stage, "bound": bound, "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk,
                "traffic": traffic_for(workload, stage, form), "peak_source": src,
                "algorithmic_flops_per_launch": flops, "avg_launch_ms": ms}
    alg = {"stats": ts * n_pts, "compress": ts * n_pts + 2 * n_pts, "pack": 2 * n_pts + res["compressed_bytes"],
           "huff_decode": res["compressed_bytes"] + 2 * n_pts, "recon": 2 * n_pts + ts * n_pts}.get(stage, 0) / nf
    a = alg / (ms * 1e6) if alg else None
    return {"kernel": stage, "bound": "hbm", "achieved": a, "peak": peak["hbm_gbs"], "unit": "GB/s",
            "frac": (a / peak["hbm_gbs"]) if a else None, "traffic": traffic_for(workload, stage, form),
            "peak_source": peak["source"], "algorithmic_bytes_per_launch": alg, "avg_launch_ms": ms}


def e2e_rate(torch, pc, r, steps):
    """The user's call with HOST buffers: pc_compress_host + pc_decompress_host of every field, pinned host
    memory, host<->device copies inside the timed region."""
    hosts = [d.cpu().pin_memory() for d in r.fields]
    outs = [torch.empty(o.numel(), dtype=torch.uint8).pin_memory() for o in r.out]
    ys = [torch.empty_like(h).pin_memory() for h in hosts]
    stage = [torch.empty_like(d) for d in r.fields]
    hf = [h.numpy() for h in hosts]
    ho = [o.numpy() for o in outs]
    hy = [y.numpy() for y in ys]
    t = []
    sizes = [0] * len(hf)
    for it in range(2 + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(len(hf)):
            sizes[i] = pc.pc_compress_host(hf[i], r.params[i], ho[i], stage[i], r.out[i], r.wsc[i])
            pc.pc_decompress_host(ho[i], sizes[i], hy[i], r.out[i], stage[i], r.wsd[i])
        if it >= 2:
            t.append(time.perf_counter() - t0)
    same = all(np.array_equal(hy[i].view(np.uint8), r.y[i].cpu().numpy().view(np.uint8)) for i in range(len(hf)))
    nbytes = sum(h.nbytes for h in hf)
    return {"value": nbytes / statistics.median(t) / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": nbytes + sum(sizes), "d2h_bytes_per_step": sum(sizes) + nbytes,
            "matches_device_path": bool(same)}, hosts


def e2e_with_training(torch, pc, hosts, spec, form, dev):
    """The whole user path from host memory, the learned part included: host->device copy, device training,
    the fixed-point form (bf16), compression, container to host, then host-buffer decompression."""
    k, h1, h2, eb = spec["k"], spec["h1"], spec["h2"], spec["eb"]
    lrs, lams = pc.default_grid()
    bufs = []
    for h in hosts:
        shape = tuple(h.shape)
        dt = pc.PC_F32 if h.dtype == torch.float32 else pc.PC_F64
        thr32 = thr_for(shape, spec["samples"])
        tp = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2))
        pmax = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2), s_in=0,
                              weights=np.zeros(pc.pc_mlp_nweights(k, h1, h2), np.float32))
        bufs.append(dict(
            d=torch.empty(shape, dtype=h.dtype, device=dev), thr32=thr32, tp=tp,
            wst=torch.empty(pc.pc_train_workspace_size(shape, dt, tp, thr32, lrs.size), dtype=torch.uint8, device=dev),
            out=torch.empty(pc.pc_compress_bound(shape, dt, pmax) + 65536, dtype=torch.uint8, device=dev),
            wsc=torch.empty(pc.pc_compress_workspace_size(shape, dt, pmax), dtype=torch.uint8, device=dev),
            ho=torch.empty(pc.pc_compress_bound(shape, dt, pmax) + 65536, dtype=torch.uint8).pin_memory(),
            hy=torch.empty_like(h).pin_memory()))
    t = []
    for it in range(4):  # one untimed pass, then the best of three
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for h, b in zip(hosts, bufs):
            b["d"].copy_(h, non_blocking=True)
            W, s_in, chosen, _ = pc.pc_train(b["d"], b["tp"], 0, b["thr32"], lrs, lams, b["wst"])
            if chosen < 0:
                p = pc.make_params(eb, BLOCK)
            else:
                p = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2), s_in=s_in,
                                   weights=W[chosen])
                if form == "bf16":
                    q = pc.pc_quantize(b["d"], p, 0, b["thr32"], b["wst"])
                    p = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_BF16, stencil=k, hidden=(h1, h2), s_in=s_in,
                                       qnet=q)
            sz = pc.pc_compress(b["d"], p, b["out"], b["wsc"])
            b["ho"][:sz].copy_(b["out"][:sz])
            _, _, wsb = pc.pc_header_info(b["ho"][:256].numpy().tobytes())
            wsd = b.get("wsd")
            if wsd is None or wsd.numel() < wsb:
                wsd = b["wsd"] = torch.empty(wsb, dtype=torch.uint8, device=dev)
            pc.pc_decompress_host(b["ho"].numpy(), sz, b["hy"].numpy(), b["out"], b["d"], wsd)
        if it >= 1:
            t.append(time.perf_counter() - t0)
    nbytes = sum(h.numel() * h.element_size() for h in hosts)
    return {"value": nbytes / min(t) / 1e9, "unit": "GB/s", "seconds": min(t),
            "includes": "H2D, device training of 16 models, fixed-point form, compress, D2H, host-buffer decompress"}


def cpu_baseline(fields_host, spec, info, form, cores_all, pts_per_slab):
    """The oracle as it stands on the host cores: all of them, and one."""
    w = info["w"] if form == "fp32" else None
    q = info["q"] if form == "bf16" else None
    pred = (info["s_in"] if (w is not None or q is not None) else 0, w, q)
    v_all, t_all, desc_all = oracle_rate(fields_host, spec, pred, cores_all, pts_per_slab, rounds=1)
    v_one, t_one, desc_one = oracle_rate(fields_host, spec, pred, 1, pts_per_slab, rounds=1)
    return {"value": v_all, "unit": "GB/s", "cores": cores_all, "kind": "oracle", "sample": desc_all,
            "seconds": sum(t_all), "one_core": {"value": v_one, "cores": 1, "sample": desc_one,
                                                 "seconds": sum(t_one)}}


def run_workload(torch, pc, name, args, dev, stream, flush, peak, nsm, dist=None, headline=False, clk=None):
    spec = dict(WORKLOADS[name])
    fields = make_fields(name, dev)
    spec["_fields"] = fields
    infos = train_predictors(torch, pc, fields, spec, dev)
    form = args.form if (headline and args.form) else spec["form"]
    if infos[0]["w"] is None or (form == "bf16" and infos[0]["q"] is None):
        form = "fp32" if infos[0]["w"] is not None else "lorenzo"
    params, pnames = zip(*[params_for(pc, spec, inf, form) for inf in infos])
    steps = args.steps if headline else max(3, min(args.steps, 10))
    if clk:
        clk.start()
        time.sleep(0.5)
    res, r = measure(torch, pc, fields, spec, list(params), steps, args.warmup, stream, flush, dist)
    clocks = clk.stop() if clk else None
    res["predictor"] = sorted(set(pnames))
    res["form"] = form
    res["hbm_roofline"] = hbm_fractions(res, peak)
    # perceptron-predicted points (the recon stage's perceptron work)
    nn_pts = 0
    coded_pts = 0
    nn_blocks = []
    for i, d in enumerate(fields):
        blob = r.out[i][: r.size[i]].cpu().numpy().tobytes()
        flags, free_pts = block_census(blob, tuple(d.shape))
        nn_pts += int(free_pts[flags].sum())
        coded_pts += int(free_pts.sum())
        nn_blocks.append(float(flags.mean()))
    res["perceptron_blocks_fraction"] = nn_blocks
    res["perceptron_points"] = nn_pts
    st = res["stages_ms_per_step"]
    dom = max(st, key=lambda k: st[k])
    nlaunch = res["stage_launches_per_step"][dom]
    sm_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    res["roofline"] = stage_roofline(name, dom, st[dom] / nlaunch, res, spec, form, nn_pts / len(fields), nsm,
                                     sm_mhz, peak, coded_pts)
    res["training"] = [{k: v for k, v in inf.items() if k not in ("w", "q")} for inf in infos]
    res["training_seconds_total"] = sum(inf["train_s"] for inf in infos) + sum(inf["quant_s"] or 0 for inf in infos)
    out = {"res": res, "runner": r, "infos": infos, "spec": spec, "form": form, "clocks": clocks}
    return out


def form_compare(torch, pc, w, args, stream, flush):
    """The same workload with the other predictor forms (bits/value and throughput), for the
    FP32-vs-fixed-point comparison and the Lorenzo-only fallback."""
    spec, infos, fields = w["spec"], w["infos"], w["spec"]["_fields"]
    forms = {}
    for form in ("fp32", "bf16", "lorenzo"):
        if form != "lorenzo" and (infos[0]["w"] is None or (form == "bf16" and infos[0]["q"] is None)):
            continue
        params = [params_for(pc, spec, inf, form)[0] for inf in infos]
        res, r = measure(torch, pc, fields, spec, params, max(3, min(args.steps, 8)), 2, stream, flush)
        r.free()
        forms[form] = {k: res[k] for k in ("compress_gbs", "decompress_gbs", "bits_per_value", "bound_held",
                                           "compress_ms", "decompress_ms", "stages_ms_per_step")}
    if "fp32" in forms and "bf16" in forms:
        forms["bf16_bits_vs_fp32"] = forms["bf16"]["bits_per_value"] / forms["fp32"]["bits_per_value"] - 1.0
    if "lorenzo" in forms:
        for f in ("fp32", "bf16"):
            if f in forms:
                forms[f"{f}_bits_vs_lorenzo"] = forms[f]["bits_per_value"] / forms["lorenzo"]["bits_per_value"] - 1.0
    return forms


def single_pass(torch, pc, w, args, stream, flush, peak, two_pass):
    """Single-pass compression with the training phase's sample codebook (Section IV.C): the Huffman
    code of the validation samples' residuals (the chosen FP32 network's, or Lorenzo's), then one pass
    over each field.  Throughput, bits/value and the bits lost against the field's own code."""
    spec, infos, fields = w["spec"], w["infos"], w["spec"]["_fields"]
    k, h1, h2, eb = spec["k"], spec["h1"], spec["h2"], spec["eb"]
    out = {}
    for form in (w["form"], "lorenzo"):
        cbs, lits, t_cb = [], [], 0.0
        for d, inf in zip(fields, infos):
            use_w = form != "lorenzo" and inf["w"] is not None
            dt = pc.PC_F32 if d.dtype == torch.float32 else pc.PC_F64
            pp = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32 if use_w else pc.PC_PRED_LORENZO, stencil=k,
                                hidden=(h1, h2), s_in=inf["s_in"] if use_w else 0,
                                weights=inf["w"] if use_w else None)
            ws = torch.empty(pc.pc_train_workspace_size(tuple(d.shape), dt, pp, inf["thr32"], 1),
                             dtype=torch.uint8, device=d.device)
            lits.append(pc.pc_sample_codebook(d, pp, 0, inf["thr32"], ws))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cbs.append(pc.pc_sample_codebook(d, pp, 0, inf["thr32"], ws, span_fill=True))
            torch.cuda.synchronize()
            t_cb += time.perf_counter() - t0
            del ws
        params = [params_for(pc, spec, inf, form, cb)[0] for inf, cb in zip(infos, cbs)]
        res, r = measure(torch, pc, fields, spec, params, max(3, min(args.steps, 10)), 2, stream, flush)
        r.free()
        e = {k2: res[k2] for k2 in ("compress_gbs", "decompress_gbs", "bits_per_value", "bound_held", "compress_ms",
                                    "decompress_ms", "stages_ms_per_step")}
        e["hbm_roofline"] = hbm_fractions(res, peak)
        e["sample_codebook_s"] = t_cb
        e["codebook"] = "span-filled sample code (every code inside the sampled span has a code word)"
        e["codebook_entries"] = [int(c.size) for c in cbs]
        # the literal reading: codes the sample never saw become balance points
        lit_bytes = 0
        for d, inf, cb in zip(fields, infos, lits):
            p = params_for(pc, spec, inf, form, cb)[0]
            lit_bytes += pc.compress(d, p).numel()
        e["literal_sample_code"] = {"bits_per_value": 8.0 * lit_bytes / res["points"],
                                    "codebook_entries": [int(c.size) for c in lits]}
        ref = two_pass.get(form)
        if ref:
            e["bits_vs_two_pass"] = res["bits_per_value"] / ref["bits_per_value"] - 1.0
            e["literal_sample_code"]["bits_vs_two_pass"] = (e["literal_sample_code"]["bits_per_value"] /
                                                            ref["bits_per_value"] - 1.0)
            e["compress_speedup_vs_two_pass"] = ref["compress_ms"] / res["compress_ms"]
        out[form] = e
    return out


def lossless_report(torch, pc, fields, params, label):
    """The lossless back-end stage (Section IV.A's fourth SZ stage) on the given fields and predictors: bits per
    value and device throughput of compression and decompression with and without it."""
    out = {"fields": label}
    for name, on in (("without", False), ("with", True)):
        tot_bytes, tc, td = 0, 0.0, 0.0
        for d, p0 in zip(fields, params):
            p = pc.pc_params.from_buffer_copy(p0)
            for attr in ("_w", "_q", "_cb"):
                if hasattr(p0, attr):
                    setattr(p, attr, getattr(p0, attr))
            p.lossless = int(on)
            blob = pc.compress(d, p)  # warm-up and buffers
            y = pc.decompress(blob)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            blob = pc.compress(d, p)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            y = pc.decompress(blob)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            tot_bytes += blob.numel()
            tc += t1 - t0
            td += t2 - t1
            del y
        npts = sum(d.numel() for d in fields)
        nb = sum(d.numel() * d.element_size() for d in fields)
        out[name] = {"bits_per_value": 8.0 * tot_bytes / npts, "compress_gbs": nb / tc / 1e9,
                     "decompress_gbs": nb / td / 1e9}
    out["bits_vs_without"] = out["with"]["bits_per_value"] / out["without"]["bits_per_value"] - 1.0
    return out


def run_batch64(torch, pc, args, dev, stream, flush, peak):
    """The many-field batch: 32 2-D float32 fields 1800 x 3600 and 32 3-D float32 fields with dims drawn
    uniformly from [64, 384]^3, spectral slopes drawn from [2, 5], eb_rel cycling 1e-2, 1e-3, 1e-4;
    block shape per field from the autotuner, a fixed-point 7-point 16/16 perceptron trained on the
    device per field (2^18 sampled stencils), everything through pc_compress_batch / pc_decompress_batch."""
    from paper_2309_09778_gb300 import gen
    from paper_2309_09778_gb300.autotune import BlockTuner
    rng = np.random.default_rng(7)
    t0 = time.perf_counter()
    fields, ebs = [], []
    for f in range(64):
        shape = (1, 1800, 3600) if f < 32 else tuple(int(v) for v in rng.integers(64, 385, 3))
        beta = float(rng.uniform(2.0, 5.0))
        fields.append(gen.signed_lognormal_device(shape, beta, 100 + 10 * f, dev, 2.0, 0.05))
        ebs.append((1e-2, 1e-3, 1e-4)[f % 3])
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    tuner = BlockTuner(os.environ.get("PC_AUTOTUNE_CACHE"))
    t0 = time.perf_counter()
    blocks = [tuner.choose(x, eb, "lorenzo", lambda b, eb=eb: pc.make_params(eb, b)) for x, eb in zip(fields, ebs)]
    tune_s = time.perf_counter() - t0
    lrs, lams = pc.default_grid()
    params = []
    t0 = time.perf_counter()
    nn = 0
    for x, eb, b in zip(fields, ebs, blocks):
        thr = thr_for(tuple(x.shape), 1 << 18)
        tp = pc.make_params(eb, b, pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16))
        ws = torch.empty(pc.pc_train_workspace_size(tuple(x.shape), pc.PC_F32, tp, thr, lrs.size), dtype=torch.uint8,
                         device=dev)
        W, s_in, chosen, _ = pc.pc_train(x, tp, 0, thr, lrs, lams, ws)
        if chosen < 0:
            params.append(pc.make_params(eb, b))
            continue
        p32 = pc.make_params(eb, b, pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16), s_in=s_in,
                             weights=W[chosen])
        q = pc.pc_quantize(x, p32, 0, thr, ws)
        params.append(pc.make_params(eb, b, pred=pc.PC_PRED_MLP_BF16, stencil=7, hidden=(16, 16), s_in=s_in, qnet=q))
        nn += 1
        del ws
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    wsb, outb = pc.pc_compress_batch_workspace_size(fields, params)
    out = torch.empty(outb, dtype=torch.uint8, device=dev)
    wsc = torch.empty(wsb, dtype=torch.uint8, device=dev)
    offs, sizes = pc.pc_compress_batch(fields, params, out, wsc, stream)
    host = out.cpu().numpy()
    hdrs = [host[offs[i]: offs[i] + 256].tobytes() for i in range(len(fields))]
    del host
    wsd = torch.empty(pc.pc_decompress_batch_workspace_size(hdrs), dtype=torch.uint8, device=dev)
    ys = [torch.empty_like(x) for x in fields]
    steps = max(3, min(args.steps, 6))
    for _ in range(2):
        offs, sizes = pc.pc_compress_batch(fields, params, out, wsc, stream)
        pc.pc_decompress_batch(out, offs, sizes, ys, wsd, stream)
    torch.cuda.synchronize()
    ok = all(bool(((y.double() - x.double()).abs() <= eb * x.double().abs()).all().item())
             for x, y, eb in zip(fields, ys, ebs))
    pc.pc_profile_enable(True)
    pc.pc_profile_read()
    tc, td = [], []
    for _ in range(steps):
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        offs, sizes = pc.pc_compress_batch(fields, params, out, wsc, stream)
        e[1].record(stream)
        pc.pc_decompress_batch(out, offs, sizes, ys, wsd, stream)
        e[2].record(stream)
        torch.cuda.synchronize()
        tc.append(e[0].elapsed_time(e[1]))
        td.append(e[1].elapsed_time(e[2]))
    prof = pc.pc_profile_read()
    pc.pc_profile_enable(False)
    nbytes = sum(x.numel() * 4 for x in fields)
    npts = sum(x.numel() for x in fields)
    tcm, tdm = statistics.median(tc), statistics.median(td)
    comp = sum(sizes)
    stages = {k: v[0] / steps for k, v in prof.items() if v[1] > 0}
    choice = {}
    for b in blocks:
        choice["x".join(str(v) for v in b)] = choice.get("x".join(str(v) for v in b), 0) + 1
    return {"fields": len(fields), "points": npts, "input_bytes": nbytes,
            "compress_gbs": nbytes / (tcm * 1e6), "decompress_gbs": nbytes / (tdm * 1e6),
            "compress_ms": tcm, "decompress_ms": tdm, "bits_per_value": 8.0 * comp / npts, "bound_held": ok,
            "perceptron_fields": nn, "block_shapes_chosen": choice, "autotune_trials": tuner.trials,
            "hbm_frac_compress": (2 * nbytes + comp) / (tcm * 1e6) / peak["hbm_gbs"],
            "hbm_frac_decompress": (nbytes + comp) / (tdm * 1e6) / peak["hbm_gbs"],
            "compress_launches": {k: prof[k][1] / steps for k in ("compress",) if k in prof},
            "stages_ms_per_step": stages,
            "setup_seconds": {"generate": gen_s, "autotune": tune_s, "train_and_quantize": train_s}}


def select_report(torch, pc, w, dev):
    """The training phase's two selection rules on the same field and samples (Section IV.C): the residual
    bit-length proxy and the simulated compression (Huffman-coded validation codes plus stored balance
    points), with the coverage rule's m; container sizes with each choice."""
    spec, fields = w["spec"], w["spec"]["_fields"]
    d = fields[0]
    k, h1, h2, eb = spec["k"], spec["h1"], spec["h2"], spec["eb"]
    thr32 = thr_for(tuple(d.shape), spec["samples"])
    lrs, lams = pc.default_grid()
    tp = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2))
    ws = torch.empty(pc.pc_train_workspace_size(tuple(d.shape), pc.PC_F32, tp, thr32, lrs.size), dtype=torch.uint8,
                     device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    W, s_in, chosen, sizes, m_cov = pc.pc_train_select(d, tp, 0, thr32, lrs, lams, ws)
    torch.cuda.synchronize()
    sel_s = time.perf_counter() - t0
    _, _, chosen_proxy, _ = pc.pc_train(d, tp, 0, thr32, lrs, lams, ws)
    del ws
    out = {"chosen_by_bitlen_proxy": int(chosen_proxy), "chosen_by_simulated_compression": int(chosen),
           "simulated_bits": [int(v) for v in sizes], "m_by_coverage_rule": int(m_cov), "seconds": sel_s}
    for label, m in (("m16", 16), ("m_coverage", m_cov)):
        p = pc.make_params(eb, BLOCK, m=m) if chosen < 0 else pc.make_params(
            eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2), m=m, s_in=s_in, weights=W[chosen])
        blob = pc.compress(d, p)
        out[f"bits_per_value_{label}"] = 8.0 * blob.numel() / d.numel()
    return out


def literal_report(torch, pc, w, dev):
    """The paper-literal data selection (Section IV.D, experimental): every point predicted from the true
    values of its neighbours, the decoder drifting on its own reconstructions.  For Lorenzo and the chosen
    FP32 network, with no, sparse and dense deliberate equilibrium points: bits/value, the drift (largest
    relative error over eb, share of points beyond eb and beyond 1.5 eb) and device throughput, beside the
    bound-safe reading; then the acceptance rule over the 16 trained models (a model counts when its
    decoded field stays within 1.5 eb everywhere)."""
    spec, fields, infos = w["spec"], w["spec"]["_fields"], w["infos"]
    d = fields[0]
    if d.dtype != torch.float32:
        return None
    k, h1, h2, eb = spec["k"], spec["h1"], spec["h2"], spec["eb"]
    info = infos[0]
    dd = d.double()
    nz = dd != 0

    def run(p):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        blob = pc.compress(d, p)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        y = pc.decompress(blob)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        e = ((y.double() - dd).abs() / dd.abs())[nz]
        nb = d.numel() * 4
        return {"bits_per_value": 8.0 * blob.numel() / d.numel(), "max_rel_err_over_eb": float(e.max()) / eb,
                "frac_beyond_eb": float((e > eb).double().mean()), "frac_beyond_1p5eb": float((e > 1.5 * eb).double().mean()),
                "compress_gbs": nb / (t1 - t0) / 1e9, "decompress_gbs": nb / (t2 - t1) / 1e9}

    out = {"field": list(d.shape), "eb_rel": eb}
    preds = [("lorenzo", None)]
    if info["w"] is not None:
        preds.append((f"mlp_fp32_s{k}_{h1}x{h2}", info["w"]))
    for name, wt in preds:
        kw = dict(pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2), s_in=info["s_in"], weights=wt) if wt is not None \
            else {}
        run(pc.make_params(eb, BLOCK, literal=True, **kw))  # warm-up
        out[name] = {"bound_safe": run(pc.make_params(eb, BLOCK, **kw))}
        for eq in (0, 64, 16):
            out[name][f"literal_eq{eq}"] = run(pc.make_params(eb, BLOCK, literal=True, eq_period=eq, **kw))
    # the 1.5x acceptance rule over the trained models
    lrs, lams = pc.default_grid()
    thr32 = thr_for(tuple(d.shape), spec["samples"])
    tp = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2))
    ws = torch.empty(pc.pc_train_workspace_size(tuple(d.shape), pc.PC_F32, tp, thr32, lrs.size), dtype=torch.uint8,
                     device=dev)
    W, s_in, _, _ = pc.pc_train(d, tp, 0, thr32, lrs, lams, ws)
    del ws
    acc = []
    for i in range(W.shape[0]):
        r = run(pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=(h1, h2), s_in=s_in,
                               weights=W[i], literal=True))
        acc.append({"model": i, "bits_per_value": r["bits_per_value"], "max_rel_err_over_eb": r["max_rel_err_over_eb"],
                    "accepted": r["max_rel_err_over_eb"] <= 1.5})
    ok = [a for a in acc if a["accepted"]]
    out["acceptance_1p5eb"] = {"models": acc, "accepted": len(ok),
                               "chosen": min(ok, key=lambda a: a["bits_per_value"])["model"] if ok else None}
    return out


def summary(w):
    res = w["res"]
    keep = ("compress_gbs", "decompress_gbs", "bits_per_value", "bound_held", "compress_ms", "decompress_ms",
            "predictor", "form", "hbm_roofline", "roofline", "perceptron_blocks_fraction", "training_seconds_total")
    return {k: res[k] for k in keep}


def run_reference(args, rank: int):
    """The reference arm: the oracle, as it stands, on the host cores, on bounded samples of the headline
    workload (the same recipe at a sub-volume size), with the oracle's own training phase (untimed)."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2309_09778_gb300 import gen
    O.build()
    spec = dict(WORKLOADS[HEADLINE])
    shp = (32, 128, 128)
    fields = [np.exp(1.5 * gen.grf(shp, 2.0, 0)).astype(np.float32), gen.grf(shp, 4.0, 3).astype(np.float32)]
    best, W, s_in, _ = O.train(fields[0], spec["eb"], block=BLOCK, k=spec["k"], h1=spec["h1"], h2=spec["h2"], seed=0)
    w = W[best] if best >= 0 else None
    q = O.quantize(fields[0], spec["eb"], w, s_in, block=BLOCK, k=spec["k"], h1=spec["h1"], h2=spec["h2"]) \
        if w is not None else None
    cores = os.cpu_count() or 1
    pred = (s_in if w is not None else 0, None, q)
    for _ in range(args.warmup):
        oracle_rate(fields, spec, pred, cores, shp[0] * shp[1] * shp[2], rounds=1)
    ts = []
    nbytes = 0
    desc = ""
    for _ in range(max(1, args.steps)):
        v, t, desc = oracle_rate(fields, spec, pred, cores, shp[0] * shp[1] * shp[2], rounds=1)
        ts.append(sum(t))
        nbytes += v * sum(t) * 1e9
    v = nbytes / sum(ts) / 1e9
    line = {"metric": METRIC, "value": v, "unit": "GB/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": len(ts), "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": HEADLINE, "eb_rel": spec["eb"], "block": list(BLOCK),
                       "predictor": f"mlp_bf16_fixed_point_s{spec['k']}_{spec['h1']}x{spec['h2']} (oracle-trained "
                                    f"on a {shp[0]}x{shp[1]}x{shp[2]} density sample)" if q is not None else "lorenzo",
                       "sample": f"{shp[0]}x{shp[1]}x{shp[2]} fields of the same recipe (density and velocity)"},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_case(form: str):
    """A small case of the headline kernels for profiler captures (inputs larger than L2, a few GB at most)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_09778_gb300.pc as pc
    from paper_2309_09778_gb300 import gen
    dev = torch.device("cuda:0")
    if form == "f64":
        # the float64 workload's recipe at half its size (151 MB)
        d = gen.wide_range_device((128, 384, 384), 3.0, 0, dev, 8.0, 0.01)
        eb, k, h, thr32, dt = 1e-5, 7, (16, 16), THR10, pc.PC_F64
    else:
        d = torch.exp(1.5 * gen.grf_device((256, 256, 512), 2.0, 0, dev)).to(torch.float32)
        eb, k, h, thr32, dt = 1e-4, 13, (32, 32), thr_for((256, 256, 512), 1 << 18), pc.PC_F32
    tp = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=h)
    lrs, lams = pc.default_grid()
    tws = torch.empty(pc.pc_train_workspace_size(d.shape, dt, tp, thr32, lrs.size), dtype=torch.uint8,
                      device=dev)
    W, s_in, chosen, _ = pc.pc_train(d, tp, 0, thr32, lrs, lams, tws)
    p = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=k, hidden=h, s_in=s_in,
                       weights=W[max(chosen, 0)])
    if form in ("bf16", "f64"):
        q = pc.pc_quantize(d, p, 0, thr32, tws)
        p = pc.make_params(eb, BLOCK, pred=pc.PC_PRED_MLP_BF16, stencil=k, hidden=h, s_in=s_in, qnet=q)
    del tws
    blob = pc.compress(d, p)
    y = pc.decompress(blob)
    torch.cuda.synchronize()
    ok = bool(((y.double() - d.double()).abs() <= eb * d.double().abs()).all().item())
    print(f"profile case {form}: chosen {chosen}, {8.0 * blob.numel() / d.numel():.3f} bits/value, bound held {ok}")
    if not ok:
        raise SystemExit(1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--form", default=None, choices=["bf16", "fp32", "lorenzo"],
                    help="predictor form of the timed step (default: the workload's)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--profile-case", default=None, choices=["bf16", "fp32", "f64"],
                    help="run one compress and one decompress of a 256x256x512 density field (one quarter of a "
                         "headline field, same recipe, 13-point 32/32 network trained on 2^18 samples), or with "
                         "f64 of a 128x384x384 float64 field (the float64 workload's recipe at half size), for "
                         "profiler captures, then exit")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_09778_gb300.pc as pc

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    peak = measured_peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    clk = ClockSampler(local)
    head = run_workload(torch, pc, args.workload, args, dev, stream, flush, peak, nsm, dist, headline=True, clk=clk)
    res, spec, r = head["res"], head["spec"], head["runner"]
    forms = {} if args.no_forms else None
    e2e, hosts = e2e_rate(torch, pc, r, max(3, min(args.steps, 10)))
    e2e_t = e2e_with_training(torch, pc, hosts, spec, head["form"], dev)
    r.free()
    sp = lossless = None
    if not args.no_forms:
        forms = form_compare(torch, pc, head, args, stream, flush)
        two = {f: forms[f] for f in ("fp32", "bf16", "lorenzo") if f in forms}
        sp = single_pass(torch, pc, head, args, stream, flush, peak, two)
        hparams = [params_for(pc, spec, inf, head["form"])[0] for inf in head["infos"]]
        lossless = [lossless_report(torch, pc, spec["_fields"], hparams, "the headline fields, headline form")]
        from paper_2309_09778_gb300 import gen
        muted = gen.signed_lognormal_device((100, 500, 500), 11 / 3, 7, dev, 2.0, 0.6)
        lossless.append(lossless_report(torch, pc, [muted], [pc.make_params(1e-3, BLOCK)],
                                        "100x500x500 float32 signed log-normal with 60% muted (zero) regions, "
                                        "Lorenzo, eb 1e-3"))
        del muted
    # plain FP32: a device copy of the fields at HBM speed
    copy_gbs = []
    for d in spec["_fields"]:
        dst = torch.empty_like(d)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        c0.record(stream)
        for _ in range(5):
            dst.copy_(d)
        c1.record(stream)
        torch.cuda.synchronize()
        copy_gbs.append(2 * d.numel() * d.element_size() * 5 / (c0.elapsed_time(c1) * 1e6))
        del dst
    cpu = None
    report = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fh = [h.numpy() for h in hosts]
        pts = (32 * 128 * 128) if spec["k"] == 13 else (64 * 128 * 128)
        cpu = cpu_baseline(fh, spec, head["infos"][0], head["form"], os.cpu_count() or 1, pts)
        report = fp64_report(fh, spec, head["infos"], os.cpu_count() or 1, pts)
    del hosts
    spec.pop("_fields")
    torch.cuda.empty_cache()
    secondary = {}
    if world == 1 and not args.no_secondary:
        for name in WORKLOADS:
            if name == args.workload:
                continue
            w = run_workload(torch, pc, name, args, dev, stream, flush, peak, nsm)
            w["runner"].free()
            secondary[name] = summary(w)
            if name == "grf100x500x500_f32" and not args.no_forms:
                secondary[name]["forms"] = form_compare(torch, pc, w, args, stream, flush)
                secondary[name]["selection_by_simulated_compression"] = select_report(torch, pc, w, dev)
                secondary[name]["literal_data_selection"] = literal_report(torch, pc, w, dev)
            w["spec"].pop("_fields")
            del w
            torch.cuda.empty_cache()
        secondary["batch64_uneven"] = run_batch64(torch, pc, args, dev, stream, flush, peak)
        torch.cuda.empty_cache()
    clocks = head["clocks"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": job_rate(world, res["input_bytes"], res["ms_per_step"]), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if spec["dtype"] == "f64" else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "fields": spec["desc"], "eb_rel": spec["eb"], "block": list(BLOCK),
                       "predictor": res["predictor"], "form": res["form"],
                       "training": f"device, {spec['samples'] or '10% of'} sampled stencils per field, 16 models",
                       "l2": "inputs larger than L2 where they are; 256 MB flush between steps",
                       "parallelism": "replicas" if world > 1 else "1 GPU",
                       "value_is": "input bytes / (compress + decompress time) per step"},
            "compress_gbs": res["compress_gbs"], "decompress_gbs": res["decompress_gbs"],
            "bits_per_value": res["bits_per_value"], "bound_held": res["bound_held"],
            "hbm_roofline": res["hbm_roofline"], "roofline": res["roofline"],
            "perceptron_blocks_fraction": res["perceptron_blocks_fraction"],
            "perceptron_forms": forms, "single_pass_sample_codebook": sp, "lossless_stage": lossless,
            "stages_ms_per_step": res["stages_ms_per_step"],
            "training": res["training"], "training_seconds_total": res["training_seconds_total"],
            "vs_fp32_plain": {"bits_per_value": 32.0 * (2 if spec["dtype"] == "f64" else 1),
                              "ratio": 32.0 * (2 if spec["dtype"] == "f64" else 1) / res["bits_per_value"],
                              "device_copy_gbs": copy_gbs},
            "cpu_baseline": cpu, "e2e": e2e, "e2e_with_training": e2e_t, "fp64_predictor_report": report,
            "secondary": secondary,
            "clocks": clocks, "gpu_launches": int(round(res["launches_per_step"] * args.steps)),
            "wall_s_timed": res["wall_s_timed"], "sm_count": nsm,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
