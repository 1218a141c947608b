#!/usr/bin/env python
"""Throughput benchmark of the GB300 compressor on one 100x500x500 float32 field.

One step = pc_compress + pc_decompress of the field (the whole hot path:
statistics, constants, transform, prediction, quantization, histogram,
codebook, packing, and the inverse path).  The field is a seeded synthetic
log-normal signed Gaussian random field (power spectrum k^-11/3, 2% exact
zeros) standing in for the paper's SEG-Y volumes, eb_rel = 1e-3, 8x8x8 blocks.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same field instead.
"""
from __future__ import annotations

import argparse
import json
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
SHAPE = (100, 500, 500)
EB = 1e-3
BLOCK = (8, 8, 8)
SAMPLE = (40, 200, 200)  # reference-arm sample per step: a corner sub-volume of the same field
THR32 = int(0.1 * 2 ** 32)  # 10% of points drawn for training (Section IV.C)


def field():
    from paper_2309_09778_gb300 import gen
    return gen.signed_lognormal(SHAPE, 11.0 / 3.0, 0, 2.0, 0.02)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""

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


def oracle_predictor(sub: np.ndarray):
    """The oracle's own training phase on the sample (10% sampling, the 16-model grid)."""
    from oracle import oracle as O
    best, W, s_in, costs = O.train(sub, EB, block=BLOCK, k=7, h1=16, h2=16, seed=0, thr32=THR32)
    return (W[best], s_in, "mlp_fp32_s7_16x16") if best >= 0 else (None, 0, "lorenzo")


def cpu_oracle_rate(x: np.ndarray, steps: int, predictor=None, shape=SAMPLE):
    """Time the oracle's compress + decompress on a corner sub-volume of the given shape."""
    from oracle import oracle as O
    sub = np.ascontiguousarray(x[: shape[0], : shape[1], : shape[2]])
    if predictor is None:
        predictor = oracle_predictor(sub)
    w, s_in = predictor[0], predictor[1]
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        st, blob = O.compress(sub, EB, block=BLOCK, weights=w, s_in=s_in)
        st2, y = O.decompress(blob)
        t.append(time.perf_counter() - t0)
        assert st == 0 and st2 == 0
    return sub.nbytes, t, predictor[2]


def run_reference(args, rank: int):
    if rank != 0:
        return
    x = field()
    nbytes, t, pname = cpu_oracle_rate(x, max(1, args.steps))
    v = nbytes * len(t) / sum(t) / 1e9
    sample = f"sub-volume {SAMPLE[0]}x{SAMPLE[1]}x{SAMPLE[2]} of the workload field, compress+decompress per step"
    line = {"metric": METRIC, "value": v, "unit": "GB/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": len(t), "warmup": 0, "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grf100x500x500_f32", "eb_rel": EB, "block": list(BLOCK),
                       "predictor": pname, "training": "oracle training phase on the sample, untimed"},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# Kernels behind each profiled stage (the codebook stage launches k_codebook and k_cb_assign; the decoder's
# scan stage k_dec_chunksum, k_dec_chunkscan and k_dec_blockoff).
KERNELS_PER_STAGE = {"codebook": 2, "dec_scan": 3}

# DRAM bytes (read + write) of one launch, from the ncu capture in profiles/k_recon_c2_fp32.md
# (FP32 form of this workload); valid while that kernel is unchanged.
TRAFFIC_PER_LAUNCH = {("recon", "fp32"): 55235584 + 43935488}

# FP32 peak from unit counts and clock: 152 SMs x 128 FP32 lanes x 2 flop (FMA) per cycle.
SMS, FP32_LANES = 152, 128


def perceptron_flops_per_point(k: int, h1: int, h2: int) -> int:
    """2 flop per weight multiply-accumulate of one forward pass (biases initialise the sums)."""
    return 2 * (k * h1 + (h1 * h2 + h2 if h2 else h1))


def block_census(blob: bytes, shape, block):
    """Per block: perceptron flag, points that are neither anchor nor balance point (from the container)."""
    import struct
    _, off_bb, off_bn, _, _ = struct.unpack_from("<5Q", blob, 176)
    nb = [-(-s // b) for s, b in zip(shape, block)]
    nblocks = nb[0] * nb[1] * nb[2]
    flags = np.frombuffer(blob, "<u4", nblocks, off_bb) >> 31
    nout = np.frombuffer(blob, "<u2", nblocks, off_bn).astype(np.int64)
    ext = [np.minimum(b, s - np.arange(n) * b) for s, b, n in zip(shape, block, nb)]
    pts = (ext[0][:, None, None] * ext[1][None, :, None] * ext[2][None, None, :]).reshape(-1)
    return flags.astype(bool), pts - nout


def roofline(stage: str, ms: float, n: int, comp_bytes: int, nn_pts: int, fpp: int, sm_mhz: float, hbm: float,
             hbm_kind: str):
    """Algorithmic work of one launch of `stage` against its bounding roof."""
    alu_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    if stage in ("recon", "compress") and fpp:
        pts = nn_pts if stage == "recon" else n
        flops = fpp * pts
        a = flops / (ms * 1e-3) / 1e12
        return {"kernel": stage, "bound": "alu", "achieved": a, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": a / alu_peak, "peak_source": f"derived: {SMS} SMs x {FP32_LANES} FP32 lanes x 2 flop x "
                f"{sm_mhz:.0f} MHz", "algorithmic_flops_per_launch": flops, "avg_launch_ms": ms}
    alg = {"stats": 4 * n, "compress": 4 * n + 2 * n, "pack": 2 * n + comp_bytes, "huff_decode": comp_bytes + 2 * n,
           "recon": 2 * n + 4 * n}.get(stage, 0)
    a = alg / (ms * 1e6) if alg else None
    return {"kernel": stage, "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
            "frac": (a / hbm) if a else None, "peak_source": hbm_kind, "algorithmic_bytes_per_launch": alg,
            "avg_launch_ms": ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", default="fp32", choices=["bf16", "fp32"],
                    help="perceptron form of the timed step (the other form is timed beside it)")
    args = ap.parse_args()
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
    x = field()
    n = x.size
    nbytes = x.nbytes
    d = torch.from_numpy(x).to(dev)
    # training phase (Section IV.C / V): on the device, before compression, timed separately
    tparams = pc.make_params(EB, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16))
    lrs, lams = pc.default_grid()
    tws = torch.empty(pc.pc_train_workspace_size(SHAPE, pc.PC_F32, tparams, THR32, lrs.size), dtype=torch.uint8,
                      device=dev)
    pc.pc_train(d, tparams, 0, THR32, lrs, lams, tws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    W, s_in, chosen, tcosts = pc.pc_train(d, tparams, 0, THR32, lrs, lams, tws)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    w = W[chosen] if chosen >= 0 else None
    # fixed-point (BF16 tensor-core) form of the chosen perceptron, from the same samples
    q = None
    quant_s = None
    p32 = pc.make_params(EB, BLOCK, pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16), s_in=s_in, weights=w)
    if w is not None:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        q = pc.pc_quantize(d, p32, 0, THR32, tws)
        torch.cuda.synchronize()
        quant_s = time.perf_counter() - t0
    del tws
    pbf = pc.make_params(EB, BLOCK, pred=pc.PC_PRED_MLP_BF16, stencil=7, hidden=(16, 16), s_in=s_in, qnet=q)
    if w is None:
        pname, params = "lorenzo", pc.make_params(EB, BLOCK)
    elif args.form == "bf16":
        pname, params = "mlp_bf16_tensorcore_s7_16x16", pbf
    else:
        pname, params = "mlp_fp32_s7_16x16", p32
    lz_size = pc.compress(d, pc.make_params(EB, BLOCK)).numel()
    cap = pc.pc_compress_bound(SHAPE, pc.PC_F32, params)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    wsc = torch.empty(pc.pc_compress_workspace_size(SHAPE, pc.PC_F32, params), dtype=torch.uint8, device=dev)
    y = torch.empty_like(d)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream(dev)
    size = pc.pc_compress(d, params, out, wsc)
    _, _, wsb = pc.pc_header_info(out[:256].cpu().numpy().tobytes())
    wsd = torch.empty(wsb, dtype=torch.uint8, device=dev)

    def step(timing):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        sz = pc.pc_compress(d, params, out, wsc, stream)
        e1.record(stream)
        pc.pc_decompress(out, sz, y, wsd, stream)
        e2.record(stream)
        timing.append((e0, e1, e2))
        return sz

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    ok = bool(((y.double() - d.double()).abs() <= EB * d.double().abs()).all().item())
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)  # let the sampler start before the timed region
    pc.pc_profile_enable(True)
    pc.pc_profile_read()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = []
    for _ in range(args.steps):
        size = step(ev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t0
    prof = pc.pc_profile_read()
    pc.pc_profile_enable(False)
    clk = clocks.stop()
    tc = sum(a.elapsed_time(b) for a, b, _ in ev) / len(ev)
    td = sum(b.elapsed_time(c) for _, b, c in ev) / len(ev)
    t_step = tc + td
    if dist:
        tt = torch.tensor([t_step, tc, td], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step, tc, td = tt.tolist()

    # end to end through the host-buffer entry points (pinned host memory)
    h_field = torch.from_numpy(x).pin_memory()
    h_out = torch.empty(cap, dtype=torch.uint8).pin_memory()
    h_y = torch.empty(SHAPE, dtype=torch.float32).pin_memory()
    dstage = torch.empty_like(d)
    hf, ho, hy = h_field.numpy(), h_out.numpy(), h_y.numpy()
    for _ in range(2):
        sz = pc.pc_compress_host(hf, params, ho, dstage, out, wsc)
        pc.pc_decompress_host(ho, sz, hy, out, dstage, wsd)
    te = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        sz = pc.pc_compress_host(hf, params, ho, dstage, out, wsc)
        pc.pc_decompress_host(ho, sz, hy, out, dstage, wsd)
        te.append(time.perf_counter() - t1)
    e2e_ok = np.array_equal(hy.view(np.uint32), y.cpu().numpy().view(np.uint32))

    # the other perceptron form on the same field, for the FP32 vs BF16 comparison
    forms = {}
    if w is not None:
        for fname, fp in (("bf16", pbf), ("fp32", p32)):
            ws2 = torch.empty(pc.pc_compress_workspace_size(SHAPE, pc.PC_F32, fp), dtype=torch.uint8, device=dev)
            o2 = torch.empty(pc.pc_compress_bound(SHAPE, pc.PC_F32, fp), dtype=torch.uint8, device=dev)
            tcs, tds = [], []
            for it in range(3 + min(args.steps, 40)):
                flush.zero_()
                a, b, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record(stream)
                sz2 = pc.pc_compress(d, fp, o2, ws2, stream)
                b.record(stream)
                pc.pc_decompress(o2, sz2, y, wsd, stream)
                c2.record(stream)
                torch.cuda.synchronize()
                if it >= 3:
                    tcs.append(a.elapsed_time(b))
                    tds.append(b.elapsed_time(c2))
            okf = bool(((y.double() - d.double()).abs() <= EB * d.double().abs()).all().item())
            forms[fname] = {"compress_gbs": nbytes / (statistics.median(tcs) * 1e6),
                            "decompress_gbs": nbytes / (statistics.median(tds) * 1e6),
                            "bits_per_value": 8.0 * sz2 / n, "bound_held": okf}
            del ws2, o2
        forms["bf16_size_vs_fp32"] = forms["bf16"]["bits_per_value"] / forms["fp32"]["bits_per_value"] - 1.0

    # plain FP32: a device copy of the field at HBM speed
    dst = torch.empty_like(d)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.zero_()
    c0.record(stream)
    for _ in range(5):
        dst.copy_(d)
    c1.record(stream)
    torch.cuda.synchronize()
    copy_gbs = 2 * nbytes * 5 / (c0.elapsed_time(c1) * 1e6)

    peak, peak_kind = peaks()
    stages = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(stages, key=lambda k: stages[k][0])
    dom_ms = stages[dom][0] / stages[dom][1]
    blob = out[:size].cpu().numpy().tobytes()
    nnflag, free_pts = block_census(blob, SHAPE, BLOCK)
    nn_pts = int(free_pts[nnflag].sum())
    fpp = perceptron_flops_per_point(7, 16, 16) if (w is not None and args.form == "fp32") else 0
    bpv = 8.0 * size / n
    launches = sum(v[1] * KERNELS_PER_STAGE.get(k, 1) for k, v in stages.items())

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            # the whole workload field, once; the oracle first trains its own predictor on it (untimed)
            nb, t, opn = cpu_oracle_rate(x, 1, shape=SHAPE)
            cpu = {"value": nb / t[0] / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
                   "sample": f"the whole {SHAPE[0]}x{SHAPE[1]}x{SHAPE[2]} field once, compress+decompress with "
                             f"the oracle's own trained {opn} predictor (training untimed), {t[0]:.1f} s"}
        line = {
            "metric": METRIC, "value": world * nbytes / (t_step * 1e6), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "grf100x500x500_f32: 100x500x500 float32 signed log-normal GRF, k^-11/3, "
                                   "2% zeros", "eb_rel": EB, "block": list(BLOCK), "predictor": pname,
                       "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "compress_gbs": nbytes / (tc * 1e6), "decompress_gbs": nbytes / (td * 1e6),
            "bits_per_value": bpv, "bound_held": ok,
            "perceptron_forms": forms,
            "training": {"seconds": train_s, "quantize_seconds": quant_s, "models": int(lrs.size),
                         "chosen": int(chosen), "s_in": int(s_in),
                         "samples_rate": THR32 / 2 ** 32, "val_cost_chosen": int(tcosts[chosen]) if chosen >= 0 else None,
                         "val_cost_lorenzo": int(tcosts[-1])},
            "bits_per_value_lorenzo_only": 8.0 * lz_size / n,
            "vs_fp32_plain": {"bits_per_value": 32.0, "ratio": 32.0 / bpv, "device_copy_gbs": copy_gbs},
            "roofline": dict(roofline(dom, dom_ms, n, size, nn_pts, fpp, clk.get("sm_max_mhz") or 2070.0, peak,
                                      peak_kind), traffic=TRAFFIC_PER_LAUNCH.get((dom, args.form))),
            "perceptron_blocks": {"fraction": float(nnflag.mean()), "points": nn_pts},
            "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": nbytes / statistics.median(te) / 1e9, "unit": "GB/s",
                    "h2d_bytes_per_step": nbytes + size, "d2h_bytes_per_step": size + nbytes,
                    "matches_device_path": e2e_ok},
            "clocks": clk, "gpu_launches": launches, "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
