"""Block-shape autotuner for the batched compressor.

For a field and a predictor form, each candidate block shape (3-D fields:
4x4x4, 8x8x8, 16x16x16; 2-D fields: 8x8, 16x32, 64x64, the same point counts)
compresses and decompresses a centred sample of the field through the
library's own entry points; among the shapes whose container is within 1% of
the smallest, the one with the shortest round trip wins (large blocks decode
with less parallelism, small ones carry more anchors).  Choices are kept in a JSON cache keyed by (dimensionality,
dtype, eb_rel, predictor form, size class), in memory and, when a path is
given, on disk, so a batch of similar fields is tuned once.  The tile of the
tensor-core stage is fixed by the hardware (128 points per MMA tile), so the
block shape is the one free parameter.
"""
from __future__ import annotations

import json
import os
import threading
import time

CAND_3D = ((4, 4, 4), (8, 8, 8), (16, 16, 16))
CAND_2D = ((1, 8, 8), (1, 16, 32), (1, 64, 64))

_lock = threading.Lock()


def size_class(shape) -> str:
    n = 1
    for s in shape:
        n *= int(s)
    return f"2^{max(0, n.bit_length() - 1) // 2 * 2}"


def key_of(shape, dtype_code: int, eb: float, form: str) -> str:
    nd = 2 if int(shape[0]) == 1 else 3
    return f"{nd}d|{'f64' if dtype_code else 'f32'}|{eb:.3g}|{form}|{size_class(shape)}"


class BlockTuner:
    def __init__(self, path: str | None = None):
        self.path = path
        self.cache: dict[str, list[int]] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.cache = {k: list(v) for k, v in json.load(f).items()}
        self.trials = 0

    def _save(self):
        if not self.path:
            return
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    @staticmethod
    def sample(field):
        """A centred crop of at most 64^3 points (3-D) or 1 x 256 x 256 (2-D)."""
        z, y, x = (int(s) for s in field.shape)
        if z == 1:
            cy, cx = min(y, 256), min(x, 256)
            return field[:, (y - cy) // 2:(y - cy) // 2 + cy, (x - cx) // 2:(x - cx) // 2 + cx].contiguous()
        c = [min(s, 64) for s in (z, y, x)]
        o = [(s - k) // 2 for s, k in zip((z, y, x), c)]
        return field[o[0]:o[0] + c[0], o[1]:o[1] + c[1], o[2]:o[2] + c[2]].contiguous()

    def choose(self, field, eb: float, form: str, make_params):
        """Best block shape for `field` (device tensor).  make_params(block) -> pc_params of the form."""
        import torch
        import paper_2309_09778_gb300.pc as pc
        dt = pc.PC_F64 if field.dtype == torch.float64 else pc.PC_F32
        k = key_of(field.shape, dt, eb, form)
        with _lock:
            if k in self.cache:
                return tuple(self.cache[k])
        sub = self.sample(field)
        cands = CAND_2D if int(field.shape[0]) == 1 else CAND_3D
        trials = []
        for b in cands:
            p = make_params(b)
            blob = pc.compress(sub, p)  # warm
            pc.decompress(blob)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            blob = pc.compress(sub, p)
            pc.decompress(blob)
            torch.cuda.synchronize()
            self.trials += 1
            trials.append((b, blob.numel(), time.perf_counter() - t0))
        smallest = min(t[1] for t in trials)
        best = min((t for t in trials if t[1] <= 1.01 * smallest), key=lambda t: t[2])
        with _lock:
            self.cache[k] = list(best[0])
            self._save()
        return best[0]
