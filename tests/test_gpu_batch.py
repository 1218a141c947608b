"""Batched compression and decompression (many fields of uneven shapes).

Fields that share dtype, block shape and predictor form go through the hot
kernel in one persistent launch over their (field, brick) work list; each
field must still come out exactly as a single-field call (and the oracle)
produces it, and the batched decoder must return every field bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2309_09778_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pc():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2309_09778_gb300.pc as pcm
    return pcm


def make_batch(pc, O):
    rng = np.random.default_rng(0)
    fields, params, oracle_args = [], [], []
    w7 = O.init_weights(7, 16, 16, seed=3)
    w7 = w7 + rng.standard_normal(w7.size).astype(np.float32) * np.float32(0.02)
    specs = [
        ((33, 40, 47), (8, 8, 8), np.float32, "lorenzo", 1e-2),
        ((24, 24, 24), (8, 8, 8), np.float32, "bf16", 1e-3),
        ((1, 50, 70), (1, 16, 32), np.float32, "lorenzo", 1e-3),
        ((17, 30, 41), (8, 8, 8), np.float64, "lorenzo", 1e-5),
        ((20, 36, 28), (8, 8, 8), np.float32, "bf16", 1e-2),
        ((16, 16, 64), (8, 8, 8), np.float32, "fp32", 1e-2),
        ((25, 19, 33), (8, 8, 8), np.float32, "fp32", 1e-3),
        ((12, 12, 12), (4, 4, 4), np.float32, "lorenzo", 1e-2),
        ((1, 60, 64), (1, 16, 32), np.float32, "lorenzo", 1e-2),
        ((30, 22, 26), (8, 8, 8), np.float32, "lorenzo", 1e-4),
    ]
    for i, (shape, block, dt, form, eb) in enumerate(specs):
        x = gen.signed_lognormal(shape, float(rng.uniform(2, 5)), 100 + 10 * i, 2.0, 0.05, dtype=dt)
        if form == "bf16":
            q = O.quantize(x, eb, w7, 3, block=block)
            p = pc.make_params(eb, block, pred=pc.PC_PRED_MLP_BF16, stencil=7, hidden=(16, 16), s_in=3, qnet=q)
            oa = dict(qnet=q, s_in=3)
        elif form == "fp32":
            p = pc.make_params(eb, block, pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16), s_in=3, weights=w7)
            oa = dict(weights=w7, s_in=3)
        else:
            p = pc.make_params(eb, block)
            oa = {}
        fields.append(x)
        params.append(p)
        oracle_args.append((eb, block, oa))
    return fields, params, oracle_args


def test_batch_matches_single_calls_and_oracle(pc, O):
    fields, params, oa = make_batch(pc, O)
    d = [torch.from_numpy(x).cuda() for x in fields]
    # the FP32 fields share one weights array (one launch needs one weights pointer)
    params[6].h_weights = params[5].h_weights
    params[6]._w = params[5]._w
    wsb, outb = pc.pc_compress_batch_workspace_size(d, params)
    out = torch.zeros(outb, dtype=torch.uint8, device="cuda")
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    for rep in range(2):
        offs, sizes = pc.pc_compress_batch(d, params, out, ws)
        host = out.cpu().numpy()
        for i, x in enumerate(fields):
            got = host[offs[i]: offs[i] + sizes[i]].tobytes()
            single = pc.compress(d[i], params[i]).cpu().numpy().tobytes()
            assert got == single, (rep, i)
            eb, block, kw = oa[i]
            st, want = O.compress(x, eb, block=block, **kw)
            assert st == 0 and got == want, (rep, i)
    # batched decompression
    hdrs = [host[offs[i]: offs[i] + 256].tobytes() for i in range(len(fields))]
    wsd = torch.empty(pc.pc_decompress_batch_workspace_size(hdrs), dtype=torch.uint8, device="cuda")
    ys = [torch.full_like(t, float("nan")) for t in d]
    pc.pc_decompress_batch(out, offs, sizes, ys, wsd)
    torch.cuda.synchronize()
    for i, x in enumerate(fields):
        ref = pc.decompress(out[offs[i]: offs[i] + sizes[i]])
        view = torch.int32 if x.dtype == np.float32 else torch.int64
        assert torch.equal(ys[i].view(view), ref.view(view)), i
        eb = oa[i][0]
        y = ys[i].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(y - x) <= eb * np.abs(x.astype(np.float64)))


def test_batch_rejects_training_requests(pc):
    x = torch.ones((16, 16, 16), dtype=torch.float32, device="cuda")
    p = pc.make_params(1e-2, (8, 8, 8), pred=pc.PC_PRED_MLP_FP32, stencil=7, hidden=(16, 16))
    with pytest.raises(pc.PcError):
        pc.pc_compress_batch_workspace_size([x], [p])


def test_autotuner_picks_a_candidate_and_caches(pc, tmp_path):
    from paper_2309_09778_gb300.autotune import BlockTuner, CAND_2D, CAND_3D
    path = str(tmp_path / "tune.json")
    t = BlockTuner(path)
    x3 = torch.from_numpy(gen.signed_lognormal((48, 64, 80), 3.0, 1, 2.0, 0.05)).cuda()
    x2 = torch.from_numpy(gen.signed_lognormal((1, 300, 400), 3.0, 2, 2.0, 0.05)).cuda()
    b3 = t.choose(x3, 1e-3, "lorenzo", lambda b: pc.make_params(1e-3, b))
    b2 = t.choose(x2, 1e-3, "lorenzo", lambda b: pc.make_params(1e-3, b))
    assert b3 in CAND_3D and b2 in CAND_2D
    n = t.trials
    assert n == len(CAND_3D) + len(CAND_2D)
    # the chosen shape is within 1% of the smallest container on the sample
    sub = t.sample(x3)
    sizes = {b: pc.compress(sub, pc.make_params(1e-3, b)).numel() for b in CAND_3D}
    assert sizes[b3] <= 1.01 * min(sizes.values())
    # cached: no new trials, and a fresh tuner reads the file
    assert t.choose(x3, 1e-3, "lorenzo", lambda b: pc.make_params(1e-3, b)) == b3 and t.trials == n
    t2 = BlockTuner(path)
    assert t2.choose(x2, 1e-3, "lorenzo", lambda b: pc.make_params(1e-3, b)) == b2 and t2.trials == 0
