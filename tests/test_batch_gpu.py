"""Batched steps (many readout streams per CUDA-graph launch) and the launch
autotuner: every stream's frames in the batch are bit-identical to the same
stream pushed alone, and tuning never changes results."""
import os

import numpy as np
import pytest

import oracle
import siggen
from helpers import TOL, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"

SPECS = [
    ("pfb", dict(N=256, T=4, win="hann")),
    ("pfb", dict(N=1024, T=8, win="kaiser")),
    ("pfb", dict(N=4096, T=8, win="kaiser")),
    ("pfb", dict(N=1024, T=16, win="hann")),     # DIRECT variant
    ("pfb", dict(N=16384, T=4, win="kaiser")),   # DIRECT variant, largest N
    ("demod", dict(L=1024, D=512, nt=64)),
    ("demod", dict(L=4096, D=2048, nt=300)),
    ("demod", dict(L=1024, D=2048, nt=100)),
]


def make_plan(lib, kind, spec, words):
    if kind == "pfb":
        return lib.Plan(spec["N"], spec["T"], window=spec["win"], beta=9.0 if spec["win"] == "kaiser" else 0.0,
                        words=words)
    return lib.Plan(0, spec["L"], window="blackman", cutoff=40e3 / 200e6, words=words, decimation=spec["D"])


def make_case(kind, spec, n, seed):
    if kind == "pfb":
        return siggen.pfb_case(n, spec["N"], min(24, spec["N"] // 4), seed=seed)
    return siggen.demod_case(n, spec["nt"], seed=seed)


def out_bufs(kind, spec, plan, F):
    nt = plan.n_tones
    full = torch.zeros((F, spec["N"]), dtype=torch.complex64, device=DEV) if kind == "pfb" else None
    tones = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    return full, tones


def test_batch_equals_streams_alone(lib):
    rng = np.random.default_rng(5)
    cases, splits = [], []
    for i, (kind, spec) in enumerate(SPECS):
        hop = spec.get("N", spec.get("D"))
        n = int(hop * rng.integers(40, 90) + rng.integers(0, hop))
        cases.append(make_case(kind, spec, n, 700 + i))
        a = int(rng.integers(1, n // 3))
        b = int(rng.integers(n // 3, 2 * n // 3))
        splits.append([0, a, b, n])
    plans_b = [make_plan(lib, k, s, c["words"]) for (k, s), c in zip(SPECS, cases)]
    plans_a = [make_plan(lib, k, s, c["words"]) for (k, s), c in zip(SPECS, cases)]
    xs = [torch.from_numpy(c["x"]).to(DEV) for c in cases]
    Fs = [p.frames_for(x.shape[0]) for p, x in zip(plans_a, xs)]
    outs_b = [out_bufs(k, s, p, F) for (k, s), p, F in zip(SPECS, plans_b, Fs)]
    outs_a = [out_bufs(k, s, p, F) for (k, s), p, F in zip(SPECS, plans_a, Fs)]
    batch = lib.Batch(plans_b)
    offs = [0] * len(SPECS)
    for step in range(3):
        chunk = [x[sp[step]:sp[step + 1]] for x, sp in zip(xs, splits)]
        got = batch.push(chunk, [o[0] for o in outs_b], [o[1] for o in outs_b], offs)
        offs = [a + b for a, b in zip(offs, got)]
    # the same streams alone, same splits
    for i, (p, x, sp) in enumerate(zip(plans_a, xs, splits)):
        off = 0
        for step in range(3):
            off += p.push_into(x[sp[step]:sp[step + 1]], outs_a[i][0], outs_a[i][1], frame_offset=off)
        assert off == offs[i] == Fs[i]
    torch.cuda.synchronize()
    for i, ((kind, spec), ob, oa) in enumerate(zip(SPECS, outs_b, outs_a)):
        if kind == "pfb":
            assert torch.equal(ob[0], oa[0]), i
        assert torch.equal(ob[1], oa[1]), i
    st = batch.stats()
    assert st["steps"] == 3 and st["graph_instantiations"] >= 1
    print("batch stats", st)
    # spot parity of one PFB and one demod stream against the oracle
    c = cases[1]
    _, h32 = oracle.pfb_prototype(1024, 8, "kaiser", 9.0)
    ref = oracle.pfb(c["x"], 1024, 8, h32.astype(np.float64), bins=plans_b[1].bins(), want_full=False)
    assert rel_rows(outs_b[1][1].cpu().numpy(), ref["tones"]).max() < TOL
    c = cases[5]
    refd = oracle.demod(c["x"], 1024, 512, oracle.lowpass("blackman", 1024, 40e3 / 200e6), c["words"])
    assert rel_rows(outs_b[5][1].cpu().numpy(), refd).max() < TOL


def test_batch_repeated_steps_update_graph_in_place(lib):
    N = 1024
    plans, xs = [], []
    for i in range(4):
        c = siggen.pfb_case(N * 64, N, 8, seed=900 + i)
        plans.append(lib.Plan(N, 8, window="hann", words=c["words"]))
        xs.append(torch.from_numpy(c["x"]).to(DEV))
    b = lib.Batch(plans)
    outs = [torch.zeros((N * 64 // N * 6, N), dtype=torch.complex64, device=DEV) for _ in plans]
    tones = [torch.zeros((8, 64 * 6), dtype=torch.complex64, device=DEV) for _ in plans]
    off = [0] * 4
    for step in range(6):
        got = b.push(xs, outs, tones, off)
        off = [a + g for a, g in zip(off, got)]
    torch.cuda.synchronize()
    st = b.stats()
    assert st["steps"] == 6
    assert st["graph_updates"] >= 4, st     # same topology: updated in place, not re-instantiated


def test_batch_rejects_bad_step_without_side_effects(lib):
    c = siggen.pfb_case(64 * 50, 64, 4, seed=3)
    p1 = lib.Plan(64, 4, window="hann", words=c["words"])
    p2 = lib.Plan(64, 4, window="hann", words=c["words"])
    b = lib.Batch([p1, p2])
    x = torch.from_numpy(c["x"]).to(DEV)
    ok_full = torch.zeros((50, 64), dtype=torch.complex64, device=DEV)
    ok_t = torch.zeros((4, 50), dtype=torch.complex64, device=DEV)
    small = torch.zeros((4, 10), dtype=torch.complex64, device=DEV)
    with pytest.raises(lib.RfrError) as ei:
        b.push([x, x], [ok_full, ok_full], [ok_t, small])
    assert ei.value.status == lib.E_SHORT
    assert p1.info()["samples_consumed"] == 0 and p2.info()["samples_consumed"] == 0
    with pytest.raises(lib.RfrError):
        lib.Batch([p1, p1])


def test_autotune_keeps_results_and_caches(lib, tmp_path, monkeypatch):
    monkeypatch.setenv("RFR_TUNE_CACHE", str(tmp_path / "tune.json"))
    for kind, spec in [("pfb", dict(N=4096, T=8, win="kaiser")), ("demod", dict(L=4096, D=2048, nt=256))]:
        hop = spec.get("N", spec.get("D"))
        c = make_case(kind, spec, hop * 300, 11)
        x = torch.from_numpy(c["x"]).to(DEV)
        a = make_plan(lib, kind, spec, c["words"])
        F = a.frames_for(x.shape[0])
        fa, ta = out_bufs(kind, spec, a, F)
        a.push_into(x, fa, ta)
        b = make_plan(lib, kind, spec, c["words"])
        ms = b.autotune(x.shape[0])
        assert ms > 0 and b.tune()["tuned"]
        assert b.info()["samples_consumed"] == 0          # stream state untouched
        fb, tb = out_bufs(kind, spec, b, F)
        b.push_into(x, fb, tb)
        torch.cuda.synchronize()
        assert torch.equal(ta, tb)
        if fa is not None:
            assert torch.equal(fa, fb)
        cp = make_plan(lib, kind, spec, c["words"])
        assert cp.autotune(x.shape[0]) == -1.0            # loaded from the cache file
        assert cp.tune() == b.tune()
    assert os.path.exists(tmp_path / "tune.json")
