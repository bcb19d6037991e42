"""The serving loop: buffers of many readouts submitted in an interleaved order
(host or device inputs), admitted under a device-memory budget and run
concurrently; every readout's frames equal (bit-identically) those of the
same readout processed alone, which are themselves within tolerance of the
FP64 oracle (checked for one PFB and one demodulation readout)."""
import numpy as np
import pytest

import oracle
import siggen
from helpers import TOL, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"

READOUTS = [
    ("pfb", dict(N=1024, T=8, win="kaiser")),
    ("demod", dict(L=1024, D=512, nt=64)),
    ("pfb", dict(N=256, T=4, win="hann")),
    ("demod", dict(L=4096, D=2048, nt=200)),
    ("pfb", dict(N=4096, T=16, win="kaiser")),
    ("demod", dict(L=1024, D=2048, nt=40)),
]


def make_plan(lib, kind, spec, words):
    if kind == "pfb":
        return lib.Plan(spec["N"], spec["T"], window=spec["win"], beta=9.0 if spec["win"] == "kaiser" else 0.0,
                        words=words, full=False)
    return lib.Plan(0, spec["L"], window="blackman", cutoff=40e3 / 200e6, words=words, decimation=spec["D"])


def setup_streams(n_buffers, seed):
    rng = np.random.default_rng(seed)
    streams = []
    for i, (kind, spec) in enumerate(READOUTS):
        hop = spec.get("N", spec.get("D"))
        n = int(hop * rng.integers(30, 60) + rng.integers(0, hop))
        if kind == "pfb":
            c = siggen.pfb_case(n, spec["N"], min(16, spec["N"] // 4), seed=seed + i)
        else:
            c = siggen.demod_case(n, spec["nt"], seed=seed + i)
        cuts = np.sort(rng.choice(np.arange(1, n), n_buffers - 1, replace=False))
        streams.append((kind, spec, c, [0, *cuts.tolist(), n]))
    return streams


def alone(lib, kind, spec, c, cuts):
    """The readout processed alone; returns (frames, per-buffer frame offsets)."""
    p = make_plan(lib, kind, spec, c["words"])
    x = torch.from_numpy(c["x"]).to(DEV)
    F = p.frames_for(x.shape[0])
    out = torch.zeros((p.n_tones, F), dtype=torch.complex64, device=DEV)
    offs, off = [], 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        offs.append(off)
        off += p.push_into(x[a:b], tones=out, frame_offset=off)
    torch.cuda.synchronize()
    return out.cpu().numpy(), offs


def interleaved(streams, seed):
    """(readout, buffer index) in a random interleaving, each readout in order."""
    rng = np.random.default_rng(seed)
    nxt = [0] * len(streams)
    order = []
    while any(nxt[i] < len(s[3]) - 1 for i, s in enumerate(streams)):
        r = int(rng.integers(0, len(streams)))
        if nxt[r] < len(streams[r][3]) - 1:
            order.append((r, nxt[r]))
            nxt[r] += 1
    return order


def serve(lib, streams, refs, budget, device_inputs, pageable_outputs=False):
    plans = [make_plan(lib, k, s, c["words"]) for k, s, c, _ in streams]
    max_n = max(max(b - a for a, b in zip(cu[:-1], cu[1:])) for *_, cu in streams)
    srv = lib.Server(plans, budget, max_n)
    if device_inputs:
        xs = [torch.from_numpy(c["x"]).to(DEV) for _, _, c, _ in streams]
        outs = [torch.zeros(r.shape, dtype=torch.complex64, device=DEV) for r, _ in refs]
    else:
        xs = [torch.from_numpy(c["x"]).pin_memory() for _, _, c, _ in streams]
        # pinned outputs are written by the server's row-copy kernel through
        # their mapping; pageable ones by 2-D copies
        outs = [torch.zeros(r.shape, dtype=torch.complex64) if pageable_outputs else
                torch.zeros(r.shape, dtype=torch.complex64).pin_memory() for r, _ in refs]
    order = interleaved(streams, 1)
    for tag, (r, j) in enumerate(order):
        cu = streams[r][3]
        srv.submit(r, xs[r][cu[j]:cu[j + 1]], tones=outs[r], frame_offset=refs[r][1][j], tag=tag)
    done = []
    while len(done) < len(order):
        done += srv.poll(64, wait_ms=100)
    st = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], done, st, len(order)


def test_server_mix_equals_alone(lib):
    streams = setup_streams(5, 400)
    refs = [alone(lib, k, s, c, cu) for k, s, c, cu in streams]
    outs, done, st, n_req = serve(lib, streams, refs, 256 << 20, device_inputs=False)
    assert st["completed"] == n_req and st["peak_bytes"] <= st["budget_bytes"]
    assert sorted(c["tag"] for c in done) == list(range(n_req))
    for c in done:
        assert c["status"] == 0 and c["t_submit_us"] <= c["t_admit_us"] <= c["t_done_us"]
    for i, (o, (r, _)) in enumerate(zip(outs, refs)):
        assert np.array_equal(o, r), i
    # the references against the oracle (one PFB, one demodulation readout)
    kind, spec, c, _ = streams[0]
    _, h32 = oracle.pfb_prototype(spec["N"], spec["T"], spec["win"], 9.0)
    bins = [oracle.word_to_bin(int(w), spec["N"]) for w in c["words"]]
    ref = oracle.pfb(c["x"], spec["N"], spec["T"], h32.astype(np.float64), bins=bins, want_full=False)
    assert rel_rows(refs[0][0], ref["tones"]).max() < TOL
    kind, spec, c, _ = streams[1]
    refd = oracle.demod(c["x"], spec["L"], spec["D"], oracle.lowpass("blackman", spec["L"], 40e3 / 200e6),
                        c["words"])
    assert rel_rows(refs[1][0], refd).max() < TOL


def test_server_pageable_host_outputs(lib):
    """Outputs in pageable host memory (no mapping): the frames still equal
    each readout processed alone."""
    streams = setup_streams(3, 450)
    refs = [alone(lib, k, s, c, cu) for k, s, c, cu in streams]
    outs, done, st, n_req = serve(lib, streams, refs, 256 << 20, device_inputs=False, pageable_outputs=True)
    assert st["completed"] == n_req
    for c in done:
        assert c["status"] == 0
    for i, (o, (r, _)) in enumerate(zip(outs, refs)):
        assert np.array_equal(o, r), i


def test_server_tight_budget_device_inputs(lib):
    streams = setup_streams(4, 500)
    refs = [alone(lib, k, s, c, cu) for k, s, c, cu in streams]
    max_n = max(max(b - a for a, b in zip(cu[:-1], cu[1:])) for *_, cu in streams)
    budget = max(1 << 20, int(max_n * 2))     # a few requests' outputs at a time
    outs, done, st, n_req = serve(lib, streams, refs, budget, device_inputs=True)
    assert st["completed"] == n_req and st["peak_bytes"] <= budget
    for o, (r, _) in zip(outs, refs):
        assert np.array_equal(o, r)


def test_server_refuses_request_larger_than_budget(lib):
    c = siggen.pfb_case(1024 * 10, 1024, 16, seed=2)
    p = make_plan(lib, *READOUTS[0], c["words"])
    srv = lib.Server([p], 1 << 20, 1 << 22)
    with pytest.raises(lib.RfrError) as ei:
        srv.submit(0, torch.zeros((1 << 22, 2), dtype=torch.int16).pin_memory(),
                   tones=torch.zeros((16, 4096), dtype=torch.complex64).pin_memory())
    assert ei.value.status == lib.E_NOMEM
    with pytest.raises(lib.RfrError):
        srv.submit(5, torch.zeros((16, 2), dtype=torch.int16).pin_memory())
    srv.close()


def test_server_reports_a_device_timeout_for_that_request_only(lib):
    """Failure detection without a GPU fault: the plan's device status word is
    set on the host (as a kernel whose bounded wait gave up would set it); the
    next request completes with RFR_E_TIMEOUT, the one after it with RFR_OK."""
    N, hop = 1024, 1024
    c = siggen.pfb_case(N * 40, N, 8, seed=3)
    p = lib.Plan(N, 4, window="hann", words=c["words"], full=False)
    srv = lib.Server([p], 64 << 20, N * 20)
    x = torch.from_numpy(c["x"]).to(DEV)
    out = torch.zeros((8, 40), dtype=torch.complex64, device=DEV)
    p.inject_device_status(1)
    got = {}
    for tag, (a, b) in enumerate([(0, N * 20), (N * 20, N * 40)]):
        srv.submit(0, x[a:b], tones=out, frame_offset=a // hop, tag=tag)
        while tag not in got:
            for d in srv.poll(8, wait_ms=100):
                got[d["tag"]] = d
    srv.close()
    assert got[0]["status"] == lib.E_TIMEOUT
    assert got[1]["status"] == lib.OK
    p.close()
