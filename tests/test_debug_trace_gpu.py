"""The RFR_DEBUG switch: with RFR_DEBUG=1 in the environment every enqueueing
call synchronises its stream and checks for errors, and results stay
bit-identical to a run without it (the switch changes when errors surface,
not what is computed).  Runs in child processes, since the switch is read
once per process."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, sys, numpy as np, torch
sys.path.insert(0, {root!r})
import siggen
from paper_1812_02200_gb300 import rfr
dev = torch.device("cuda", 0)
c = siggen.pfb_case(1000 * 30, 1000, 8, seed=5)
x = torch.from_numpy(c["x"]).to(dev)
p = rfr.Plan(1000, 4, window="hann", words=c["words"], decimation=500)
F = p.frames_for(x.shape[0])
full = torch.empty((F, 1000), dtype=torch.complex64, device=dev)
tones = torch.empty((8, F), dtype=torch.complex64, device=dev)
p.push_into(x, full, tones)
d = siggen.demod_case(512 * 40, 8, seed=6)
q = rfr.Plan(0, 1024, window="blackman", cutoff=1e-3, words=d["words"], decimation=512)
td = torch.empty((8, q.frames_for(d["x"].shape[0])), dtype=torch.complex64, device=dev)
q.push_into(torch.from_numpy(d["x"]).to(dev), tones=td)
b = rfr.Batch([p])
b.push([x[:5000]], [full], [tones], [0])
tb = torch.empty((4096, 2), dtype=torch.int16, device=dev)
rfr.Tx(d["words"], np.full(8, 500.0)).synthesize(0, tb)
rfr.chirp_synthesize(1 << 60, 77, 1000.0, 0, tb)
torch.cuda.synchronize()
h = hashlib.sha256()
for t in (full, tones, td, tb):
    h.update(t.cpu().numpy().tobytes())
print(h.hexdigest())
"""


def _run(debug):
    env = dict(os.environ)
    env["RFR_DEBUG"] = "1" if debug else "0"
    r = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout.strip().splitlines()[-1]


def test_debug_switch_changes_no_result():
    assert _run(True) == _run(False)
