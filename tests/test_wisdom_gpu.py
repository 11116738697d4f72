"""Autotune results persist across processes in the file GBFFT_WISDOM names
(runtime validation of the model, Sec. 3.2, done once per device and shape):
a first process tunes a plan and appends its choice; a fresh process with the
same file reads that choice instead of timing candidates again, and the plan
it builds computes the same transform."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

CHILD = r"""
import json, sys
sys.path.insert(0, {root!r})
import numpy as np, torch
from paper_1505_08067_gb300 import gbfft, synth
out = {{}}
for n, batch in ((1024, 64), (2 ** 20, 4)):
    x = torch.from_numpy(synth.uniform(31, batch, n)).cuda()
    with gbfft.Plan(n, batch, -1, autotune=1) as p:
        y = p.execute(x).cpu().numpy()
        out[str(n)] = {{"tuning": p.describe().get("tuning"),
                        "checksum": [float(np.abs(y).sum()), float(y.real.sum())]}}
print(json.dumps(out))
"""


def _child(env):
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_wisdom_file_written_and_read_back(tmp_path):
    path = tmp_path / "wisdom.txt"
    env = dict(os.environ, GBFFT_WISDOM=str(path))
    first = _child(env)
    assert path.exists()
    lines = path.read_text().splitlines()
    assert len(lines) >= 2 and all("|" in ln for ln in lines)
    second = _child(env)
    for n in ("1024", str(2 ** 20)):
        t1, t2 = first[n]["tuning"], second[n]["tuning"]
        assert "chosen" in t1 and "candidates" in t1, t1
        assert "cached" in t2 and "candidates" not in t2, t2
        assert t2["cached"] == t1["chosen"]
        a, b = first[n]["checksum"], second[n]["checksum"]
        assert abs(a[0] - b[0]) <= 1e-5 * abs(a[0]) and abs(a[1] - b[1]) <= 1e-4 * abs(a[0])
    assert path.read_text().splitlines() == lines      # nothing tuned twice
    # entries keyed by another build of the library are not reused
    path.write_text("".join("stale-build/" + ln.split("/", 1)[1] + "\n" for ln in lines))
    third = _child(env)
    for n in ("1024", str(2 ** 20)):
        assert "candidates" in third[n]["tuning"], third[n]["tuning"]
