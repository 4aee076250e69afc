"""The checked build (nvcc -DMDAS_CHECKED: every index read from the pair list
or a lookup table is tested against its array; a failure records an error
instead of an out-of-range access) runs MD with exchange trials, batched
trials, an MDAS move and constant-pressure MD of a small bilayer with no check
firing, and gives the bits of the release build."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json
import numpy as np
from paper_2005_08348_gb300 import mdas, synth
m = synth.mcmd_small()
s = mdas.System(m, precision="fp32")
s.md_steps(60, swap_every=3)
s.swap_trials(64)
r = s.alchemical_move(2, 3, 2)
p = mdas.System(m, precision="fp32", pcouple=dict(nstpcouple=5))
p.md_steps(20, swap_every=2)
h = hashlib.sha256()
for x in (s, p):
    st = x.get_state()
    for k in ("pos_u", "vel", "ltype", "box"):
        h.update(np.ascontiguousarray(st[k]).tobytes())
print(json.dumps({"lib": mdas.library_path(), "hash": h.hexdigest(), "w": r["w"]}))
"""


def _run(checked):
    env = dict(os.environ, MDAS_CHECKED="1" if checked else "0")
    out = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=1200)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_checked_build_runs_clean_and_agrees_with_release():
    rel, chk = _run(False), _run(True)
    assert rel["lib"].endswith("libmdas.so") and chk["lib"].endswith("libmdas_checked.so")
    assert chk["hash"] == rel["hash"] and chk["w"] == rel["w"]
