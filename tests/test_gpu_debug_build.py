"""The MACE_DEBUG build (libmace_debug.so, device-side bounds checks on the
indices the kernels read from stored data): on valid inputs no check fires
and the reconstructions equal the release build's, for the fixed schedule
with two chains (FP32 and BF16 matrices), the work-queue schedule, and a
team of two warps on an agent of 150 views.  Run in a child process (MACE_DEBUG=1 selects the library when
the binding loads)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(tests)r)
from paper_1911_09278_gb300 import build as gbuild
gbuild.build(debug=%(debug)s)
import paper_1911_09278_gb300 as mace
from helpers import case
out = {"lib": mace.LIB_PATH}
# 22-23 views per agent (the kernels that decode one column ahead), and one
# agent of 150 views (the decode-at-use kernels, a team of two warps)
for name, V, N, dtype, kw in [("fixed", 90, 4, "f32", dict(chains=2)), ("bf16", 90, 4, "bf16", dict(chains=2)),
                              ("queue", 90, 4, "f32", dict(schedule=1)),
                              ("team", 150, 1, "f32", dict(schedule=1, warps_per_voxel=2))]:
    c = case(64, V, 95, N, "qggmrf")
    sm = mace.mace_build_sysmatrix(64, 64, V, 95, N, dtype=dtype, sv_size=4)
    prm = mace.make_params(prior="qggmrf", sigma_x=c["sigma_x"], sigma=0.3, sigma_mode=1, concurrency=1,
                           sweeps_per_iter=2, symmetric=True, recompute_every=10, **kw)
    y = np.stack([c["y"]] * 2)
    lam = np.stack([c["lam"]] * 2)
    st = mace.mace_init(sm, y, lam, prm, batch=2)
    r, conv = st.iterate(40)
    out[name] = np.asarray(st.consensus(), np.float64).ravel().tolist()
    st.close()
    sm.close()
print("RESULT " + json.dumps(out))
"""


def _run(debug):
    env = dict(os.environ)
    env["MACE_DEBUG"] = "1" if debug else "0"
    code = SCRIPT % dict(root=ROOT, tests=os.path.join(ROOT, "tests"), debug=debug)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_debug_build_matches_release():
    dbg, rel = _run(True), _run(False)
    assert dbg["lib"].endswith("libmace_debug.so") and rel["lib"].endswith("libmace.so")
    for name in ("fixed", "bf16", "queue", "team"):
        a, b = np.array(dbg[name]), np.array(rel[name])
        err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        print("%s: debug vs release relative difference %.1e" % (name, err))
        assert err < 1e-5, name
