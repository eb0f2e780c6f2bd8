"""The bounds-checked build (-DSPH_CHECKED): every index read from device
data is tested before use.  On valid inputs it reports no error and gives the
same bits as the ordinary build (the checks change no arithmetic); it runs in
a child process because a process loads one library."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np
sys.path.insert(0, ROOT)
from paper_1702_07760_gb300 import build as B, sph, workloads as WL
lib = B.build(checked=CHECKED)
sph.load(lib)
out = {}
w = WL.drop_tank(3, (14, 15, 22), drop_d_dx=8, seed=95, perturb=True)
dt = WL.stable_dt(w.params)
a = sph.Simulation.from_workload(w)
a.eval_rates()
out["acc"] = a.read("acc")
a.run(dt, 30)
out["pos"], out["rho"] = a.read("pos"), a.read("rho")
b = sph.Simulation.from_workload(w)
b.run_persistent(dt, 30)
out["pos_p"] = b.read("pos")
ws = WL.drop_batch_2d(k=4, seed=96, d_range=(5.0, 8.0), perturb=True)
dtb, sc = WL.batch_dt(ws)
c = sph.Simulation.batch(ws)
c.set_dt_scales(sc)
c.run_persistent(dtb, 20)
out["pos_b"] = c.read("pos")
f = WL.wave_tank_small()
m = f.meta["piston"]
s = sph.Simulation.from_workload(f)
s.set_piston(m["axis"], m["amp"], m["omega"], m["phase"], m["t_end"])
s.run(WL.stable_dt(f.params), 5)
out["pos_f"] = s.read("pos")
np.savez(OUT, **out)
"""


def _run(tmp_path, checked: bool):
    out = tmp_path / f"{'checked' if checked else 'plain'}.npz"
    code = CHILD.replace("ROOT", repr(ROOT)).replace("CHECKED", str(checked)).replace("OUT", repr(str(out)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_checked_build_matches_the_ordinary_build(tmp_path):
    a = _run(tmp_path, False)
    b = _run(tmp_path, True)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
