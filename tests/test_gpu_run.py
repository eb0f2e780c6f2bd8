"""The command-line runner: JSON-lines diagnostics, checkpoint and resume."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def runner():
    from paper_1702_07760_gb300 import build as B
    from paper_1702_07760_gb300 import run, sph
    B.build()
    sph.load()
    return run


def test_log_lines_and_conservation(runner, tmp_path):
    log = tmp_path / "a.jsonl"
    assert runner.main(["--workload", "drop_2d", "--steps", "40", "--every", "10", "--log", str(log)]) == 0
    recs = [json.loads(s) for s in log.read_text().splitlines()]
    assert [r["step"] for r in recs] == [0, 10, 20, 30, 40]
    t = [r["t"] for r in recs]
    assert all(b > a for a, b in zip(t, t[1:]))
    m = [r["mass"] for r in recs]
    assert max(abs(x / m[0] - 1) for x in m) < 1e-12      # fluid mass is carried, not integrated
    assert all(r["n_oil"] == recs[0]["n_oil"] > 0 for r in recs)
    assert recs[-1]["centroid"][1] > recs[0]["centroid"][1]  # the drop rises


def test_checkpoint_resume_is_bit_exact(runner, tmp_path):
    """40 steps in one go and 20 + resume + 20 give the same state bit for
    bit (a list build every step, so the particle order is the same)."""
    a, b = tmp_path / "a.npz", tmp_path / "b.npz"
    common = ["--workload", "drop_2d", "--every", "100", "--log", str(tmp_path / "l.jsonl"), "--rebuild-every", "1"]
    assert runner.main(common + ["--steps", "40", "--checkpoint", str(a)]) == 0
    assert runner.main(common + ["--steps", "20", "--checkpoint", str(b)]) == 0
    assert runner.main(["--resume", str(b), "--steps", "20", "--every", "100", "--log", str(tmp_path / "m.jsonl"),
                        "--rebuild-every", "1", "--checkpoint", str(b)]) == 0
    A, B = np.load(a), np.load(b)
    assert int(A["step"]) == int(B["step"]) == 40
    for f in ("x", "u", "rho"):
        assert np.array_equal(A[f], B[f]), f
    assert abs(float(A["t"]) - float(B["t"])) < 1e-15


def test_flume_runner_moves_the_piston(runner, tmp_path):
    log = tmp_path / "f.jsonl"
    ck = tmp_path / "f.npz"
    assert runner.main(["--workload", "wave_tank_small", "--steps", "30", "--every", "15", "--log", str(log),
                        "--checkpoint", str(ck)]) == 0
    c = np.load(ck)
    from paper_1702_07760_gb300 import workloads as WL
    w = WL.wave_tank_small()
    pis = w.wall == 2
    assert np.abs(c["x"][pis, 0] - w.x[pis, 0]).max() > 0


def test_paper_sphere_rises_and_stretches_vertically(runner, tmp_path):
    """The paper's first drop example (0.2 m tank, d = 0.04 m sphere, d_p =
    5 mm, alpha_s = 0.05): by t = 0.42 s it has risen and, as the paper
    describes, lengthened vertically (its oil cloud is taller than wide)."""
    log = tmp_path / "s.jsonl"
    assert runner.main(["--workload", "paper_sphere", "--t-end", "0.42", "--every", "100000",
                        "--log", str(log)]) == 0
    recs = [json.loads(s) for s in log.read_text().splitlines()]
    first, last = recs[0], recs[-1]
    assert abs(last["t"] - 0.42) < 1e-4
    assert last["centroid"][2] - first["centroid"][2] > 0.01        # risen by more than 2 d_p
    assert first["oil_aspect"] < 1.02 and last["oil_aspect"] > 1.1   # taller than wide
    assert last["n_oil"] == first["n_oil"] and abs(last["mass"] / first["mass"] - 1) < 1e-12


def test_drop_3d_diagnostics_every_100_steps(runner, tmp_path):
    """The benchmark workload (656 600 particles) for 300 steps with the
    diagnostics every 100 steps: the FP64 mass is carried exactly, the oil
    count is constant and the drop starts to rise."""
    log = tmp_path / "d.jsonl"
    assert runner.main(["--workload", "drop_3d", "--steps", "300", "--every", "100", "--log", str(log)]) == 0
    recs = [json.loads(s) for s in log.read_text().splitlines()]
    assert [r["step"] for r in recs] == [0, 100, 200, 300]
    assert all(abs(r["mass"] / recs[0]["mass"] - 1) < 1e-12 for r in recs)
    assert all(r["n_oil"] == recs[0]["n_oil"] for r in recs)
    assert recs[-1]["centroid"][2] > recs[0]["centroid"][2]
    assert all(r["u_max"] < 0.1 * 7.92 for r in recs)   # Mach < 0.1 (c0 = 7.92 m/s)
