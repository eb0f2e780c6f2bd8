"""Periodic axes, the piston wave maker and the breaking-wave flume through
the C ABI, against the FP64 oracle (the flume set-up of Sec. "Laboratory
experiment & numerical setup": cross-tank periodic boundary, piston-type
wave maker).

Tolerances as in the drop-rise parity tests: bit-exact cell ids, order and
neighbour sets on grid-quantised positions; 1e-5 relative on single-step
density, density rate and acceleration; positions after a step within 1e-9 dx
(the FP64 integration of FP32 rates over one step), after a few steps within
1e-6 dx.  Positions are compared through the minimum image along a periodic
axis.

In the flume, still water half a metre deep, the acceleration is the small
difference between a pressure gradient and gravity, while each pressure pair
term is of order (P/rho)/h, about 75 g at the bed.  The FP32 sums round at
the size of those terms, so the acceleration error of particle i is held to
the bound of the FP32 arithmetic, (k_i + 8) u S_i with S_i the sum of the
magnitudes of its pair terms (tests/acc_bounds.py), and the per-particle
error against max(|a_i|, |g|) is printed beside it; after one step the
velocity error is held to dt times that bound.
"""
import math

import numpy as np
import pytest

import oracle
from acc_bounds import ROUNDINGS_PER_TERM, U32, acc_error_report, term_magnitudes
from paper_1702_07760_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def sphmod():
    from paper_1702_07760_gb300 import build as B
    from paper_1702_07760_gb300 import sph
    B.build()
    sph.load()
    return sph


def periodic_tank(dim, seed, quantise=None, drift=0.0):
    """Drop tank with its side walls removed along axis 0 (2-D) or 1 (3-D),
    which becomes periodic; the period holds whole super-cells."""
    shape = (36, 30) if dim == 2 else (14, 18, 16)
    axis = 0 if dim == 2 else 1
    w = WL.drop_tank(dim, shape, drop_d_dx=8, seed=seed, perturb=quantise is None, quantise=quantise)
    p = w.params
    dx = p["dx"]
    L = shape[axis] * dx
    keep = (w.x[:, axis] > 0.0 - 0.5 * dx) & (w.x[:, axis] < L + 0.5 * dx) & ~(
        (w.wall == 1) & ((w.x[:, axis] < 0.0) | (w.x[:, axis] > L)))
    x = w.x[keep].copy()
    x[:, axis] = np.mod(x[:, axis], L)
    RL = 2 * p["h"] + 2 * p["skin"]
    msc = int(L // RL)
    p["cell_size"] = L / msc / 2.0
    p["box_lo"][axis], p["box_hi"][axis] = 0.0, L
    p["periodic"] = 1 << axis
    u = w.u[keep].copy()
    u[w.wall[keep] == 0, axis] += drift * p["c0"]
    return WL.Workload(f"periodic_{dim}d", p, np.ascontiguousarray(x), u, w.rho[keep].copy(),
                       w.phase[keep].copy(), w.wall[keep].copy(), dict(w.meta, axis=axis, period=L))


def min_image(d, p):
    d = d.copy()
    for k in range(int(p["dim"])):
        if (int(p.get("periodic", 0)) >> k) & 1:
            L = p["box_hi"][k] - p["box_lo"][k]
            d[:, k] -= L * np.round(d[:, k] / L)
    return d


def rel_field(g, r):
    g = np.asarray(g).reshape(len(g), -1)
    r = np.asarray(r).reshape(len(r), -1)
    return np.linalg.norm(g - r, axis=1).max() / np.linalg.norm(r, axis=1).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_cells_order_and_neighbours_bit_exact(sphmod, dim):
    w = periodic_tank(dim, seed=40 + dim, quantise=16)
    sim = sphmod.Simulation.from_workload(w)
    sim.build_cells()
    cells = sim.read("cell")
    ref_cells = oracle.cell_ids(w.params, w.x)
    assert np.array_equal(cells, ref_cells)
    assert np.array_equal(sim.read("order"), oracle.sort_perm(ref_cells).astype(np.int32))
    s_gpu, l_gpu = sim.neighbours()
    s_ref, l_ref = oracle.neighbours(w.params, w.x, "brute")
    assert np.array_equal(s_gpu, s_ref)
    assert np.array_equal(l_gpu, l_ref)
    # pairs across the periodic boundary are among them
    ax = w.meta["axis"]
    i = np.repeat(np.arange(w.n), np.diff(s_ref))
    assert (np.abs(w.x[i, ax] - w.x[l_ref, ax]) > 0.5 * w.meta["period"]).sum() > 50
    sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_evaluation_matches_oracle(sphmod, dim):
    w = periodic_tank(dim, seed=50 + dim)
    sim = sphmod.Simulation.from_workload(w)
    sim.eval_rates()
    ref = oracle.evaluate(w.params, w.x, w.u, w.rho, w.phase, w.wall, renorm=True)
    fl = w.wall == 0
    e_rho = np.abs(sim.read("rho_eval") / ref["rho"] - 1).max()
    e_a = rel_field(sim.read("acc")[fl], ref["a"][fl])
    e_dr = rel_field(sim.read("drho"), ref["drho"])
    e_T = rel_field(sim.read("tensor"), ref["T"])
    print(f"\n[periodic {dim}d n={w.n}] rho {e_rho:.2e} acc {e_a:.2e} drho {e_dr:.2e} T {e_T:.2e}")
    assert e_rho <= TOL and e_a <= TOL and e_dr <= TOL and e_T <= 1e-4
    sim.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_steps_match_oracle(sphmod, dim):
    """A drift along the periodic axis carries particles across it; the lists
    are rebuilt on the way (positions wrap at each build)."""
    w = periodic_tank(dim, seed=60 + dim, drift=0.05)
    p = w.params
    dt = WL.stable_dt(p)
    n = 30
    sim = sphmod.Simulation.from_workload(w)
    sim.run(dt, n)
    xr, ur, rr = oracle.run(p, w.x, w.u, w.rho, w.phase, w.wall, dt, n)
    x = sim.read("pos")
    ax = w.meta["axis"]
    assert x[:, ax].min() >= 0.0 and x[:, ax].max() < w.meta["period"]
    crossed = (np.abs(xr[:, ax] - w.x[:, ax]) > 0.5 * w.meta["period"]).sum()
    e_x = np.abs(min_image(x - xr, p)).max() / p["dx"]
    e_u = rel_field(sim.read("vel") - w.u, ur - w.u)
    e_r = np.abs(sim.read("rho") / rr - 1).max()
    print(f"\n[periodic {dim}d, {n} steps, {crossed} crossed, {sim.list_builds} builds] "
          f"|dx|/dx {e_x:.2e} du {e_u:.2e} rho {e_r:.2e}")
    assert crossed > 0 and sim.list_builds >= 2
    assert e_x < 1e-6 and e_u < 1e-4 and e_r < TOL
    sim.close()


def pressure_scale(p, ref):
    """a_P = max_i |P_i| / rho_i / h from an oracle evaluation."""
    return float(np.max(np.abs(ref["P"]) / ref["rho"]) / p["h"])


def step_velocity_errors(p, w, ref, u_gpu, u_ref, dt):
    """One step from the state of w: (max over fluid particles of |du_i| /
    (dt (k_i + 8) u S_i), and of |du_i| / (dt max(|a_i|, |g|))), with S_i, k_i
    and a_i those of the rates at the start of the step."""
    S, k = term_magnitudes(p, w.x, w.u, ref["rho"], ref["P"], ref["T"], w.phase, w.wall)
    fl = w.wall == 0
    du = np.linalg.norm(u_gpu[fl] - u_ref[fl], axis=1)
    bound = dt * (k[fl] + ROUNDINGS_PER_TERM) * U32 * S[fl]
    floor = dt * np.maximum(np.linalg.norm(ref["a"][fl], axis=1), np.linalg.norm(p["g"]))
    return float((du / bound).max()), float((du / floor).max())


def piston_tank(seed):
    w = WL.drop_tank(2, (40, 24), drop_d_dx=8, seed=seed, perturb=True)
    wall = w.wall.copy()
    wall[(w.wall == 1) & (w.x[:, 0] < 0.0)] = 2
    p = w.params
    p["box_lo"][0] -= 6 * p["dx"]
    return WL.Workload("piston_tank", p, w.x, w.u, w.rho, w.phase, wall, w.meta)


@pytest.mark.parametrize("persistent", [False, True])
def test_piston_steps_match_oracle(sphmod, persistent):
    w = piston_tank(seed=70)
    p = w.params
    dt = WL.stable_dt(p)
    # a stroke of one dx at up to 0.05 c0 (WCSPH keeps |u| <= 0.1 c0)
    om = 0.1 * p["c0"] / p["dx"]
    m = dict(axis=0, amp=[0.5 * p["dx"]], omega=[om], phase=[-math.pi / 2], t_end=math.pi / om)
    n = int(math.ceil(m["t_end"] / dt)) + 5
    sim = sphmod.Simulation.from_workload(w)
    sim.set_piston(m["axis"], m["amp"], m["omega"], m["phase"], m["t_end"])
    if persistent:
        sim.run_persistent(dt, 40)
        sim.run_persistent(dt, n - 40)
    else:
        sim.run(dt, n)
    xr, ur, rr = oracle.run(p, w.x, w.u, w.rho, w.phase, w.wall, dt, n, piston=m)
    x, u = sim.read("pos"), sim.read("vel")
    pis = w.wall == 2
    t = 0.0
    for _ in range(n):
        t += dt
    assert sim.time == t
    X = oracle.piston_disp(m, t)
    assert abs(X - p["dx"]) < 1e-12  # the stroke is complete (rest after t_end)
    assert np.abs(x[pis] - xr[pis]).max() < 1e-12 * p["dx"]
    assert np.abs(u[pis] - ur[pis]).max() < 1e-12 * p["c0"]
    e_x = np.abs(x - xr).max() / p["dx"]
    e_r = np.abs(sim.read("rho") / rr - 1).max()
    print(f"\n[piston, {n} steps, persistent={persistent}] |dx|/dx {e_x:.2e} rho {e_r:.2e}")
    assert e_x < 1e-6 and e_r < TOL
    sim.close()


def test_flume_small_matches_oracle(sphmod):
    """The scaled flume: periodic across, piston, slope, oil slick; one step
    from rest and a few steps while the piston moves (clock set to 0.3 s)."""
    w = WL.wave_tank_small()
    p, m = w.params, w.meta["piston"]
    dt = WL.stable_dt(p)
    sim = sphmod.Simulation.from_workload(w)
    sim.set_piston(m["axis"], m["amp"], m["omega"], m["phase"], m["t_end"])
    # rates at the initial state
    sim.eval_rates()
    ref = oracle.evaluate(p, w.x, w.u, w.rho, w.phase, w.wall, renorm=True)
    aP = pressure_scale(p, ref)
    e_rho = np.abs(sim.read("rho_eval") / ref["rho"] - 1).max()
    b_a, b_u, e_pp = acc_error_report(p, w.x, w.u, ref, sim.read("acc"), w.phase, w.wall)
    e_T = rel_field(sim.read("tensor"), ref["T"])
    print(f"\n[flume small n={w.n}, rates] a_P = {aP / 9.81:.1f} g; rho {e_rho:.2e} acc per particle "
          f"(floor |g|) {e_pp:.2e}, of the FP32 bound {b_a:.3f} (in u S_i {b_u:.2f}); T {e_T:.2e}")
    assert e_rho < TOL and b_a <= 1.0 and e_T < 1e-4
    sim.step(dt)
    xr, ur, rr = oracle.run(p, w.x, w.u, w.rho, w.phase, w.wall, dt, 1, piston=m)
    e_x = np.abs(min_image(sim.read("pos") - xr, p)).max() / p["dx"]
    b_s, e_s = step_velocity_errors(p, w, ref, sim.read("vel"), ur, dt)
    e_r = np.abs(sim.read("rho") / rr - 1).max()
    print(f"[flume small, 1 step] |dx|/dx {e_x:.2e} du per particle (floor dt |g|) {e_s:.2e}, of the FP32 bound "
          f"{b_s:.3f}; rho {e_r:.2e}")
    assert e_x < 1e-9 and b_s <= 1.0 and e_r < TOL
    # moving piston: state from the oracle's step, clock at 0.3 s
    t0 = 0.3
    u0 = ur.copy()
    u0[w.wall == 2, 0] = oracle.piston_vel(m, t0)
    s2 = sphmod.Simulation(p, xr, u0, rr, w.phase, w.wall)
    s2.set_piston(m["axis"], m["amp"], m["omega"], m["phase"], m["t_end"])
    s2.set_time(t0)
    n = 8
    s2.run(dt, n)
    xr2, ur2, rr2 = oracle.run(p, xr, u0, rr, w.phase, w.wall, dt, n, first_step=1, piston=m, t0=t0)
    pis = w.wall == 2
    assert np.abs(s2.read("pos")[pis] - xr2[pis]).max() < 1e-12
    moved = np.abs(xr2[pis, 0] - xr[pis, 0]).max()
    e_x = np.abs(min_image(s2.read("pos") - xr2, p)).max() / p["dx"]
    e_r = np.abs(s2.read("rho") / rr2 - 1).max()
    print(f"[flume small, {n} steps from t = {t0}] piston moved {moved / p['dx']:.3f} dx; "
          f"|dx|/dx {e_x:.2e} rho {e_r:.2e}")
    assert moved > 1e-3 * p["dx"] and e_x < 1e-6 and e_r < TOL
    sim.close()
    s2.close()


def test_flume_full_size_step_matches_oracle(sphmod):
    """The full flume (4.0 x 0.3 x 0.5 m of water at dx = 5 mm, 4.9 M
    particles), one graph-replayed step as the benchmark runs it, against one
    oracle step of the whole tank; every particle compared."""
    w = WL.wave_tank()
    p, m = w.params, w.meta["piston"]
    dt = WL.stable_dt(p)
    sim = sphmod.Simulation.from_workload(w)
    sim.set_piston(m["axis"], m["amp"], m["omega"], m["phase"], m["t_end"])
    sim.run(dt, 1, graph=True)
    x, u, rho = sim.read("pos"), sim.read("vel"), sim.read("rho")
    sim.close()
    xr, ur, rr = oracle.run(p, w.x, w.u, w.rho, w.phase, w.wall, dt, 1, piston=m)
    ref = oracle.evaluate(p, w.x, w.u, w.rho, w.phase, w.wall, renorm=True)
    aP = pressure_scale(p, ref)
    e_x = np.abs(min_image(x - xr, p)).max() / p["dx"]
    b_s, e_s = step_velocity_errors(p, w, ref, u, ur, dt)
    e_r = np.abs(rho / rr - 1).max()
    print(f"\n[flume full n={w.n}, 1 step] a_P = {aP / 9.81:.1f} g; |dx|/dx {e_x:.2e} du per particle "
          f"(floor dt |g|) {e_s:.2e}, of the FP32 bound {b_s:.3f}; rho {e_r:.2e}")
    assert e_x < 1e-9 and b_s <= 1.0 and e_r < TOL


def test_time_and_suggested_dt(sphmod):
    w = WL.drop_tank(2, (30, 40), drop_d_dx=10, seed=80, perturb=True)
    p = w.params
    sim = sphmod.Simulation.from_workload(w)
    # before any evaluation: the parameter bounds only
    assert sim.suggest_dt() == oracle.suggest_dt(p)
    dt = WL.stable_dt(p)
    sim.run(dt, 5)
    t = 0.0
    for _ in range(5):
        t += dt
    assert sim.time == t
    sim.set_time(1.25)
    assert sim.time == 1.25
    # a strong body force makes the acceleration bound the active one
    q = dict(p, g=[0.0, -2.0e5, 0.0])
    s2 = sphmod.Simulation(q, w.x, w.u, w.rho, w.phase, w.wall)
    s2.eval_rates()
    ref = oracle.evaluate(q, w.x, w.u, w.rho, w.phase, w.wall, renorm=True)
    d_ref = oracle.suggest_dt(q, ref["a"], w.wall)
    assert d_ref < oracle.suggest_dt(q)
    assert abs(s2.suggest_dt() / d_ref - 1) < 1e-5
    sim.close()
    s2.close()


def test_create_from_device_arrays(sphmod):
    import torch
    w = WL.wave_tank_small()
    dev = torch.device("cuda")
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(w, k))).to(dev) for k in ("x", "u", "rho", "phase", "wall")}
    torch.cuda.synchronize()
    a = sphmod.Simulation.from_device(w.params, w.n, t["x"].data_ptr(), t["u"].data_ptr(), t["rho"].data_ptr(),
                                      t["phase"].data_ptr(), t["wall"].data_ptr())
    b = sphmod.Simulation.from_workload(w)
    dt = WL.stable_dt(w.params)
    a.run(dt, 3)
    b.run(dt, 3)
    for f in ("pos", "vel", "rho"):
        assert np.array_equal(a.read(f), b.read(f)), f
    a.close()
    b.close()


def test_surrogate_rejects_piston_handles(sphmod):
    from paper_1702_07760_gb300 import surrogate_layout as SL
    w = WL.wave_tank_small()
    sim = sphmod.Simulation.from_workload(w)
    weights = SL.init_weights(3, seed=1)
    a, b = SL.n_in(3), SL.n_out(3)
    norm = SL.make_norm(3, np.zeros(a), np.ones(a), np.zeros(b), np.ones(b), 50.0, 1e-3, 1.0, 1.0)
    with pytest.raises(sphmod.SphError) as e:
        sim.surrogate_init(weights, norm)
    assert "piston" in str(e.value)
    sim.close()


def test_interface_error_matches_oracle(sphmod):
    """sph_oil_occupancy_diff: the oil occupancy cells of two states and their
    symmetric difference, the same as the oracle's count (integer work,
    FP64 cell decisions on both sides)."""
    w = WL.drop_tank(3, (20, 20, 30), drop_d_dx=10, seed=91, perturb=True)
    p = w.params
    rng = np.random.Generator(np.random.PCG64(92))
    x2 = w.x.copy()
    oil = w.phase == 1
    x2[oil] += rng.uniform(-0.8, 0.8, (oil.sum(), 3)) * p["dx"]
    a = sphmod.Simulation.from_workload(w)
    b = sphmod.Simulation(p, x2, w.u, w.rho, w.phase, w.wall)
    c = sphmod.Simulation.from_workload(w)
    assert a.interface_error(c) == 0.0
    e = b.interface_error(a)
    ref = oracle.interface_error(p, x2, w.x, w.phase, w.wall)
    assert e == ref and e > 0
    for s in (a, b, c):
        s.close()
