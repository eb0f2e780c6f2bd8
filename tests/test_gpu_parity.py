"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (FP32 interactions against an FP64 oracle):
* cell ids, sort order and neighbour sets: bit-exact on grid-quantised
  positions (dyadic jitter, so no pair distance lies within FP32 rounding of
  the support radius 2h);
* density after renormalisation and density rate: max over particles of
  |x_gpu - x_ref| / |x_ref| <= 1e-5 (density), and <= 1e-5 of the field's
  largest magnitude (density rate);
* acceleration: max_i |a_gpu,i - a_ref,i| / max_i |a_ref,i| <= 1e-5 (the
  normwise relative error), and per particle the bound of the FP32
  arithmetic, |a_gpu,i - a_ref,i| <= (k_i + 8) u S_i with S_i the sum of the
  magnitudes of particle i's pair terms and u = 2^-24 (tests/acc_bounds.py).
  The per-particle error against max(|a_ref,i|, |g|) is printed: it exceeds
  1e-5 because the pressure sums cancel 50 to 400 times; storing positions
  as int cell + FP32 offset alone (everything else exact) already gives
  1.8e-5 on the 2-D parity state.
"""
import numpy as np
import pytest

import oracle
from acc_bounds import acc_error_report
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


def rel_err_field(gpu, ref):
    """max_i |gpu_i - ref_i| / max_i |ref_i| (vectors: Euclidean norms)."""
    g = np.atleast_2d(gpu.T).T
    r = np.atleast_2d(ref.T).T
    num = np.linalg.norm((g - r).reshape(len(g), -1), axis=1)
    den = np.linalg.norm(r.reshape(len(r), -1), axis=1)
    return num.max() / den.max()


def rel_err_particle(gpu, ref, floor):
    g = np.atleast_2d(gpu.T).T
    r = np.atleast_2d(ref.T).T
    num = np.linalg.norm((g - r).reshape(len(g), -1), axis=1)
    den = np.maximum(np.linalg.norm(r.reshape(len(r), -1), axis=1), floor)
    return (num / den).max()


CASES = {
    "2d_small": lambda: WL.drop_tank(2, (40, 60), drop_d_dx=12, seed=5, perturb=True),
    "2d_cfg": lambda: WL.drop_2d(seed=0, perturb=True),
    "3d_small": lambda: WL.drop_tank(3, (20, 20, 36), drop_d_dx=10, seed=7, perturb=True),
    # kinematic viscosity form (Eq. visc_1): nu = mu / rho0 per phase
    "2d_kinematic": lambda: WL.drop_tank(2, (40, 60), drop_d_dx=12, seed=8, perturb=True, visc_form=1),
    "3d_kinematic": lambda: WL.drop_tank(3, (20, 20, 36), drop_d_dx=10, seed=9, perturb=True, visc_form=1),
    # boundary particles keep their continuity density (the long runs' stabilisation)
    "2d_walls_kept": lambda: WL.drop_tank(2, (40, 60), drop_d_dx=12, seed=5, perturb=True, renorm_walls=0),
    "3d_walls_kept": lambda: WL.drop_tank(3, (20, 20, 36), drop_d_dx=10, seed=7, perturb=True, renorm_walls=0),
}


@pytest.mark.parametrize("case", ["2d_small", "3d_small"])
def test_cells_order_and_neighbours_bit_exact(sphmod, case):
    dim = 2 if case.startswith("2d") else 3
    shape = (37, 53) if dim == 2 else (13, 17, 19)   # ragged sizes, several 256-thread tiles
    w = WL.drop_tank(dim, shape, drop_d_dx=8, seed=13, quantise=16)
    sim = sphmod.Simulation.from_workload(w)
    sim.build_cells()
    cells = sim.read("cell")
    order = sim.read("order")
    ref_cells = oracle.cell_ids(w.params, w.x)
    assert np.array_equal(cells, ref_cells)
    assert np.array_equal(order, oracle.sort_perm(ref_cells).astype(np.int32))
    s_gpu, l_gpu = sim.neighbours()
    s_ref, l_ref = oracle.neighbours(w.params, w.x, "brute")
    assert np.array_equal(s_gpu, s_ref)
    assert np.array_equal(l_gpu, l_ref)
    # the same pairs by class: across phases, two static boundary particles,
    # a static boundary particle with another
    I = np.repeat(np.arange(w.n), np.diff(s_ref))
    J = l_ref.astype(np.int64)
    st = w.wall == 1
    ref_classes = (len(J), int((w.phase[I] != w.phase[J]).sum()), int((st[I] & st[J]).sum()),
                   int((st[I] & ~st[J]).sum()))
    assert sim.pair_classes() == ref_classes
    assert sim.pair_stats() == ref_classes[:2]
    assert ref_classes[2] > 0 and ref_classes[3] > 0
    sim.close()


@pytest.mark.parametrize("case", list(CASES))
def test_single_evaluation_matches_oracle(sphmod, case):
    w = CASES[case]()
    p = w.params
    sim = sphmod.Simulation.from_workload(w)
    sim.eval_rates()
    got = {k: sim.read(k) for k in ("rho_eval", "pressure", "acc", "drho", "tensor")}
    ref = oracle.evaluate(p, w.x, w.u, w.rho, w.phase, w.wall, renorm=True)
    fl = w.wall == 0
    e_rho = np.abs(got["rho_eval"] / ref["rho"] - 1).max()
    e_p = rel_err_field(got["pressure"], ref["P"])
    e_a = rel_err_field(got["acc"][fl], ref["a"][fl])
    b_a, b_u, e_a_pp = acc_error_report(p, w.x, w.u, ref, got["acc"], w.phase, w.wall)
    e_dr = rel_err_field(got["drho"], ref["drho"])
    e_T = rel_err_field(got["tensor"], ref["T"])
    print(f"\n[{case}] n={w.n} rho {e_rho:.2e} P {e_p:.2e} acc {e_a:.2e} (per particle, floor |g|: "
          f"{e_a_pp:.2e}; of the FP32 bound {b_a:.3f}, in u S_i {b_u:.2f}) drho {e_dr:.2e} T {e_T:.2e}")
    assert np.all(got["acc"][~fl] == 0.0)
    assert e_rho <= TOL
    assert e_p <= TOL
    assert e_a <= TOL
    assert b_a <= 1.0
    assert e_dr <= TOL
    assert e_T <= 1e-4
    sim.close()


@pytest.mark.parametrize("visc_form,renorm_walls", [(0, 1), (1, 1), (0, 0)])
def test_one_step_matches_oracle(sphmod, visc_form, renorm_walls):
    w = WL.drop_2d(seed=2, perturb=True, visc_form=visc_form, renorm_walls=renorm_walls)
    p = w.params
    dt = WL.stable_dt(p)
    sim = sphmod.Simulation.from_workload(w)
    sim.step(dt)
    sim.sync()
    x, u, rho = sim.read("pos"), sim.read("vel"), sim.read("rho")
    xr, ur, rr = oracle.run(p, w.x, w.u, w.rho, w.phase, w.wall, dt, 1)
    dx = p["dx"]
    e_x = np.abs(x - xr).max() / dx
    e_u = rel_err_field(u - w.u, ur - w.u)        # velocity increment dt * a*
    e_r = np.abs(rho / rr - 1).max()
    print(f"\n[one step, visc_form {visc_form}, renorm_walls {renorm_walls}] |dx|/dx {e_x:.2e} du {e_u:.2e} "
          f"rho {e_r:.2e}")
    assert e_x < 1e-9
    assert e_u < TOL
    assert e_r < TOL
    sim.close()


def _phases(w, kind, seed):
    """A copy of workload w with its fluid phases replaced: 'water' (one
    phase: no interface anywhere) or 'mixed' (each fluid particle oil with
    probability 1/2: every fluid particle has an other-phase neighbour)."""
    ph = w.phase.copy()
    fl = w.wall == 0
    if kind == "water":
        ph[fl] = 0
    else:
        ph[fl] = np.random.Generator(np.random.PCG64(seed)).integers(0, 2, int(fl.sum()))
    return ph


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", ["water", "mixed"])
def test_degenerate_phase_layouts_two_steps_match_oracle(sphmod, dim, kind):
    """Two steps (both stages, renormalisation, list build) with no
    interface at all, and with every fluid particle next to the other phase
    (the interface pass then takes every particle, one warp each)."""
    w = (WL.drop_tank(2, (30, 40), drop_d_dx=10, seed=21, perturb=True) if dim == 2 else
         WL.drop_tank(3, (12, 13, 16), drop_d_dx=6, seed=22, perturb=True))
    p = w.params
    ph = _phases(w, kind, 23 + dim)
    # the hydrostatic initial density moved to each particle's new phase
    r0 = np.asarray(p["rho0"], np.float64)
    rho0 = w.rho - r0[w.phase] + r0[ph]
    dt = WL.stable_dt(p)
    sim = sphmod.Simulation(p, w.x, w.u, rho0, ph, w.wall)
    sim.run(dt, 2)
    x, u, rho = sim.read("pos"), sim.read("vel"), sim.read("rho")
    T = sim.read("tensor")
    xr, ur, rr = oracle.run(p, w.x, w.u, rho0, ph, w.wall, dt, 2)
    e_x = np.abs(x - xr).max() / p["dx"]
    e_u = rel_err_field(u - w.u, ur - w.u)
    e_r = np.abs(rho / rr - 1).max()
    print(f"\n[{kind} {dim}-D, two steps] |dx|/dx {e_x:.2e} du {e_u:.2e} rho {e_r:.2e}")
    # the second step's positions carry the first step's FP32 velocity
    # increment (dt * a with a relative error ~1e-6)
    assert e_x < 1e-8
    assert e_u < TOL
    assert e_r < TOL
    if kind == "water":
        assert np.all(T == 0.0)
    else:
        assert np.abs(T).max() > 0.0
    sim.close()


def test_graph_replay_is_bit_identical_to_eager(sphmod):
    w = WL.drop_tank(2, (30, 40), drop_d_dx=10, seed=3, perturb=True)
    dt = WL.stable_dt(w.params)
    a = sphmod.Simulation.from_workload(w)
    b = sphmod.Simulation.from_workload(w)
    a.run(dt, 9, graph=False)
    b.run(dt, 9, graph=True)
    for f in ("pos", "vel", "rho"):
        assert np.array_equal(a.read(f), b.read(f)), f
    assert a.step_index == b.step_index == 9


@pytest.mark.parametrize("rebuild_every", [0, 3])
def test_graph_conditional_rebuilds_match_eager(sphmod, rebuild_every):
    """The replayed graph launches the cell-list chain only through its
    conditional node: over many steps with several list builds (decided by
    displacement, or every third step) it matches the eager sequence bit for
    bit and builds the lists on the same steps."""
    w = WL.drop_tank(3, (14, 15, 22), drop_d_dx=8, seed=97, perturb=True)
    p = dict(w.params, rebuild_every=rebuild_every)
    dt = WL.stable_dt(p)
    a = sphmod.Simulation(p, w.x, w.u, w.rho, w.phase, w.wall)
    b = sphmod.Simulation(p, w.x, w.u, w.rho, w.phase, w.wall)
    for k in (1, 7, 40, 12):
        a.run(dt, k, graph=False)
        b.run(dt, k, graph=True)
        assert a.list_builds == b.list_builds
    for f in ("pos", "vel", "rho"):
        assert np.array_equal(a.read(f), b.read(f)), f
    assert a.step_index == b.step_index == 60
    assert b.list_builds >= (20 if rebuild_every == 3 else 1)


def test_advance_host_equals_set_run_read(sphmod):
    """sph_advance_host (upload, steps, read back in one call) gives the bits
    of sph_set_state + sph_run + sph_read_state, in place and into other
    arrays, and rejects bad arguments."""
    w = WL.drop_tank(3, (14, 15, 22), drop_d_dx=8, seed=98, perturb=True)
    dt = WL.stable_dt(w.params)
    a = sphmod.Simulation.from_workload(w)
    b = sphmod.Simulation.from_workload(w)
    a.run(dt, 3)
    b.run(dt, 3)
    x, u, r = a.read("pos"), a.read("vel"), a.read("rho")
    x[:, 0] += 1e-7  # a small move: the lists are kept
    xa, ua, ra = x.copy(), u.copy(), r.copy()
    a.set_state(xa, ua, ra)
    a.run(dt, 4)
    a.read_state(xa, ua, ra)
    xb, ub, rb = x.copy(), u.copy(), r.copy()
    b.advance_host(dt, 4, xb, ub, rb)  # in place
    for p, q in ((xa, xb), (ua, ub), (ra, rb)):
        assert np.array_equal(p, q)
    assert a.step_index == b.step_index == 7
    out = (np.empty_like(x), np.empty_like(u), np.empty_like(r))
    a.advance_host(dt, 2, xa, ua, ra, out=out)
    b.set_state(xb, ub, rb)
    b.run(dt, 2)
    for p, q in zip(out, (b.read("pos"), b.read("vel"), b.read("rho"))):
        assert np.array_equal(p, q)
    with pytest.raises(sphmod.SphError):
        a.advance_host(-dt, 1, xa, ua, ra)
    with pytest.raises(sphmod.SphError):
        a.advance_host(dt, -1, xa, ua, ra)


def test_host_round_trip_matches_device_arrays(sphmod):
    """State uploads and reads through pinned or pageable host memory (staged
    copies) give the bits of the same calls on device arrays (read and written
    in place), for sph_set_state / sph_read_state and sph_advance_host, at a
    size of several thousand 256-thread blocks."""
    import ctypes as C
    import torch
    w = WL.drop_tank(3, (40, 40, 48), drop_d_dx=12, seed=99, perturb=True)
    dt = WL.stable_dt(w.params)
    L = sphmod.load()
    dp = lambda t: C.cast(t.data_ptr(), C.POINTER(C.c_double))
    a = sphmod.Simulation.from_workload(w)
    b = sphmod.Simulation.from_workload(w)
    a.run(dt, 2)
    b.run(dt, 2)
    x, u, r = a.read("pos"), a.read("vel"), a.read("rho")
    x[:, 0] += 1e-7
    pin = lambda v: torch.from_numpy(v).pin_memory().numpy()
    hx, hu, hr = pin(x), pin(u), pin(r)
    a.set_state(hx, hu, hr)
    a.run(dt, 3)
    a.read_state(hx, hu, hr)
    dx, du, dr = (torch.from_numpy(v).cuda() for v in (x, u, r))
    torch.cuda.synchronize()
    sphmod._check(L.sph_set_state(b._h, dp(dx), dp(du), dp(dr)))
    b.run(dt, 3)
    ox, ou, orho = torch.empty_like(dx), torch.empty_like(du), torch.empty_like(dr)
    sphmod._check(L.sph_read_state(b._h, dp(ox), dp(ou), dp(orho)))
    torch.cuda.synchronize()
    for p, q in ((hx, ox), (hu, ou), (hr, orho)):
        assert np.array_equal(p, q.cpu().numpy())
    # the one-call round trip from pageable memory against device arrays
    px, pu, pr = hx.copy(), hu.copy(), hr.copy()
    a.advance_host(dt, 2, px, pu, pr)
    sphmod._check(L.sph_advance_host(b._h, dt, 2, dp(ox), dp(ou), dp(orho), dp(ox), dp(ou), dp(orho)))
    torch.cuda.synchronize()
    for p, q in ((px, ox), (pu, ou), (pr, orho)):
        assert np.array_equal(p, q.cpu().numpy())
    a.close()
    b.close()


def test_restart_is_bit_exact(sphmod):
    """With a list build every step the particle order after a restart is
    the one the uninterrupted run has, so the runs agree bit for bit."""
    w = WL.drop_tank(2, (30, 40), drop_d_dx=10, seed=4, perturb=True)
    p = dict(w.params, rebuild_every=1)
    dt = WL.stable_dt(p)
    a = sphmod.Simulation(p, w.x, w.u, w.rho, w.phase, w.wall)
    a.run(dt, 20)
    b = sphmod.Simulation(p, w.x, w.u, w.rho, w.phase, w.wall)
    b.run(dt, 10)
    x, u, r = b.read("pos"), b.read("vel"), b.read("rho")
    c = sphmod.Simulation(p, x, u, r, w.phase, w.wall)
    c.run(dt, 10)
    for f in ("pos", "vel", "rho"):
        assert np.array_equal(a.read(f), c.read(f)), f
    assert a.list_builds == 20


def _static_walls_moving(w, seed):
    """Velocities of the workload with its static boundary particles given
    seeded values, which they keep (boundary particles do not integrate)."""
    rng = np.random.default_rng(seed)
    u = w.u.copy()
    st = w.wall == 1
    u[st] = rng.uniform(-0.01, 0.01, size=(int(st.sum()), u.shape[1])) * w.params["c0"]
    return u


@pytest.mark.parametrize("case", ["2d_small", "3d_small"])
def test_static_walls_in_motion_take_whole_lists(sphmod, case):
    """While every static boundary particle is at rest, its static boundary
    neighbours sit at the end of its list and the force sweep stops before
    them (their pairs add exact zeros: u_ij = 0, and a boundary particle's
    acceleration is not used); the parity tests above cover that form.  Once
    one moves, those pairs carry u_ij != 0 and the sweep takes whole lists:
    the boundary particles' density rates against the oracle with moving
    walls from the start, and after a state with moving walls is loaded onto
    lists built while they were at rest (set_state keeps the lists), one step
    against the oracle."""
    w = CASES[case]()
    p = w.params
    st = w.wall == 1
    um = _static_walls_moving(w, 11)
    sim = sphmod.Simulation(p, w.x, um, w.rho, w.phase, w.wall)
    sim.eval_rates()
    drho = sim.read("drho")
    sim.close()
    ref = oracle.evaluate(p, w.x, um, w.rho, w.phase, w.wall, renorm=True)
    ref_rest = oracle.evaluate(p, w.x, w.u, w.rho, w.phase, w.wall, renorm=True)
    e_w = rel_err_field(drho[st], ref["drho"][st])
    moved = rel_err_field(ref_rest["drho"][st], ref["drho"][st])   # what the wall-wall pairs add
    dt = WL.stable_dt(p)
    sim = sphmod.Simulation.from_workload(w)
    sim.step(dt)
    b0 = sim.list_builds
    x, u, r = sim.read("pos"), sim.read("vel"), sim.read("rho")
    u[st] = um[st]
    sim.set_state(x, u, r)
    sim.step(dt)
    kept = sim.list_builds == b0
    x1, u1, r1 = sim.read("pos"), sim.read("vel"), sim.read("rho")
    sim.close()
    xr, ur, rr = oracle.run(p, x, u, r, w.phase, w.wall, dt, 1)
    e_x = np.abs(x1 - xr).max() / p["dx"]
    e_u = rel_err_field(u1 - u, ur - u)
    e_r = np.abs(r1 / rr - 1).max()
    e_rw = np.abs(r1[st] - rr[st]).max() / np.abs(rr[st] - r[st]).max()
    print(f"\n[{case}, static walls moving] wall drho {e_w:.2e} (the wall-wall pairs change it by {moved:.2e}); "
          f"after set_state (lists kept: {kept}) |dx|/dx {e_x:.2e} du {e_u:.2e} rho {e_r:.2e}, "
          f"wall density change {e_rw:.2e}")
    assert moved > 1e-2
    assert e_w <= TOL
    assert kept
    assert e_x < 1e-8 and e_u < TOL and e_r < TOL and e_rw < 1e-4


def test_set_state_keeps_valid_lists(sphmod):
    """Loading back the state a handle holds keeps its cell order and list
    (no rebuild) and leaves the trajectory bit for bit unchanged."""
    w = WL.drop_tank(2, (40, 60), drop_d_dx=12, seed=14, perturb=True)
    dt = WL.stable_dt(w.params)
    a = sphmod.Simulation.from_workload(w)
    b = sphmod.Simulation.from_workload(w)
    a.run(dt, 12, graph=False)
    b.run(dt, 12, graph=False)
    for k in range(4):
        x, u, r = b.read("pos"), b.read("vel"), b.read("rho")
        b.set_state(x, u, r)
        b.step(dt)
        a.step(dt)
        assert np.array_equal(a.read("pos"), b.read("pos")), k
        assert a.list_builds == b.list_builds
    for f in ("vel", "rho", "order"):
        assert np.array_equal(a.read(f), b.read(f)), f


@pytest.mark.parametrize("move", ["far", "skin", "nan"])
def test_set_state_rebuilds_when_the_skin_is_exceeded(sphmod, move):
    """A loaded state with a particle beyond the skin test (or non-finite)
    rebuilds; the run then equals one created at that state."""
    w = WL.drop_tank(2, (40, 60), drop_d_dx=12, seed=15, perturb=True)
    p = w.params
    dt = WL.stable_dt(p)
    s = sphmod.Simulation.from_workload(w)
    s.run(dt, 6, graph=False)
    x, u, r = s.read("pos"), s.read("vel"), s.read("rho")
    fluid = np.flatnonzero(w.wall == 0)
    if move == "far":
        x2 = x.copy()                         # two distant fluid particles trade places
        i, j = fluid[0], fluid[-1]
        x2[[i, j]] = x2[[j, i]]
    else:
        x2 = x.copy()
        # every particle is within 0.98 skin of its build position, so a move of
        # 2 skin ends beyond the test whatever the direction of the earlier drift
        x2[fluid[len(fluid) // 2], 0] += 2.0 * p["skin"] if move == "skin" else np.nan
    builds = s.list_builds
    s.set_state(x2, u, r)
    if move == "nan":
        with pytest.raises(sphmod.SphError):
            s.step(dt)
            s.sync()
        return
    s.step(dt)
    s.sync()
    assert s.list_builds == builds + 1
    t = sphmod.Simulation(p, x2, u, r, w.phase, w.wall)
    t.step(dt)
    assert np.allclose(s.read("pos"), t.read("pos"), rtol=0, atol=1e-9 * p["dx"])
    assert np.allclose(s.read("rho"), t.read("rho"), rtol=1e-6, atol=0)


def test_adaptive_list_rebuild_matches_every_step_build(sphmod):
    """The displacement-driven rebuild skips builds and changes only the
    summation order (FP32 rounding), never the neighbour sets."""
    w = WL.drop_tank(2, (40, 60), drop_d_dx=12, seed=6, perturb=True)
    dt = WL.stable_dt(w.params)
    every = sphmod.Simulation(dict(w.params, rebuild_every=1), w.x, w.u, w.rho, w.phase, w.wall)
    adapt = sphmod.Simulation(w.params, w.x, w.u, w.rho, w.phase, w.wall)
    every.run(dt, 30)
    adapt.run(dt, 30)
    assert every.list_builds == 30
    assert 1 <= adapt.list_builds < 30
    dx = w.params["dx"]
    assert np.abs(every.read("pos") - adapt.read("pos")).max() < 1e-6 * dx
    rel = np.abs(every.read("rho") / adapt.read("rho") - 1).max()
    assert rel < 1e-6
    ue, ua = every.read("vel"), adapt.read("vel")
    assert np.abs(ue - ua).max() < 1e-5 * np.abs(ue).max()


def test_diagnostics_match_oracle(sphmod):
    w = WL.drop_tank(3, (16, 16, 24), drop_d_dx=8, seed=9, perturb=True)
    sim = sphmod.Simulation.from_workload(w)
    d = sim.diagnostics()
    r = oracle.diagnostics(w.params, w.x, w.u, w.phase, w.wall)
    assert abs(d["mass"] / r["mass"] - 1) < 1e-12
    assert np.allclose(d["momentum"], r["momentum"], rtol=1e-10, atol=1e-12 * r["mass"])
    assert abs(d["e_kin"] / r["e_kin"] - 1) < 1e-10
    assert abs(d["e_pot"] / r["e_pot"] - 1) < 1e-10
    assert np.allclose(d["centroid"], r["centroid"], rtol=1e-12)
    assert abs(d["sphericity"] - r["sphericity"]) < 1e-9
    assert abs(d["u_max"] - r["u_max"]) < 1e-12
    assert d["n_oil"] == r["n_oil"]


def test_errors_are_reported_not_faulted(sphmod):
    w = WL.drop_tank(2, (20, 20), drop_d_dx=6, seed=1)
    dt = WL.stable_dt(w.params)
    sim = sphmod.Simulation.from_workload(w)
    # a non-finite velocity made on the host
    u = w.u.copy()
    u[np.nonzero(w.wall == 0)[0][0], 0] = np.nan
    sim.set_state(w.x, u, w.rho)
    with pytest.raises(sphmod.SphError) as e:
        sim.run(dt, 2)
    assert e.value.code == -4
    # one particle fast enough that the predictor carries it 1.2 cell edges:
    # beyond the skin whatever its offset in the cell
    sim2 = sphmod.Simulation.from_workload(w)
    u = w.u.copy()
    fl = np.nonzero(w.wall == 0)[0]
    k = fl[np.argmin(np.linalg.norm(w.x[fl] - w.x[fl].mean(0), axis=1))]
    u[k, 0] = 2 * 1.2 * w.params["cell_size"] / dt
    sim2.set_state(w.x, u, w.rho)
    with pytest.raises(sphmod.SphError) as e:
        sim2.run(dt, 1)
    assert e.value.code == -5
    with pytest.raises(sphmod.SphError):
        sim2.step(-1.0)


def test_empty_simulation(sphmod):
    w = WL.drop_tank(2, (4, 4))
    sim = sphmod.Simulation(w.params, w.x[:0], w.u[:0], w.rho[:0], w.phase[:0], w.wall[:0])
    sim.run(1e-6, 3)
    assert sim.read("pos").shape == (0, 2)
    assert sim.step_index == 3


@pytest.mark.slow
def test_200_steps_drift_against_oracle(sphmod):
    """2-D drop rise, 200 steps: FP32 GPU vs FP64 oracle drift report."""
    w = WL.drop_2d(seed=0)
    p = w.params
    dt = WL.stable_dt(p)
    sim = sphmod.Simulation.from_workload(w)
    sim.run(dt, 200)
    x, u, rho = sim.read("pos"), sim.read("vel"), sim.read("rho")
    xr, ur, rr = oracle.run(p, w.x, w.u, w.rho, w.phase, w.wall, dt, 200)
    e_x = np.abs(x - xr).max() / p["dx"]
    e_u = np.abs(u - ur).max() / max(np.abs(ur).max(), 1e-12)
    e_r = np.abs(rho / rr - 1).max()
    dg = sim.diagnostics()
    dr = oracle.diagnostics(p, xr, ur, w.phase, w.wall)
    e_c = np.linalg.norm(dg["centroid"] - dr["centroid"]) / (2 * w.meta["drop_radius"])
    print(f"\n[200 steps] max|dx|/dx {e_x:.2e} u {e_u:.2e} rho {e_r:.2e} centroid/D {e_c:.2e}")
    assert e_x < 1e-4 and e_r < 1e-4 and e_c < 1e-6 and e_u < 1e-2


def test_full_size_3d_evaluation(sphmod):
    """656 600-particle 3-D drop rise, the benchmark's workload and launch
    configuration: single evaluation against the oracle on every particle."""
    w = WL.drop_3d(perturb=True)
    p = w.params
    sim = sphmod.Simulation.from_workload(w)
    sim.eval_rates()
    got_r, got_a, got_d = sim.read("rho_eval"), sim.read("acc"), sim.read("drho")
    ref = oracle.evaluate(p, w.x, w.u, w.rho, w.phase, w.wall, renorm=True)
    fl = w.wall == 0
    e_rho = np.abs(got_r / ref["rho"] - 1).max()
    e_a = rel_err_field(got_a[fl], ref["a"][fl])
    b_a, b_u, e_a_pp = acc_error_report(p, w.x, w.u, ref, got_a, w.phase, w.wall)
    e_dr = rel_err_field(got_d, ref["drho"])
    print(f"\n[3d full n={w.n}] rho {e_rho:.2e} acc {e_a:.2e} (per particle {e_a_pp:.2e}; of the FP32 bound "
          f"{b_a:.3f}, in u S_i {b_u:.2f}) drho {e_dr:.2e}")
    assert e_rho <= TOL and e_a <= TOL and e_dr <= TOL and b_a <= 1.0


def test_pinned_buffers_are_read_and_written_in_place(sphmod):
    """sph_read_state / sph_read into pinned host memory and sph_set_state
    from it give the same values as the pageable path; device arrays are
    read and written in place."""
    import torch
    w = WL.drop_tank(3, (14, 15, 22), drop_d_dx=8, seed=90, perturb=True)
    dt = WL.stable_dt(w.params)
    a = sphmod.Simulation.from_workload(w)
    b = sphmod.Simulation.from_workload(w)
    a.run(dt, 7)
    b.run(dt, 7)
    pin = lambda *s: torch.empty(s, dtype=torch.float64, pin_memory=True).numpy()
    n, d = w.n, 3
    x, u, r = pin(n, d), pin(n, d), pin(n)
    a.read_state(x, u, r)
    assert np.array_equal(x, b.read("pos")) and np.array_equal(u, b.read("vel")) and np.array_equal(r, b.read("rho"))
    acc = pin(n, d)
    a.read("acc", out=acc)
    assert np.array_equal(acc, b.read("acc"))
    # load from pinned (a) and from pageable copies (b), then step both
    x[:, 0] += 0.3 * p_skin(w)
    a.set_state(x, u, r)
    b.set_state(np.array(x), np.array(u), np.array(r))
    a.run(dt, 3)
    b.run(dt, 3)
    for f in ("pos", "vel", "rho", "order"):
        assert np.array_equal(a.read(f), b.read(f)), f
    # device tensors in place
    dx = torch.empty((n, d), dtype=torch.float64, device="cuda")
    from paper_1702_07760_gb300 import sph as S
    import ctypes as C
    S._check(S.load().sph_read(a._h, S.FIELD["pos"], C.c_void_p(dx.data_ptr()), dx.numel() * 8))
    assert np.array_equal(dx.cpu().numpy(), b.read("pos"))
    a.close()
    b.close()


@pytest.mark.parametrize("dim", [2, 3])
def test_pinned_state_reads_in_whole_lines_match_staged_reads(sphmod, dim):
    """Reading the state into pinned host memory (one kernel writes x, u and
    rho in place, x and u in whole lines through shared memory) gives the
    bits of the staged read into pageable arrays: at a particle count whose
    last 256-particle tile is ragged and holds an odd number of doubles, and
    with a pinned x that starts off a 16-byte boundary (which takes the
    staged path).  Loading from pinned memory matches loading from pageable
    copies."""
    import torch
    w = (WL.drop_tank(2, (37, 53), drop_d_dx=10, seed=21, perturb=True) if dim == 2
         else WL.drop_tank(3, (13, 17, 19), drop_d_dx=8, seed=22, perturb=True))
    n = w.n
    assert n % 2 == 1 and n % 256 != 0
    dt = WL.stable_dt(w.params)
    a = sphmod.Simulation.from_workload(w)
    b = sphmod.Simulation.from_workload(w)
    a.run(dt, 3)
    b.run(dt, 3)
    pin = lambda *s: torch.empty(s, dtype=torch.float64, pin_memory=True).numpy()
    x, u, r = pin(n, dim), pin(n, dim), pin(n)
    a.read_state(x, u, r)
    xs, us, rs = np.empty((n, dim)), np.empty((n, dim)), np.empty(n)
    a.read_state(xs, us, rs)
    assert np.array_equal(x, xs) and np.array_equal(u, us) and np.array_equal(r, rs)
    assert np.array_equal(xs, b.read("pos")) and np.array_equal(rs, b.read("rho"))
    big = pin(n * dim + 1)
    xm = big[1:].reshape(n, dim)                  # 8 bytes off a 16-byte boundary
    assert xm.ctypes.data % 16 == 8
    a.read_state(xm, u, r)
    assert np.array_equal(xm, xs)
    # load from pinned memory (a) and from pageable copies (b), then step both
    x[:, 0] += 0.3 * p_skin(w)
    a.set_state(x, u, r)
    b.set_state(np.array(x), np.array(u), np.array(r))
    a.run(dt, 2)
    b.run(dt, 2)
    for f in ("pos", "vel", "rho"):
        assert np.array_equal(a.read(f), b.read(f)), f
    a.close()
    b.close()


def p_skin(w):
    return w.params["skin"]


def test_perturbation_is_seeded_keyed_on_particle_id_and_fluid_only(sphmod):
    """sph_perturb_state: the same seed gives the same state whatever the
    particle order (a handle whose lists were rebuilt in another order), walls
    are untouched, and the velocity noise has the requested spread."""
    w = WL.drop_tank(3, (20, 20, 30), drop_d_dx=10, seed=93, perturb=True)
    a = sphmod.Simulation.from_workload(w)
    b = sphmod.Simulation.from_workload(w)
    b.run(WL.stable_dt(w.params), 3)
    b.set_state(w.x, w.u, w.rho)          # same state, another sorted order
    a.perturb(0.01, 1e-4, 12345)
    b.perturb(0.01, 1e-4, 12345)
    ua, ub = a.read("vel"), b.read("vel")
    assert np.array_equal(ua, ub) and np.array_equal(a.read("rho"), b.read("rho"))
    wl = w.wall == 1
    assert np.array_equal(ua[wl], w.u[wl])
    du = (ua - w.u)[~wl]
    assert abs(du.std() / 0.01 - 1) < 0.02 and abs(du.mean()) < 1e-3
    dr = (a.read("rho") / w.rho - 1)[~wl]
    assert abs(dr.std() / 1e-4 - 1) < 0.05
    a.close()
    b.close()


def test_fp32_peak_measurement_is_plausible(sphmod):
    """sph_fp32_peak (the force sweep's roofline denominator): FMA chains on
    every SM reach a rate between a quarter of and just above the unit-count
    bound (number of SMs x 128 lanes x 2 flops x the maximum SM clock), and
    longer chains give the same rate."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bound = sms * 128 * 2 * 2.2e9 / 1e12
    t1, ms1 = sphmod.fp32_peak(8, 2048)
    t2, ms2 = sphmod.fp32_peak(8, 4096)
    print(f"\n[fp32 peak] {t1:.1f} TFLOP/s ({ms1:.3f} ms), {t2:.1f} TFLOP/s ({ms2:.3f} ms); bound {bound:.1f}")
    assert 0.25 * bound < t1 < bound and 0.25 * bound < t2 < bound
    assert abs(t2 / t1 - 1) < 0.1 and ms2 > 1.5 * ms1
