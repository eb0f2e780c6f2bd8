"""Pins of the FP64 CPU oracle against facts the paper and the mathematics fix.

Each test checks a property that does not come from re-typing the oracle's
own formula: closed forms, conservation laws the paper claims, reductions
between equations the paper states, library routines, brute force, exact
kinematics, and the physical limits (hydrostatic column, Laplace jump).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1702_07760_gb300 import workloads as WL


def patch(dim=2, shape=(12, 12), seed=3, jitter=0.05, two_phase=True, g=0.0, **kw):
    """Free particle patch (no walls): every particle is a full participant."""
    w = WL.drop_tank(dim, shape, wall_layers=0, seed=seed, jitter_dx=jitter,
                     drop_d_dx=min(shape) * 0.6 if two_phase else 0.0, **kw)
    w.params["g"] = [0.0, 0.0, 0.0] if g == 0.0 else w.params["g"]
    # open box with room around the patch
    for k in range(dim):
        w.params["box_lo"][k] -= 4 * w.params["h"]
        w.params["box_hi"][k] += 4 * w.params["h"]
    return w


# --------------------------------------------------------------------------
# Smoothing kernel (Wendland C2, support 2h)

@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_normalisation(dim):
    h = 1.3e-3
    area = (lambda r: 2 * math.pi * r) if dim == 2 else (lambda r: 4 * math.pi * r * r)
    tot, _ = integrate.quad(lambda r: oracle.W(dim, h, r) * area(r), 0, 2 * h, epsabs=1e-14, epsrel=1e-13)
    assert abs(tot - 1.0) < 1e-10
    # first moment of the gradient: int r dW/dr dV = -dim (int x_a d_b W dV = -delta_ab)
    mom, _ = integrate.quad(lambda r: r * oracle.dWdr(dim, h, r) * area(r), 0, 2 * h,
                            epsabs=1e-14, epsrel=1e-13)
    assert abs(mom + dim) < 1e-9
    # compact support and W(0) = alpha_d
    assert oracle.W(dim, h, 2 * h) == 0.0 and oracle.dWdr(dim, h, 2.0 * h) == 0.0
    alpha = 7 / (4 * math.pi * h * h) if dim == 2 else 21 / (16 * math.pi * h ** 3)
    assert abs(oracle.W(dim, h, 0.0) / alpha - 1) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_derivative_matches_finite_difference(dim):
    h = 1.0
    for r in np.linspace(0.05, 1.95, 39):
        e = 1e-6
        fd = (oracle.W(dim, h, r + e) - oracle.W(dim, h, r - e)) / (2 * e)
        assert abs(fd - oracle.dWdr(dim, h, r)) < 1e-8 * max(1.0, abs(fd))


@pytest.mark.parametrize("dim", [2, 3])
def test_lattice_partition_of_unity(dim):
    """On a perfect lattice sum_j V grad W_ij = 0 (symmetry) and
    sum_j V W_ij ~ 1 (quadrature of the normalised kernel)."""
    dx, h = 1.0, 1.3
    rng = range(-3, 4)
    pts = np.array([p for p in np.ndindex(*([7] * dim))], float) - 3.0
    r = np.linalg.norm(pts, axis=1)
    W = np.array([oracle.W(dim, h, v) for v in r])
    F = np.array([oracle.dWdr(dim, h, v) / v if v > 0 else 0.0 for v in r])
    s = (W * dx ** dim).sum()
    grad = (F[:, None] * (-pts)).sum(axis=0)
    assert np.abs(grad).max() < 1e-14
    assert abs(s - 1.0) < 0.02
    del rng


# --------------------------------------------------------------------------
# Equation of state (Eqs. state and beta)

def test_eos_speed_of_sound_and_exponent():
    w = WL.drop_2d()
    p = w.params
    for ph in (0, 1):
        rho0 = p["rho0"][ph]
        assert oracle.eos(p, ph, rho0) == 0.0
        e = 1e-4 * rho0
        d1 = (oracle.eos(p, ph, rho0 + e) - oracle.eos(p, ph, rho0 - e)) / (2 * e)
        # dP/drho at rho0 is the squared reference sound speed C_s0^2
        assert abs(d1 / p["c0"] ** 2 - 1) < 1e-7
        d2 = (oracle.eos(p, ph, rho0 + e) - 2 * oracle.eos(p, ph, rho0) + oracle.eos(p, ph, rho0 - e)) / e ** 2
        # d2P/drho2 at rho0 = (gamma - 1) C_s0^2 / rho0 pins gamma = 7
        assert abs(d2 / ((7 - 1) * p["c0"] ** 2 / rho0) - 1) < 1e-5
        for pr in (-50.0, 0.0, 3.0, 300.0):
            assert abs(oracle.eos(p, ph, oracle.eos_inverse(p, ph, pr)) - pr) < 1e-9


def test_hydrostatic_density_gives_rho_g_h():
    w = WL.drop_2d()
    p = w.params
    g = 9.81
    for depth in (0.0, 0.004, 0.032):
        rho = oracle.eos_inverse(p, 0, p["rho0"][0] * g * depth)
        assert abs(oracle.eos(p, 0, rho) - p["rho0"][0] * g * depth) < 1e-9


# --------------------------------------------------------------------------
# Neighbour sets, cell ids and the sort permutation

@pytest.mark.parametrize("dim,shape", [(2, (20, 24)), (3, (8, 9, 10))])
def test_neighbours_brute_vs_cells(dim, shape):
    w = WL.drop_tank(dim, shape, quantise=16, seed=7)
    s1, l1 = oracle.neighbours(w.params, w.x, "brute")
    s2, l2 = oracle.neighbours(w.params, w.x, "cells")
    assert np.array_equal(s1, s2) and np.array_equal(l1, l2)
    # symmetric relation, no self
    n = w.n
    rows = np.repeat(np.arange(n), np.diff(s1))
    pairs = set(zip(rows.tolist(), l1.tolist()))
    assert all((j, i) in pairs for i, j in pairs)
    assert all(i != j for i, j in pairs)
    # brute force in numpy
    d2 = ((w.x[:, None, :] - w.x[None, :, :]) ** 2).sum(-1)
    mask = (d2 < (2 * w.params["h"]) ** 2) & ~np.eye(n, dtype=bool)
    assert mask.sum() == len(l1)
    for i in range(0, n, max(1, n // 50)):
        assert np.array_equal(np.nonzero(mask[i])[0], l1[s1[i]:s1[i + 1]])


def test_cell_ids_and_sort_perm_match_library_routines():
    w = WL.drop_tank(3, (10, 11, 12), quantise=16, seed=11)
    p = w.params
    cells = oracle.cell_ids(p, w.x)
    dims = oracle.grid_dims(p)
    c = np.floor((w.x - np.array(p["box_lo"])) / p["cell_size"]).astype(np.int64)
    ref = c[:, 0] + dims[0] * (c[:, 1] + dims[1] * c[:, 2])
    assert np.array_equal(cells, ref)
    perm = oracle.sort_perm(cells)
    assert np.array_equal(perm, np.lexsort((np.arange(w.n), cells)))
    # particles outside the box are reported
    x2 = w.x.copy()
    x2[5, 1] = p["box_hi"][1] + 10 * p["cell_size"]
    assert oracle.cell_ids(p, x2)[5] == -1


# --------------------------------------------------------------------------
# Renormalisation (Eq. ct_dist_3)

def test_renormalisation_invariants():
    w = patch(2, (14, 14), seed=5, jitter=0.2)
    p = w.params
    rho = np.array(p["rho0"])[w.phase].astype(float)
    out = oracle.evaluate(p, w.x, w.u, rho, w.phase, w.wall, renorm=True)
    # every same-phase density equal to its rho0 -> each phase returns its own rho0
    assert np.abs(out["rho"] / rho - 1).max() < 1e-14
    # a phase of uniform density rho_c returns rho_c whatever the other phase holds
    rho2 = rho.copy()
    rho2[w.phase == 1] = 913.0
    rho2[w.phase == 0] = np.linspace(990, 1010, int((w.phase == 0).sum()))
    out2 = oracle.evaluate(p, w.x, w.u, rho2, w.phase, w.wall, renorm=True)
    assert np.abs(out2["rho"][w.phase == 1] / 913.0 - 1).max() < 1e-14
    # without renormalisation the density passes through
    out3 = oracle.evaluate(p, w.x, w.u, rho2, w.phase, w.wall, renorm=False)
    assert np.array_equal(out3["rho"], rho2)


def test_renormalisation_isolated_particle_keeps_density():
    """A particle with no same-phase neighbour: the sums hold only itself."""
    w = patch(2, (9, 9), two_phase=False)
    ph = w.phase.copy()
    centre = np.argmin(np.linalg.norm(w.x - w.x.mean(0), axis=1))
    ph[centre] = 1
    rho = np.full(w.n, 1000.0)
    rho[centre] = 905.5
    out = oracle.evaluate(w.params, w.x, w.u, rho, ph, w.wall, renorm=True)
    assert abs(out["rho"][centre] - 905.5) < 1e-12


def _wall_tank():
    """A one-phase (water) tank with fluid at 1000 and boundary particles at
    1010, and each fluid particle's distance to the nearest boundary particle."""
    w = WL.drop_tank(2, (12, 12), drop_d_dx=4, seed=31)
    walls = w.wall > 0
    rho = np.where(walls, 1010.0, 1000.0)
    x = w.x
    d_fl = np.sqrt(((x[~walls, None, :] - x[None, walls, :]) ** 2).sum(-1)).min(1)
    d_wall = np.sqrt(((x[walls, None, :] - x[None, ~walls, :]) ** 2).sum(-1)).min(1)
    return w, np.zeros(w.n, np.uint8), walls, rho, d_fl, d_wall


def test_renormalisation_of_boundary_particles_as_water():
    """The paper's reading (renorm_walls = 1): dynamic boundary particles share
    the fluid's continuity equation (Sec. III), and Eq. ct_dist_3 is part of
    its discretisation (Sec. II-B), so they are renormalised like water.  A
    Shepard average is a convex combination of the same-phase densities in
    its support: boundary particles with no fluid particle within 2h keep
    1010 exactly, those within 2h of the fluid land strictly between 1000 and
    1010, and likewise for the fluid; a uniform density is returned as is."""
    w, ph, walls, rho, d_fl, d_wall = _wall_tank()
    p = dict(w.params, renorm_walls=1)
    h2 = 2 * p["h"]
    out = oracle.evaluate(p, w.x, w.u, rho, ph, w.wall, renorm=True)
    rw, rf = out["rho"][walls], out["rho"][~walls]
    far_w, near_w = d_wall >= h2 * (1 + 1e-9), d_wall < h2 * (1 - 1e-9)
    assert far_w.any() and near_w.any()
    assert np.abs(rw[far_w] / 1010.0 - 1).max() < 1e-14
    assert np.all(rw[near_w] > 1000.0) and np.all(rw[near_w] < 1010.0)
    far_f, near_f = d_fl >= h2 * (1 + 1e-9), d_fl < h2 * (1 - 1e-9)
    assert np.abs(rf[far_f] / 1000.0 - 1).max() < 1e-14
    assert np.all(rf[near_f] > 1000.0) and np.all(rf[near_f] < 1010.0)
    uni = oracle.evaluate(p, w.x, w.u, np.full(w.n, 1003.0), ph, w.wall, renorm=True)
    assert np.abs(uni["rho"] / 1003.0 - 1).max() < 1e-14


def test_renormalisation_can_leave_boundary_particles_alone():
    """The stabilisation of long runs (renorm_walls = 0): boundary particles
    keep their continuity density (it passes through unchanged), while a
    fluid particle within 2h of a wall still counts the wall particles
    (water) in its Shepard sums; the fluid's values equal those of the
    paper's reading."""
    w, ph, walls, rho, d_fl, _ = _wall_tank()
    p = dict(w.params, renorm_walls=0)
    out = oracle.evaluate(p, w.x, w.u, rho, ph, w.wall, renorm=True)
    assert np.array_equal(out["rho"][walls], rho[walls])
    near, far = d_fl < 2 * p["h"] * (1 - 1e-9), d_fl >= 2 * p["h"] * (1 + 1e-9)
    r = out["rho"][~walls]
    assert far.any() and near.any()
    assert np.abs(r[far] / 1000.0 - 1).max() < 1e-14
    assert np.all(r[near] > 1000.0) and np.all(r[near] < 1010.0)
    lit = oracle.evaluate(dict(w.params, renorm_walls=1), w.x, w.u, rho, ph, w.wall, renorm=True)
    assert np.array_equal(lit["rho"][~walls], r)
    assert not np.array_equal(lit["rho"][walls], rho[walls])


# --------------------------------------------------------------------------
# Continuity (Eqs. ct_dist_1, ct_dist_2)

def test_continuity_reduces_to_single_phase_form():
    """With uniform density Eq. ct_dist_2 equals Eq. ct_dist_1."""
    w = patch(2, (12, 12), two_phase=False, seed=9, jitter=0.1)
    p = w.params
    rng = np.random.default_rng(0)
    u = rng.normal(size=w.u.shape)
    rho = np.full(w.n, 1000.0)
    out = oracle.evaluate(p, w.x, u, rho, w.phase, w.wall, renorm=False)
    s, l = oracle.neighbours(p, w.x)
    ref = np.zeros(w.n)
    for i in range(w.n):
        for j in l[s[i]:s[i + 1]]:
            r = w.x[i] - w.x[j]
            rn = np.linalg.norm(r)
            gw = oracle.dWdr(2, p["h"], rn) / rn * r
            ref[i] += p["mass"][0] * np.dot(u[i] - u[j], gw)
    assert np.abs(out["drho"] - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_continuity_translation_and_divergence(dim):
    shape = (14, 14) if dim == 2 else (9, 9, 9)
    w = patch(dim, shape, two_phase=False, jitter=0.0)
    p = w.params
    rho = np.full(w.n, 1000.0)
    # rigid translation: no compression
    u = np.tile(np.arange(1, dim + 1, dtype=float), (w.n, 1))
    out = oracle.evaluate(p, w.x, u, rho, w.phase, w.wall, renorm=False)
    assert np.abs(out["drho"]).max() < 1e-9
    # linear field u = E x: interior Drho/rho ~ -div u = -trace(E)
    E = np.diag(np.arange(1, dim + 1, dtype=float)) * 10.0
    u = w.x @ E.T
    out = oracle.evaluate(p, w.x, u, rho, w.phase, w.wall, renorm=False)
    c = w.x.mean(0)
    interior = np.all(np.abs(w.x - c) < 1.5 * p["dx"], axis=1)
    ratio = out["drho"][interior] / rho[interior] / (-np.trace(E))
    assert np.all(np.abs(ratio - 1) < 0.03)


# --------------------------------------------------------------------------
# Momentum conservation of the pair terms (pressure Eq. dist_p_1, dynamic
# viscosity Eq. visc_2, surface tension F_s/rho), gravity off

@pytest.mark.parametrize("dim", [2, 3])
def test_pair_terms_conserve_momentum(dim):
    shape = (12, 12) if dim == 2 else (7, 7, 7)
    w = patch(dim, shape, seed=21, jitter=0.15)
    p = w.params
    rng = np.random.default_rng(1)
    rho = np.array(p["rho0"])[w.phase] * (1 + rng.uniform(-0.01, 0.01, w.n))
    u = rng.normal(size=w.u.shape) * 0.1
    out = oracle.evaluate(p, w.x, u, rho, w.phase, w.wall, renorm=False)
    m = np.array(p["mass"])[w.phase]
    ma = m[:, None] * out["a"]
    assert np.abs(ma.sum(0)).max() < 1e-12 * np.abs(ma).sum()
    # angular momentum: pressure alone is a central force
    u0 = np.zeros_like(u)
    p2 = dict(p, alpha_s=0.0)
    out = oracle.evaluate(p2, w.x, u0, rho, w.phase, w.wall, renorm=False)
    ma = m[:, None] * out["a"]
    if dim == 2:
        torque = (w.x[:, 0] * ma[:, 1] - w.x[:, 1] * ma[:, 0]).sum()
        scale = (np.linalg.norm(w.x, axis=1) * np.linalg.norm(ma, axis=1)).sum()
    else:
        tq = np.cross(w.x, ma).sum(0)
        torque = np.abs(tq).max()
        scale = (np.linalg.norm(w.x, axis=1) * np.linalg.norm(ma, axis=1)).sum()
    assert abs(torque) < 1e-12 * scale
    # pressure pushes a compressed pair apart
    x = np.array([[0.0, 0.0], [1.0, 0.0]]) * p["dx"] + 5 * p["h"]
    pp = dict(patch(2, (2, 1), two_phase=False).params, alpha_s=0.0)
    pp["box_lo"] = [0.0, 0.0, 0.0]
    pp["box_hi"] = [20 * p["h"], 20 * p["h"], 0.0]
    out = oracle.evaluate(pp, x, np.zeros((2, 2)), np.array([1001.0, 1001.0]),
                          np.zeros(2, np.uint8), np.zeros(2, np.uint8), renorm=False)
    assert out["a"][0, 0] < 0 < out["a"][1, 0]


# --------------------------------------------------------------------------
# Viscosity (Eqs. kvis, visc_1, visc_2)

def test_viscosity_forms_reduce_to_lo_shao_for_one_phase():
    w = patch(2, (12, 12), two_phase=False, seed=2, jitter=0.1)
    p = dict(w.params, alpha_s=0.0)
    rng = np.random.default_rng(4)
    u = rng.normal(size=w.u.shape)
    rho = np.full(w.n, 1000.0)   # P = 0: only viscosity acts
    a_mu = oracle.evaluate(p, w.x, u, rho, w.phase, w.wall, renorm=False)["a"]
    a_nu = oracle.evaluate(dict(p, visc_form=1), w.x, u, rho, w.phase, w.wall, renorm=False)["a"]
    s, l = oracle.neighbours(p, w.x)
    nu0 = p["mu"][0] / p["rho0"][0]
    ref = np.zeros_like(u)
    for i in range(w.n):
        for j in l[s[i]:s[i + 1]]:
            r = w.x[i] - w.x[j]
            rn = np.linalg.norm(r)
            gw = oracle.dWdr(2, p["h"], rn) / rn * r
            ref[i] += p["mass"][0] * 4 * nu0 / (rho[i] + rho[j]) * np.dot(r, gw) / (rn ** 2 + p["delta"] ** 2) * (u[i] - u[j])
    assert np.abs(a_mu - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(a_nu - ref).max() < 1e-10 * np.abs(ref).max()


def test_viscosity_laplacian_of_parabolic_profile():
    """u_x = y^2 has a Laplacian of 2: interior viscous acceleration ~ 2 nu."""
    w = patch(2, (20, 20), two_phase=False, jitter=0.0)
    p = dict(w.params, alpha_s=0.0)
    rho = np.full(w.n, 1000.0)
    c = w.x.mean(0)
    u = np.zeros_like(w.x)
    u[:, 0] = (w.x[:, 1] - c[1]) ** 2
    a = oracle.evaluate(p, w.x, u, rho, w.phase, w.wall, renorm=False)["a"]
    interior = np.all(np.abs(w.x - c) < 2.5 * p["dx"], axis=1)
    nu = p["mu"][0] / 1000.0
    ratio = a[interior, 0] / (2 * nu)
    assert np.all(np.abs(ratio - 1) < 0.05)
    assert np.abs(a[interior, 1]).max() < 1e-6 * 2 * nu
    # uniform velocity: no viscous force
    a0 = oracle.evaluate(p, w.x, np.ones_like(u), rho, w.phase, w.wall, renorm=False)["a"]
    assert np.abs(a0).max() < 1e-12


def test_harmonic_mean_viscosity_between_phases():
    """Two particles of different phase: the pair force uses
    2 mu_a mu_b / (mu_a + mu_b), symmetric in the pair."""
    h = 1.3e-3
    base = patch(2, (2, 1), two_phase=False).params
    p = dict(base, alpha_s=0.0, h=h, delta=0.1 * h, cell_size=2.05 * h, mass=[1.0, 1.0],
             rho0=[1000.0, 1000.0], mu=[1e-3, 1e-1], box_lo=[0, 0, 0], box_hi=[1, 1, 0])
    x = np.array([[0.5, 0.5], [0.5 + 0.8 * h, 0.5]])
    u = np.array([[0.0, 1.0], [0.0, 0.0]])
    rho = np.array([1000.0, 1000.0])
    a_ab = oracle.evaluate(p, x, u, rho, np.array([0, 1], np.uint8), np.zeros(2, np.uint8), False)["a"]
    p_same = dict(p, mu=[2 * 1e-3 * 1e-1 / (1e-3 + 1e-1)] * 2)
    a_mm = oracle.evaluate(p_same, x, u, rho, np.array([0, 0], np.uint8), np.zeros(2, np.uint8), False)["a"]
    assert np.abs(a_ab - a_mm).max() < 1e-13 * np.abs(a_mm).max()


# --------------------------------------------------------------------------
# Colour gradient (Eq. cd) and surface stress tensor (Eq. csf)

@pytest.mark.parametrize("dim", [2, 3])
def test_colour_gradient_and_tensor_closed_forms(dim):
    shape = (14, 14) if dim == 2 else (8, 8, 8)
    w = patch(dim, shape, seed=8, jitter=0.1)
    p = w.params
    rho = np.array(p["rho0"])[w.phase] * 1.001
    out = oracle.evaluate(p, w.x, w.u, rho, w.phase, w.wall, renorm=False)
    gc, T = out["gradC"], out["T"]
    s, l = oracle.neighbours(p, w.x)
    has_other = np.array([np.any(w.phase[l[s[i]:s[i + 1]]] != w.phase[i]) for i in range(w.n)])
    # zero away from the interface, non-zero on it
    assert np.all(gc[~has_other] == 0.0) and np.all(T[~has_other] == 0.0)
    assert np.all(np.linalg.norm(gc[has_other], axis=1) > 0)
    nrm = np.linalg.norm(gc, axis=1)
    k = has_other
    tr = np.trace(T, axis1=1, axis2=2)
    assert np.abs(tr[k]).max() < 1e-12 * (p["alpha_s"] * nrm[k]).max()
    # T . gradC = alpha_s |gradC| (1/d - 1) gradC
    TgC = np.einsum("nab,nb->na", T, gc)
    ref = p["alpha_s"] * nrm[:, None] * (1 / dim - 1) * gc
    assert np.abs(TgC[k] - ref[k]).max() < 1e-12 * np.abs(ref[k]).max()
    # T is symmetric and its largest eigenvalue magnitude is alpha_s |gradC| (1 - 1/d)
    assert np.abs(T - np.transpose(T, (0, 2, 1))).max() == 0.0
    ev = np.linalg.eigvalsh(T[k])
    assert np.allclose(np.abs(ev).max(1), p["alpha_s"] * nrm[k] * (1 - 1 / dim), rtol=1e-12)
    # the gradient points from the particle towards the other phase
    cen = np.array(w.meta["drop_centre"])
    oil_edge = k & (w.phase == 1)
    assert np.all(np.sum(gc[oil_edge] * (w.x[oil_edge] - cen), axis=1) > 0)
    wat_edge = k & (w.phase == 0)
    assert np.all(np.sum(gc[wat_edge] * (w.x[wat_edge] - cen), axis=1) < 0)


# --------------------------------------------------------------------------
# Integrator (explicit midpoint predictor-corrector)

def test_free_particle_exact_kinematics():
    p = patch(2, (2, 1), two_phase=False).params
    p = dict(p, g=[0.0, -9.81, 0.0], h=0.5, delta=0.05, cell_size=1.025,
             box_lo=[-10.0, -10.0, 0.0], box_hi=[10.0, 10.0, 0.0])
    x0 = np.array([[0.1, 0.2]])
    u0 = np.array([[0.3, 0.7]])
    dt, n = 1e-3, 250
    x, u, rho = oracle.run(p, x0, u0, np.array([1000.0]), np.zeros(1, np.uint8), np.zeros(1, np.uint8), dt, n)
    t = dt * n
    g = np.array([0.0, -9.81])
    assert np.abs(u - (u0 + g * t)).max() < 1e-12
    assert np.abs(x - (x0 + u0 * t + 0.5 * g * t * t)).max() < 1e-12
    assert rho[0] == 1000.0
    # walls do not move
    x, u, _ = oracle.run(p, x0, u0, np.array([1000.0]), np.zeros(1, np.uint8), np.ones(1, np.uint8), dt, 10)
    assert np.array_equal(x, x0) and np.array_equal(u, u0)


# --------------------------------------------------------------------------
# Diagnostics

def test_diagnostics_match_numpy():
    w = WL.drop_tank(3, (10, 10, 16), drop_d_dx=6, seed=4, perturb=True)
    p = w.params
    # stretch the drop into an ellipsoid with axes 1 : 1 : 2
    oil = w.phase == 1
    c = w.x[oil].mean(0)
    x = w.x.copy()
    x[oil, 2] = c[2] + 2 * (x[oil, 2] - c[2])
    d = oracle.diagnostics(p, x, w.u, w.phase, w.wall)
    fl = w.wall == 0
    m = np.array(p["mass"])[w.phase]
    assert abs(d["mass"] - m[fl].sum()) < 1e-12 * d["mass"]
    assert np.allclose(d["momentum"], (m[fl, None] * w.u[fl]).sum(0), rtol=1e-12, atol=1e-18)
    assert abs(d["e_kin"] - 0.5 * (m[fl] * (w.u[fl] ** 2).sum(1)).sum()) < 1e-12 * d["e_kin"]
    assert np.allclose(d["centroid"], x[oil].mean(0), rtol=1e-13)
    ev = np.linalg.eigvalsh(np.cov((x[oil] - x[oil].mean(0)).T, bias=True))
    assert abs(d["sphericity"] - np.sqrt(ev[0] / ev[-1])) < 1e-10
    assert 0.45 < d["sphericity"] < 0.55
    assert d["n_oil"] == int(oil.sum())


# --------------------------------------------------------------------------
# Physical limits: hydrostatic column and Laplace jump (need a relaxation)

def _laplace_jump(dim, n, r_dx, steps, skip, every=10, shell=(1.45, 1.7)):
    """Time-averaged p_in - p_out of a static drop (periodic box, no gravity,
    equal densities, no renormalisation), in units of (dim - 1) alpha_s / R:
    p_in over the particles within R/2 of the drop's centroid, p_out over the
    shell between shell[0] R and shell[1] R (beyond the interface layer of
    width 2h = 2.6 dx), sampled every `every` steps after `skip`."""
    w = WL.static_drop(dim, n, r_dx)
    p = w.params
    x, u, rho = w.x, w.u, w.rho
    dt = WL.stable_dt(p)
    R = w.meta["drop_radius"]
    L = n * p["dx"]
    vals = []
    for k in range(steps // every):
        x, u, rho = oracle.run(p, x, u, rho, w.phase, w.wall, dt, every, first_step=k * every)
        if (k + 1) * every <= skip:
            continue
        P = np.array([oracle.eos(p, 0, r) for r in rho])
        d = x - x[w.phase == 1].mean(0)
        d -= L * np.round(d / L)          # minimum image in the periodic box
        rr = np.linalg.norm(d, axis=1)
        inside, outside = rr < 0.5 * R, (rr > shell[0] * R) & (rr < shell[1] * R)
        vals.append((P[inside].mean() - P[outside].mean()) / ((dim - 1) * p["alpha_s"] / R))
    return float(np.mean(vals))


@pytest.mark.slow
def test_hydrostatic_column_relaxes_to_rho_g_h():
    """Open-top water column (free surface, renormalisation every step):
    mid-depth pressure settles at rho0 g H/2."""
    w = WL.drop_tank(2, (16, 40), drop_d_dx=0.0, seed=2, jitter_dx=0.0, mu=(5e-3, 5e-3), lid=False)
    p = w.params
    depth, g = p["depth"], 9.81
    pr = p["rho0"][0] * g * (depth - w.x[:, 1])
    rho = np.array([oracle.eos_inverse(p, 0, v) for v in pr])
    dt = WL.stable_dt(p)
    x, u = w.x, w.u
    fl = w.wall == 0
    ref = p["rho0"][0] * g * 0.5 * depth
    vals = []
    for k in range(12):
        x, u, rho = oracle.run(p, x, u, rho, w.phase, w.wall, dt, 500, first_step=k * 500)
        if k < 5:
            continue
        P = np.array([oracle.eos(p, 0, r) for r in rho])
        mid = fl & (np.abs(x[:, 1] - 0.5 * depth) < p["dx"]) & (np.abs(x[:, 0] - x[fl, 0].mean()) < 4 * p["dx"])
        vals.append(P[mid].mean() / ref)
    assert abs(np.mean(vals) - 1) < 0.03, vals
    assert np.abs(u[fl]).max() < 0.05 * math.sqrt(g * depth)


@pytest.mark.slow
def test_laplace_pressure_jump_2d():
    """Static 2-D drop: p_in - p_out = alpha_s / R (the jump the CSF tensor of
    Eq. csf must sustain; curvature 1/R).  Without renormalisation (the
    paper: Eq. ct_dist_2 alone suffices without a free surface, Sec. II-B)
    the time-averaged jump is within 10 % of alpha_s / R at R = 8 dx
    (measured 0.95), and it follows the 1/R law: R = 8 dx and R = 12 dx give
    the same jump in units of alpha_s / R within 5 %."""
    m8 = _laplace_jump(2, 40, 8, steps=1000, skip=500)
    m12 = _laplace_jump(2, 56, 12, steps=2000, skip=800)
    assert abs(m8 - 1) < 0.10, m8
    assert abs(m12 - 1) < 0.10, m12
    assert abs(m8 / m12 - 1) < 0.05, (m8, m12)


@pytest.mark.slow
def test_laplace_pressure_jump_3d():
    """Static 3-D drop: p_in - p_out = 2 alpha_s / R (curvature 2/R; the
    isotropic part of T, |grad C|^2 / d I with d = 3, only reshapes the
    pressure inside the interface layer).  Within 10 % at R = 8 dx (measured
    0.97-0.98)."""
    m = _laplace_jump(3, 28, 8, steps=600, skip=300)
    assert abs(m - 1) < 0.10, m
