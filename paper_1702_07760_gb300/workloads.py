"""Seeded synthetic inputs for the two-phase SPH particle loop.

This module builds initial states only: particle lattices, wall layers, the
oil drop, the seeded jitter and perturbations, and the physical parameters of
each workload.  It holds none of the method's arithmetic (no kernel, no
equation of state, no rates), so both the CUDA path and the CPU oracle can
consume its arrays.

Workloads (oil drop rising in still water, after the paper's Sec. III
numerical examples, re-sized as synthetic cases):

* ``drop_2d``: 2-D box of 64 x 128 fluid particles, dx = 0.25 mm, three layers
  of dynamic wall particles on every side (9 380 particles), drop diameter
  16 dx centred at (W/2, H/4).
* ``drop_3d``: 3-D box of 64 x 64 x 128 fluid particles with the same
  spacing, fluids and kernel (656 600 particles with walls).

Fluids: water rho0 = 1000 kg/m^3, mu = 1e-3 Pa s; oil rho0 = 900 kg/m^3,
mu = 1e-2 Pa s; tension alpha_s = 0.02 N/m; g = 9.81 m/s^2 along -y (2-D)
or -z (3-D); smoothing length h = 1.3 dx; gamma = 7;
c0 = 10 sqrt(2 g H) with H the fluid depth; particle mass rho0 dx^dim per
phase; delta = 0.1 h.

Initial density is the linearised hydrostatic profile
rho = rho0_phase + rho0_water g (H - y) / c0^2 (a physical initial condition,
not the method's equation of state).  Random numbers come from
``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

WATER, OIL = 0, 1


@dataclass
class Workload:
    name: str
    params: dict
    x: np.ndarray        # (n, dim) float64 positions
    u: np.ndarray        # (n, dim) float64 velocities
    rho: np.ndarray      # (n,) float64 densities
    phase: np.ndarray    # (n,) uint8, 0 water / 1 oil
    wall: np.ndarray     # (n,) uint8, 1 for dynamic boundary particles
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.x)

    @property
    def dim(self) -> int:
        return int(self.params["dim"])

    def copy(self) -> "Workload":
        return Workload(self.name, dict(self.params), self.x.copy(), self.u.copy(),
                        self.rho.copy(), self.phase.copy(), self.wall.copy(), dict(self.meta))


def fluid_params(dim: int, dx: float, depth: float, *, rho0=(1000.0, 900.0),
                 mu=(1e-3, 1e-2), alpha_s=0.02, g=9.81, h_over_dx=1.3,
                 c0=None, visc_form=0, renorm_every=1, renorm_walls=1, skin_h=0.025, cell_h=None) -> dict:
    """Physical and numerical parameters of a drop-rise workload.

    ``renorm_walls`` = 1 renormalises the dynamic boundary particles like
    water (the paper's reading); 0 keeps their continuity density (the
    stabilisation that long runs of the paper's open-top tank select).

    ``skin_h`` is the neighbour-list margin in units of h (the list holds pairs
    closer than 2h + 2 skin); ``cell_h`` is the hashing-cell edge in units of
    h, by default half the list radius, h + skin.
    """
    h = h_over_dx * dx
    if c0 is None:
        c0 = 10.0 * np.sqrt(2.0 * g * depth)
    grav = [0.0, 0.0, 0.0]
    grav[dim - 1] = -g
    skin = skin_h * h
    cell = (cell_h * h) if cell_h is not None else h + skin
    return dict(
        dim=dim, dx=dx, h=h, c0=float(c0), gamma=7.0, delta=0.1 * h,
        alpha_s=float(alpha_s), g=grav, rho0=list(map(float, rho0)), mu=list(map(float, mu)),
        mass=[float(r) * dx ** dim for r in rho0], visc_form=int(visc_form),
        renorm_every=int(renorm_every), renorm_walls=int(renorm_walls), cell_size=cell, skin=skin, depth=depth,
        box_lo=[0.0, 0.0, 0.0], box_hi=[0.0, 0.0, 0.0],
    )


def _lattice(shape, lo_cells: int):
    """Integer lattice coordinates of a box of `shape` cells extended by
    `lo_cells` layers on every side, plus a mask of the interior cells."""
    axes = [np.arange(-lo_cells, s + lo_cells) for s in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    # x fastest in memory order does not matter; keep (x, y[, z]) ordering
    ijk = np.stack([g.ravel(order="F") for g in grids], axis=1)
    inside = np.ones(len(ijk), bool)
    for k, s in enumerate(shape):
        inside &= (ijk[:, k] >= 0) & (ijk[:, k] < s)
    return ijk, inside


def drop_tank(dim: int, shape, dx: float = 2.5e-4, drop_d_dx: float = 16.0,
              drop_centre_frac=None, wall_layers: int = 3, seed: int = 0,
              jitter_dx: float = 1e-3, perturb: bool = False, quantise: int | None = None,
              lid: bool = True, name: str | None = None, drop_shape: str = "sphere", **param_kw) -> Workload:
    """A closed box of fluid lattice `shape` (particles per axis) with an oil
    drop of diameter `drop_d_dx` * dx and `wall_layers` layers of dynamic wall
    particles on every side.

    perturb:  add the parity perturbation (u ~ U(-0.01, 0.01) c0 per component
              on fluid particles, rho *= 1 + U(-1e-3, 1e-3)).
    lid:      keep the wall layers above the fluid (closed box); without
              them the fluid has a free surface at y = H, the side walls rise
              a quarter of the depth above it and the box half the depth.
    quantise: if given, the jitter is drawn as an integer multiple of
              dx / quantise in [-quantise/4, quantise/4] (grid-quantised test
              positions for exact neighbour-set comparisons).
    drop_shape: "sphere" (diameter drop_d_dx dx) or "cube" (side drop_d_dx dx).
    """
    shape = tuple(int(s) for s in shape)
    assert len(shape) == dim
    rng = np.random.Generator(np.random.PCG64(seed))
    depth = shape[dim - 1] * dx
    p = fluid_params(dim, dx, depth, **param_kw)
    if lid:
        ijk, inside = _lattice(shape, wall_layers)
    else:
        # open top: the side walls rise a quarter of the depth above the
        # surface; no lid layers and no particles in the air above the fluid
        nh = int(np.ceil(0.25 * shape[dim - 1]))
        ext = shape[:dim - 1] + (shape[dim - 1] + nh,)
        ijk, inside = _lattice(ext, wall_layers)
        z = ijk[:, dim - 1]
        air = inside & (z >= shape[dim - 1])
        keep = (z < shape[dim - 1] + nh) & ~air
        ijk, inside = ijk[keep], inside[keep]
    x = (ijk + 0.5) * dx
    wall = (~inside).astype(np.uint8)
    fl = inside
    nfl = int(fl.sum())
    if quantise:
        q = int(quantise)
        jit = rng.integers(-(q // 4), q // 4 + 1, size=(nfl, dim)) * (dx / q)
    else:
        jit = rng.uniform(-jitter_dx, jitter_dx, size=(nfl, dim)) * dx
    x[fl] += jit
    if drop_centre_frac is None:
        drop_centre_frac = [0.5] * (dim - 1) + [0.25]
    centre = np.array([f * s * dx for f, s in zip(drop_centre_frac, shape)])
    r_drop = 0.5 * drop_d_dx * dx
    lattice_pos = (ijk + 0.5) * dx
    if drop_shape == "cube":
        in_drop = fl & (np.max(np.abs(lattice_pos - centre), axis=1) < r_drop)
    else:
        in_drop = fl & (np.sum((lattice_pos - centre) ** 2, axis=1) < r_drop ** 2)
    phase = np.where(in_drop, OIL, WATER).astype(np.uint8)
    # linearised hydrostatic initial density
    y = x[:, dim - 1]
    g = abs(p["g"][dim - 1])
    p_h = p["rho0"][WATER] * g * (depth - y)
    rho = np.array(p["rho0"])[phase] + p_h / p["c0"] ** 2
    u = np.zeros_like(x)
    if perturb:
        u[fl] = rng.uniform(-0.01, 0.01, size=(nfl, dim)) * p["c0"]
        rho *= 1.0 + rng.uniform(-1e-3, 1e-3, size=len(rho))
    lo = -wall_layers * dx
    for k in range(dim):
        p["box_lo"][k] = lo
        p["box_hi"][k] = shape[k] * dx + wall_layers * dx
    if not lid:
        # headroom above an open surface: the side walls' height plus a quarter depth
        p["box_hi"][dim - 1] = (shape[dim - 1] + 2 * int(np.ceil(0.25 * shape[dim - 1]))) * dx
    meta = dict(shape=shape, drop_centre=centre.tolist(), drop_radius=r_drop, seed=seed,
                n_fluid=nfl, n_wall=int(wall.sum()), n_oil=int(in_drop.sum()))
    nm = name or f"drop_{dim}d_" + "x".join(map(str, shape))
    return Workload(nm, p, np.ascontiguousarray(x), u, rho, phase, wall, meta)


def drop_2d(seed: int = 0, perturb: bool = False, **kw) -> Workload:
    """2-D oil drop rise: 64 x 128 fluid particles + 3 wall layers (9 380)."""
    return drop_tank(2, (64, 128), seed=seed, perturb=perturb, name="drop_2d_64x128", **kw)


def drop_3d(seed: int = 1000, perturb: bool = False, **kw) -> Workload:
    """3-D oil drop rise: 64 x 64 x 128 fluid particles + 3 wall layers (656 600)."""
    return drop_tank(3, (64, 64, 128), seed=seed, perturb=perturb, name="drop_3d_64x64x128", **kw)


def paper_drop(shape: str = "sphere", seed: int = 1100, **kw) -> Workload:
    """The paper's oil-drop examples (Sec. "Numerical examples on oil-water
    interaction"): a 0.2 m cubic tank filled 0.2 m deep, particle size 5 mm
    (40 x 40 x 40 fluid particles, 3 wall layers, open top), an oil sphere of
    diameter 0.04 m or a cube of side 0.04 m centred 0.04 m above the bottom,
    tension alpha_s = 0.05 N/m."""
    return drop_tank(3, (40, 40, 40), dx=5e-3, drop_d_dx=8.0, drop_centre_frac=[0.5, 0.5, 0.2],
                     lid=False, seed=seed, alpha_s=0.05, drop_shape=shape, name=f"paper_drop_{shape}", **kw)


def static_drop(dim: int, n: int, r_dx: float, dx: float = 2.5e-4, mu: float = 0.2, c0: float = 2.5,
                alpha_s: float = 0.02, renorm_every: int = 0) -> Workload:
    """A drop of radius r_dx dx at the centre of a fully periodic box of n^dim
    particles on a perfect lattice (no walls, no gravity), both fluids of
    density 1000 and viscosity mu, at rest at uniform density: the static
    drop whose pressure jump the surface-tension force must sustain.  mu =
    0.2 Pa s damps the drop's shape oscillations near critically, so the
    pressure field settles within a few hundred steps; c0 = 2.5 m/s keeps
    the flow's Mach number below 0.01.  The cell edge is the box edge over a
    whole number of cells."""
    p = fluid_params(dim, dx, n * dx, rho0=(1000.0, 1000.0), mu=(mu, mu), alpha_s=alpha_s, c0=c0,
                     renorm_every=renorm_every)
    p["g"] = [0.0, 0.0, 0.0]
    axes = [np.arange(n)] * dim
    ijk = np.stack([g.ravel() for g in np.meshgrid(*axes, indexing="ij")], axis=1)
    x = (ijk + 0.5) * dx
    centre = np.full(dim, 0.5 * n * dx)
    r_drop = r_dx * dx
    oil = ((x - centre) ** 2).sum(1) < r_drop ** 2
    p["cell_size"] = n * dx / int(np.floor(n * dx / p["cell_size"] + 1e-9))
    p["periodic"] = (1 << dim) - 1
    p["box_lo"] = [0.0, 0.0, 0.0]
    p["box_hi"] = [n * dx if k < dim else 0.0 for k in range(3)]
    meta = dict(shape=(n,) * dim, drop_centre=centre.tolist(), drop_radius=r_drop, seed=None,
                n_fluid=len(x), n_wall=0, n_oil=int(oil.sum()))
    return Workload(f"static_drop_{dim}d_{n}_r{r_dx:g}", p, np.ascontiguousarray(x), np.zeros_like(x),
                    np.full(len(x), 1000.0), oil.astype(np.uint8), np.zeros(len(x), np.uint8), meta)


def stable_dt(p: dict, cfl: float = 0.25) -> float:
    """Acoustic time step 0.25 h / c0 used by the drop-rise workloads."""
    return cfl * p["h"] / p["c0"]


def drop_batch_2d(k: int = 256, seed: int = 3000, dx: float = 2.5e-4, wall_layers: int = 3,
                  d_range=(8.0, 40.0), mu_ratio_range=(1.0, 100.0), sigma_range=(0.01, 0.05),
                  rho_ratio_range=(0.80, 0.95), perturb: bool = False) -> list:
    """k independent 2-D drop-rise instances of uneven size for the batched form.

    Per instance q, drawn in order from ``Generator(PCG64(seed))``: the drop
    diameter D/dx log-uniform in d_range, the oil/water viscosity ratio
    log-uniform in mu_ratio_range, the tension alpha_s uniform in sigma_range
    and the oil/water density ratio uniform in rho_ratio_range.  The tank is
    4D x 8D of fluid lattice (2 048 to 51 200 fluid particles for D/dx in
    [8, 40]) in a closed box of wall layers, the drop at (W/2, H/4); its
    jitter is seeded with seed + 1 + q.  Water is rho0 = 1000, mu = 1e-3.
    All instances share dx (so h, delta and the cell size); c0 = 10 sqrt(2 g H)
    follows each tank's depth, so each has its own acoustic step.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(k):
        ddx = float(np.exp(rng.uniform(np.log(d_range[0]), np.log(d_range[1]))))
        mu_ratio = float(np.exp(rng.uniform(np.log(mu_ratio_range[0]), np.log(mu_ratio_range[1]))))
        sigma = float(rng.uniform(*sigma_range))
        rho_ratio = float(rng.uniform(*rho_ratio_range))
        shape = (max(4, int(round(4 * ddx))), max(8, int(round(8 * ddx))))
        w = drop_tank(2, shape, dx=dx, drop_d_dx=ddx, wall_layers=wall_layers, seed=seed + 1 + q,
                      perturb=perturb, rho0=(1000.0, 1000.0 * rho_ratio), mu=(1e-3, 1e-3 * mu_ratio),
                      alpha_s=sigma, name=f"drop_batch_{seed}_{q}")
        w.meta.update(drop_d_dx=ddx, mu_ratio=mu_ratio, sigma=sigma, rho_ratio=rho_ratio)
        out.append(w)
    return out


def batch_dt(workloads, cfl: float = 0.25):
    """Common step dt (the largest instance step) and each instance's scale
    dt_q / dt in (0, 1] for a batch advanced together."""
    dts = np.array([stable_dt(w.params, cfl) for w in workloads])
    dt = float(dts.max())
    return dt, dts / dt


# --------------------------------------------------------------------------
# Breaking-wave flume (the set-up of Sec. "Laboratory experiment & numerical
# setup", re-sized as a synthetic case): a long tank, periodic across its
# width, a piston-type wave maker at one end, a 1:10 plane slope at the
# other, and a thin oil slick on the surface where the wave group focuses.
# The piston signal comes from linear wave theory (dispersion relation and
# the piston transfer function), which is input design, not SPH.

def dispersion_k(omega: float, depth: float, g: float = 9.81) -> float:
    """Wavenumber k of linear water waves, omega^2 = g k tanh(k d) (Newton)."""
    k = max(omega * omega / g, omega / np.sqrt(g * depth))
    for _ in range(100):
        t = np.tanh(k * depth)
        f = g * k * t - omega * omega
        df = g * t + g * k * depth * (1.0 - t * t)
        step = f / df
        k -= step
        if abs(step) < 1e-15 * k:
            break
    return float(k)


def piston_transfer(k: float, depth: float) -> float:
    """Wave height over piston stroke, H/S = 2 (cosh 2kd - 1) / (sinh 2kd + 2kd),
    for a piston wave maker in linear theory."""
    a = 2.0 * k * depth
    return float(2.0 * (np.cosh(a) - 1.0) / (np.sinh(a) + a))


def group_velocity(omega: float, k: float, depth: float) -> float:
    a = 2.0 * k * depth
    return float(0.5 * omega / k * (1.0 + a / np.sinh(a)))


def focused_group(seed: int, depth: float, x_focus: float, ncomp: int = 5, f_lo: float = 0.8,
                  f_hi: float = 1.4, crest: float | None = None, g: float = 9.81) -> dict:
    """Piston motion that focuses `ncomp` linear components (frequencies evenly
    spaced in [f_lo, f_hi] Hz, seeded amplitudes summing to `crest`, default
    0.16 depth) at distance x_focus from the piston at time t_f.

    Component c of the surface elevation is a_c cos(k_c (x - x_f) - w_c (t - t_f));
    the piston makes it with displacement (a_c / F_c) sin(w_c t + phi_c),
    phi_c = k_c x_f - w_c t_f, F_c the transfer function.  t_f is the first time
    after the slowest group arrives at which the piston's initial velocity is
    zero, so the motion starts from rest."""
    rng = np.random.Generator(np.random.PCG64(seed))
    crest = 0.16 * depth if crest is None else crest
    f = np.linspace(f_lo, f_hi, ncomp)
    w = rng.uniform(0.5, 1.5, ncomp)
    a = crest * w / w.sum()
    omega = 2.0 * np.pi * f
    k = np.array([dispersion_k(o, depth, g) for o in omega])
    F = np.array([piston_transfer(kk, depth) for kk in k])
    amp = a / F
    u0 = lambda tf: float(np.sum(amp * omega * np.cos(k * x_focus - omega * tf)))
    t0 = x_focus / min(group_velocity(o, kk, depth) for o, kk in zip(omega, k))
    ts = t0 + np.arange(0.0, 4.0, 1e-3)
    vals = np.array([u0(t) for t in ts])
    idx = np.flatnonzero(np.sign(vals[:-1]) != np.sign(vals[1:]))[0]
    lo_t, hi_t = ts[idx], ts[idx + 1]
    for _ in range(80):
        mid = 0.5 * (lo_t + hi_t)
        if np.sign(u0(mid)) == np.sign(u0(lo_t)):
            lo_t = mid
        else:
            hi_t = mid
    t_f = 0.5 * (lo_t + hi_t)
    return dict(axis=0, amp=amp.tolist(), omega=omega.tolist(), phase=(k * x_focus - omega * t_f).tolist(),
                t_end=float("inf"), t_focus=t_f, elevation=a.tolist(), k=k.tolist())


def wave_tank(dx: float = 5e-3, length: float = 4.0, width: float = 0.3, depth: float = 0.5,
              height: float = 0.6, slope: float = 0.1, slope_toe: float = 3.0, x_focus: float = 2.5,
              oil_len: float = 0.3, wall_layers: int = 3, seed: int = 2000, jitter_dx: float = 1e-3,
              name: str | None = None, **param_kw) -> Workload:
    """3-D flume (x along the tank, y across, z up), periodic in y.

    Fluid: the lattice of length x width x depth (cells of dx) above the slope.
    Boundary particles (wall_layers each): the bed below z = 0 (running on
    behind the piston as far as its stroke can take it), the end wall
    beyond x = length, and a plane slope z = slope (x - slope_toe) for
    x > slope_toe (the layers just under it).  The wall layers before x = 0
    are the piston (wall = 2), driven by ``meta["piston"]`` (a focused group,
    see ``focused_group``); the piston and end wall rise to `height`.  Oil:
    the top particle layer over |x - x_focus| < oil_len / 2."""
    nx, ny = int(round(length / dx)), int(round(width / dx))
    nz, nzw = int(round(depth / dx)), int(round(height / dx))
    L = wall_layers
    rng = np.random.Generator(np.random.PCG64(seed))
    p = fluid_params(3, dx, depth, **param_kw)
    # cells tile the period in whole super-cells (two cells of at least h + skin)
    RL = 2.0 * p["h"] + 2.0 * p["skin"]
    msc = int(np.floor(width / RL))
    p["cell_size"] = width / msc / 2.0
    p["periodic"] = 2
    motion = focused_group(seed + 1, depth, x_focus)
    reach = 2.0 * float(np.sum(np.abs(motion["amp"])))      # bound on |X(t)|
    # the bed runs on behind the piston for its whole backward stroke (the
    # water follows the piston face there)
    nb = int(np.ceil(reach / dx)) + 1
    i, j, k = np.meshgrid(np.arange(-L - nb, nx + L), np.arange(ny), np.arange(-L, nzw), indexing="ij")
    i, j, k = i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")
    xc, zc = (i + 0.5) * dx, (k + 0.5) * dx
    zs = np.where(xc > slope_toe, slope * (xc - slope_toe), -np.inf)
    bed = k < 0
    piston = (i >= -L) & (i < 0) & (k >= 0)
    endw = (i >= nx) & (k >= 0)
    inside = (i >= 0) & (i < nx) & (k >= 0)
    slope_layer = inside & (zc < zs) & (zc >= zs - L * dx)
    fluid = inside & (k < nz) & (zc >= zs)
    keep = bed | piston | endw | slope_layer | fluid
    i, j, k, xc, zc = i[keep], j[keep], k[keep], xc[keep], zc[keep]
    wall = np.zeros(len(i), np.uint8)
    wall[(bed | endw | slope_layer)[keep]] = 1
    wall[piston[keep]] = 2
    fl = fluid[keep]
    x = np.stack([xc, (j + 0.5) * dx, zc], axis=1)
    nfl = int(fl.sum())
    x[fl] += rng.uniform(-jitter_dx, jitter_dx, size=(nfl, 3)) * dx
    # stay inside the period after the jitter
    x[:, 1] = np.mod(x[:, 1], width)
    oil = fl & (k == nz - 1) & (np.abs(xc - x_focus) < 0.5 * oil_len)
    phase = np.where(oil, OIL, WATER).astype(np.uint8)
    g = abs(p["g"][2])
    rho = np.array(p["rho0"])[phase] + p["rho0"][WATER] * g * (depth - x[:, 2]) / p["c0"] ** 2
    rho = np.where(wall > 0, p["rho0"][WATER] + p["rho0"][WATER] * g * np.maximum(depth - x[:, 2], 0.0)
                   / p["c0"] ** 2, rho)
    u = np.zeros_like(x)
    p["box_lo"] = [-(L + nb + 1) * dx, 0.0, -L * dx]
    p["box_hi"] = [length + L * dx + dx, width, height + 0.4 * depth]
    meta = dict(piston=motion, n_fluid=nfl, n_wall=int((wall == 1).sum()), n_piston=int((wall == 2).sum()),
                n_oil=int(oil.sum()), depth=depth, length=length, width=width, seed=seed)
    nm = name or f"wave_tank_{nx}x{ny}x{nz}"
    return Workload(nm, p, np.ascontiguousarray(x), u, rho, phase, wall, meta)


def wave_tank_small(seed: int = 2100, **kw) -> Workload:
    """A scaled flume with the same features (dx = 5 mm, 0.6 x 0.06 x 0.1 m
    water, about 31 k particles) for parity against the oracle."""
    args = dict(length=0.6, width=0.06, depth=0.1, height=0.15, slope_toe=0.45, x_focus=0.3, oil_len=0.1,
                seed=seed, name="wave_tank_small")
    args.update(kw)
    return wave_tank(**args)
