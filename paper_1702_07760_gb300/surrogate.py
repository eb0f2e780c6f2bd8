"""Training data, normalisation and training loop of the learned k-step
surrogate.

Every arithmetic step of the network (forward, backward, Adam) runs in
libsph (include/sph_surrogate.h); this module only orchestrates it: it records
snapshots of plain-SPH trajectories into device memory (torch tensors in
original particle order), derives the normalisation block from them, and
feeds (state, state k steps later) pairs to the training entry point.
"""
from __future__ import annotations

import numpy as np

from . import surrogate_layout as SL


class Snapshots:
    """States of one trajectory every k plain steps, on the device, with the
    plain method's rates at each state on the host (for normalisation)."""

    def __init__(self, torch, n: int, dim: int, count: int, device="cuda"):
        self.torch = torch
        self.x = torch.zeros((count, n, dim), dtype=torch.float64, device=device)
        self.u = torch.zeros((count, n, dim), dtype=torch.float64, device=device)
        self.r = torch.zeros((count, n), dtype=torch.float64, device=device)
        self.a = np.zeros((count, n, dim))
        self.drdt = np.zeros((count, n))
        self.count = 0

    def ptrs(self, t: int):
        return self.x[t].data_ptr(), self.u[t].data_ptr(), self.r[t].data_ptr()

    def __len__(self):
        return self.count


def record(sim, dt: float, k: int, count: int, torch, warmup_steps: int = 0) -> Snapshots:
    """Runs the plain method and keeps the state every k steps (count states)."""
    if warmup_steps:
        sim.run(dt, warmup_steps)
    snaps = Snapshots(torch, sim.n, sim.dim, count)
    for t in range(count):
        if t:
            sim.run(dt, k)
        sim.snapshot_to(*snaps.ptrs(t))
        sim.eval_rates()
        snaps.a[t] = sim.read("acc")
        snaps.drdt[t] = sim.read("drho")
        snaps.count = t + 1
    torch.cuda.synchronize()
    return snaps


def fit_norm(params: dict, phase, wall, snap_sets, k_ref: float, t_jump: float) -> np.ndarray:
    """Normalisation block from recorded trajectories (every k plain steps,
    t_jump = k dt apart): inputs (velocity, density deviation, explicit jumps
    of the rates) and outputs (the corrections to the trapezoid rule and to
    the explicit jumps) scaled to unit spread over fluid particles;
    the phase and wall flags pass unscaled; the edge state differences are
    scaled by their spread over neighbour pairs closer than 2h in the last
    state of the first trajectory."""
    from scipy.spatial import cKDTree

    dim = int(params["dim"])
    rho0 = np.asarray(params["rho0"], float)[phase]
    fl = wall == 0
    T = t_jump
    us, drs, tas, tds, cxs, dus, ddrs = [], [], [], [], [], [], []
    for s in snap_sets:
        x = s.x[:s.count].cpu().numpy()
        u = s.u[:s.count].cpu().numpy()
        r = s.r[:s.count].cpu().numpy()
        a, drdt = s.a[:s.count], s.drdt[:s.count]
        us.append(u[:, fl].reshape(-1, dim))
        drs.append(((r - rho0) / rho0)[:, fl].ravel())
        tas.append((T * a)[:, fl].reshape(-1, dim))
        tds.append((T * drdt / rho0).ravel())
        corr = (x[1:] - x[:-1]) - 0.5 * T * (u[1:] + u[:-1])
        cxs.append(corr[:, fl].reshape(-1, dim))
        dus.append((u[1:] - u[:-1] - T * a[:-1])[:, fl].reshape(-1, dim))
        ddrs.append(((r[1:] - r[:-1]) / rho0 - T * drdt[:-1] / rho0).ravel())
    u, dr = np.concatenate(us), np.concatenate(drs)
    ta, td = np.concatenate(tas), np.concatenate(tds)
    cx, du, ddr = np.concatenate(cxs), np.concatenate(dus), np.concatenate(ddrs)
    tiny = 1e-30
    mu_in = np.concatenate([np.zeros(dim), [dr.mean()], [0.0, 0.0], ta.mean(0), [td.mean()]])
    sd_in = np.concatenate([np.full(dim, max(u.std(), tiny)), [max(dr.std(), tiny)], [1.0, 1.0],
                            np.maximum(ta.std(0), tiny), [max(td.std(), tiny)]])
    mu_out = np.concatenate([cx.mean(0), du.mean(0), [ddr.mean()]])
    sd_out = np.concatenate([np.maximum(cx.std(0), tiny), np.maximum(du.std(0), tiny), [max(ddr.std(), tiny)]])
    s0 = snap_sets[0]
    t = s0.count - 1
    x0, u0, r0 = s0.x[t].cpu().numpy(), s0.u[t].cpu().numpy(), s0.r[t].cpu().numpy()
    pairs = cKDTree(x0).query_pairs(2.0 * params["h"], output_type="ndarray")
    delta = (r0 - rho0) / rho0
    sd_eu = max(float((u0[pairs[:, 0]] - u0[pairs[:, 1]]).std()), tiny)
    sd_er = max(float((delta[pairs[:, 0]] - delta[pairs[:, 1]]).std()), tiny)
    return SL.make_norm(dim, mu_in, sd_in, mu_out, sd_out, k_ref, t_jump, sd_eu, sd_er)


def increment_scales(snaps: Snapshots, wall) -> tuple[float, float]:
    """RMS over the fluid particles of the velocity and relative density
    changes between consecutive snapshots (one jump)."""
    torch = snaps.torch
    fl = torch.as_tensor(np.asarray(wall) == 0, device=snaps.u.device)
    du = snaps.u[1:snaps.count] - snaps.u[:snaps.count - 1]
    dr = (snaps.r[1:snaps.count] - snaps.r[:snaps.count - 1]) / snaps.r[:snaps.count - 1]
    return (float(du[:, fl].pow(2).mean().sqrt()), float(dr[:, fl].pow(2).mean().sqrt()))


def train(sim, snap_sets, iters: int, lr: float = 1e-3, lr_final: float = 5e-5, seed: int = 0, log_every: int = 0,
          noise: tuple[float, float] | None = None):
    """Adam on random (state, state k steps later) pairs of the recorded
    trajectories with a cosine learning-rate decay; returns the loss history.
    With noise = (sigma_u, sigma_rho) the input state of every pair is
    perturbed (sph_perturb_state) while the target stays the recorded one, so
    the network also learns to correct states a little off the trajectory
    (the input noise of learned particle simulators).  Leaves the handle at
    the last training state."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = [(si, t) for si, s in enumerate(snap_sets) for t in range(len(s) - 1)]
    hist = []
    for it in range(iters):
        si, t = pairs[rng.integers(len(pairs))]
        s = snap_sets[si]
        sim.load_snapshot(*s.ptrs(t))
        if noise is not None:
            sim.perturb(noise[0], noise[1], seed * 1_000_003 + it)
        frac = it / max(iters - 1, 1)
        lr_t = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * frac))
        loss, _ = sim.surrogate_train_step(*s.ptrs(t + 1), lr=lr_t, update=True)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"[train] it {it} loss {loss:.4e} lr {lr_t:.2e}", flush=True)
    return np.array(hist)


def _time_main(argv=None):
    """Times surrogate jumps (and optionally training steps) on a drop-rise
    workload with seeded random weights and a fixed normalisation:

        python -m paper_1702_07760_gb300.surrogate --workload drop_3d --jumps 3 --train-steps 0
    """
    import argparse
    import json
    import time

    import torch

    from . import build as B
    from . import sph
    from . import workloads as WL

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="drop_3d", choices=["drop_3d", "drop_3d_32x32x128", "drop_2d"])
    ap.add_argument("--jumps", type=int, default=3)
    ap.add_argument("--train-steps", type=int, default=0)
    a = ap.parse_args(argv)
    B.build()
    sph.load()
    torch.cuda.set_device(0)
    if a.workload == "drop_3d":
        w = WL.drop_3d()
    elif a.workload == "drop_2d":
        w = WL.drop_2d()
    else:
        w = WL.drop_tank(3, (32, 32, 128), drop_d_dx=16, seed=5, name="drop_3d_32x32x128")
    dim = w.dim
    dt = WL.stable_dt(w.params)
    n_in, n_out = SL.n_in(dim), SL.n_out(dim)
    norm = SL.make_norm(dim, np.zeros(n_in), np.ones(n_in), np.zeros(n_out), np.full(n_out, 1e-6),
                        80.0 if dim == 3 else 20.0, 8 * dt, 1e-3, 1e-4)
    sim = sph.Simulation.from_workload(w)
    sim.surrogate_init(SL.init_weights(dim, seed=1, out_scale=1e-3), norm)
    out = {"workload": a.workload, "particles": w.n}
    if a.jumps:
        sim.surrogate_advance(8)
        sim.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.jumps):
            sim.surrogate_advance(8)
        sim.sync()
        out["ms_per_jump"] = (time.perf_counter() - t0) / a.jumps * 1e3
    if a.train_steps:
        tx, tu, tr = (torch.tensor(v, dtype=torch.float64, device="cuda") for v in (w.x, w.u, w.rho))
        ptr = (tx.data_ptr(), tu.data_ptr(), tr.data_ptr())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.train_steps):
            sim.load_snapshot(*ptr)
            sim.surrogate_train_step(*ptr, lr=1e-6)
        torch.cuda.synchronize()
        out["ms_per_train_step"] = (time.perf_counter() - t0) / a.train_steps * 1e3
    sim.close()
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    _time_main()
