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


def train(sim, snap_sets, iters: int, lr: float = 1e-3, lr_final: float = 5e-5, seed: int = 0, log_every: int = 0):
    """Adam on random (state, state k steps later) pairs of the recorded
    trajectories with a cosine learning-rate decay; returns the loss history.
    Leaves the handle at the last training state."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = [(si, t) for si, s in enumerate(snap_sets) for t in range(len(s) - 1)]
    hist = []
    for it in range(iters):
        si, t = pairs[rng.integers(len(pairs))]
        s = snap_sets[si]
        sim.load_snapshot(*s.ptrs(t))
        frac = it / max(iters - 1, 1)
        lr_t = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * frac))
        loss, _ = sim.surrogate_train_step(*s.ptrs(t + 1), lr=lr_t, update=True)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"[train] it {it} loss {loss:.4e} lr {lr_t:.2e}", flush=True)
    return np.array(hist)
