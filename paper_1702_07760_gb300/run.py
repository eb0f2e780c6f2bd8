"""Command-line runner: advances a workload on the GPU and logs FP64
diagnostics as JSON lines, with checkpoints and resume.

    python -m paper_1702_07760_gb300.run --workload drop_3d --steps 2000 --every 100 --log drop.jsonl
    python -m paper_1702_07760_gb300.run --workload paper_sphere --t-end 1.3 --at 0.42,0.74,1.04,1.22
    python -m paper_1702_07760_gb300.run --workload wave_tank --steps 20000 --every 500 \\
        --checkpoint tank.npz --checkpoint-every 5000
    python -m paper_1702_07760_gb300.run --resume tank.npz --steps 5000

Each log line holds the step, the time, the diagnostics of the C ABI (mass,
momentum, kinetic and potential energy, oil centroid, sphericity, max |u|,
oil count), the oil cloud's vertical and horizontal spread (standard
deviations of the oil positions, from a read of the state) and their ratio,
the list builds so far and the wall-clock seconds; a device error ends the
run with a line naming it (exit status 2).  A checkpoint stores the
state (x, u, rho in original order), the clock and the step count with the
workload's name and seed; resuming rebuilds the workload's phases, walls and
parameters from that name and seed and continues from the stored state (the
device step counter, which only schedules the renormalisation when
renorm_every > 1, restarts at zero).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import sph
from . import workloads as WL

WORKLOADS = {
    "drop_2d": lambda seed: WL.drop_2d(seed=seed),
    "drop_3d": lambda seed: WL.drop_3d(seed=seed),
    "paper_sphere": lambda seed: WL.paper_drop("sphere", seed=seed),
    "paper_cube": lambda seed: WL.paper_drop("cube", seed=seed),
    "wave_tank": lambda seed: WL.wave_tank(seed=seed),
    "wave_tank_small": lambda seed: WL.wave_tank_small(seed=seed),
}
DEFAULT_SEED = {"drop_2d": 0, "drop_3d": 1000, "paper_sphere": 1100, "paper_cube": 1100, "wave_tank": 2000,
                "wave_tank_small": 2100}


def make_workload(name: str, seed: int | None):
    if name not in WORKLOADS:
        raise SystemExit(f"unknown workload {name!r}; choose from {sorted(WORKLOADS)}")
    return WORKLOADS[name](DEFAULT_SEED[name] if seed is None else seed)


def oil_spread(x: np.ndarray, phase: np.ndarray, wall: np.ndarray, dim: int):
    """(vertical std, horizontal std) of the oil particles' positions."""
    oil = (phase == 1) & (wall == 0)
    if not oil.any():
        return 0.0, 0.0
    p = x[oil]
    sv = float(p[:, dim - 1].std())
    sh = float(np.sqrt(np.mean(p[:, :dim - 1].var(axis=0))))
    return sv, sh


def record(sim, w, step: int, t0: float) -> dict:
    d = sim.diagnostics()
    sv, sh = oil_spread(sim.read("pos"), w.phase, w.wall, w.dim)
    return {"step": step, "t": sim.time, "mass": d["mass"], "momentum": d["momentum"].tolist(),
            "e_kin": d["e_kin"], "e_pot": d["e_pot"], "centroid": d["centroid"].tolist(),
            "sphericity": d["sphericity"], "u_max": d["u_max"], "n_oil": d["n_oil"],
            "oil_std_vertical": sv, "oil_std_horizontal": sh, "oil_aspect": sv / sh if sh > 0 else None,
            "list_builds": sim.list_builds, "wall_s": time.perf_counter() - t0}


def save_checkpoint(path: str, sim, name: str, seed: int, step: int):
    np.savez(path, x=sim.read("pos"), u=sim.read("vel"), rho=sim.read("rho"), t=sim.time, step=step,
             workload=name, seed=seed)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="drop_3d")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--steps", type=int, default=None, help="steps to run (default: up to --t-end)")
    ap.add_argument("--t-end", type=float, default=None, help="physical end time (s)")
    ap.add_argument("--dt", type=float, default=None, help="step size (default 0.25 h / c0)")
    ap.add_argument("--every", type=int, default=100, help="log every this many steps")
    ap.add_argument("--at", default="", help="comma-separated times (s) to log at as well")
    ap.add_argument("--log", default="-", help="JSON-lines output ('-' = stdout)")
    ap.add_argument("--checkpoint", default=None, help="checkpoint file written every --checkpoint-every steps")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", default=None, help="checkpoint to continue from")
    ap.add_argument("--rebuild-every", type=int, default=None, help="list rebuild cadence (0: by displacement)")
    ap.add_argument("--persistent", action="store_true", help="advance with the persistent kernel")
    ap.add_argument("--visc-form", type=int, default=None, choices=[0, 1],
                    help="viscous term: 0 dynamic (Eq. visc_2), 1 kinematic (Eq. visc_1)")
    ap.add_argument("--renorm-walls", type=int, default=None, choices=[0, 1],
                    help="1: boundary particles renormalised as water (the paper's reading, default); "
                         "0: they keep their continuity density (the stabilisation of long open-top runs)")
    args = ap.parse_args(argv)

    step0, t_start = 0, 0.0
    if args.resume:
        ck = np.load(args.resume)
        name, seed = str(ck["workload"]), int(ck["seed"])
        w = make_workload(name, seed)
        w.x, w.u, w.rho = ck["x"], ck["u"], ck["rho"]
        step0, t_start = int(ck["step"]), float(ck["t"])
    else:
        name, seed = args.workload, (DEFAULT_SEED.get(args.workload, 0) if args.seed is None else args.seed)
        w = make_workload(name, seed)
    if args.rebuild_every is not None:
        w.params["rebuild_every"] = int(args.rebuild_every)
    if args.visc_form is not None:
        w.params["visc_form"] = int(args.visc_form)
    if args.renorm_walls is not None:
        w.params["renorm_walls"] = int(args.renorm_walls)
    dt = args.dt or WL.stable_dt(w.params)
    if args.steps is None and args.t_end is None:
        raise SystemExit("give --steps or --t-end")
    sim = sph.Simulation.from_workload(w)
    sim.set_time(t_start)
    m = w.meta.get("piston")
    if m is not None:
        sim.set_piston(m["axis"], m["amp"], m["omega"], m["phase"], m["t_end"])
    nsteps = args.steps if args.steps is not None else int(np.ceil((args.t_end - t_start) / dt - 1e-9))
    marks = sorted({int(round((float(a) - t_start) / dt)) for a in args.at.split(",") if a.strip()})
    out = sys.stdout if args.log == "-" else open(args.log, "a")
    t0 = time.perf_counter()
    stops = sorted({k for k in range(0, nsteps + 1, max(args.every, 1))} | {nsteps} |
                   {k for k in marks if 0 <= k <= nsteps} |
                   ({k for k in range(0, nsteps + 1, args.checkpoint_every)} if args.checkpoint_every > 0 else set()))
    done = 0
    for k in stops:
        if k > done:
            try:
                if args.persistent:
                    sim.run_persistent(dt, k - done)
                else:
                    sim.run(dt, k - done)
            except sph.SphError as e:
                # a device error (a particle out of the box, a non-finite value, ...)
                # ends the run with a last line naming it
                out.write(json.dumps({"workload": name, "step_after": step0 + done, "error": str(e)}) + "\n")
                out.flush()
                if out is not sys.stdout:
                    out.close()
                sim.close()
                return 2
            done = k
        rec = record(sim, w, step0 + done, t0)
        rec["workload"] = name
        out.write(json.dumps(rec) + "\n")
        out.flush()
        if args.checkpoint and args.checkpoint_every > 0 and done % args.checkpoint_every == 0 and done > 0:
            save_checkpoint(args.checkpoint, sim, name, seed, step0 + done)
    if args.checkpoint:
        save_checkpoint(args.checkpoint, sim, name, seed, step0 + done)
    if out is not sys.stdout:
        out.close()
    sim.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
