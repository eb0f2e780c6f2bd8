"""Workloads and pins against the values the paper prints (tests/golden/
paper_values.txt, each line with the section it comes from)."""
import math
import os

import numpy as np

import oracle
from paper_1702_07760_gb300 import workloads as WL

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_values.txt")):
        line = line.split("|")[0].strip()
        if not line or line.startswith("#"):
            continue
        key, val = (t.strip() for t in line.split("=", 1))
        nums = [float(v) for v in val.split() if not v.startswith("[")]
        out[key] = nums if len(nums) > 1 else nums[0]
    return out


G = golden()


def test_tait_exponent():
    for w in (WL.drop_2d(), WL.paper_drop("sphere"), WL.wave_tank_small()):
        assert w.params["gamma"] == G["tait_gamma"]


def test_paper_drop_examples_use_the_printed_set_up():
    for shape, size_key in (("sphere", "drop_sphere_diameter"), ("cube", "drop_cube_side")):
        w = WL.paper_drop(shape)
        p, dx = w.params, w.params["dx"]
        assert dx == G["drop_particle_size"]
        assert p["alpha_s"] == G["drop_alpha_s"]
        fl = w.wall == 0
        # the fluid lattice fills the printed depth (cell centres from dx/2 to depth - dx/2)
        assert abs(w.x[fl, 2].max() + dx / 2 - G["drop_water_depth"]) < 0.1 * dx
        oil = (w.phase == 1) & fl
        extent = w.x[oil, 2].max() - w.x[oil, 2].min() + dx
        assert abs(extent - G[size_key]) < 1.01 * dx


def test_piston_stroke_from_the_printed_formula():
    S, f, T = G["piston_stroke"], G["piston_frequency"], G["piston_duration"]
    m = dict(axis=0, amp=[S / 2], omega=[2 * math.pi * f], phase=[-math.pi / 2], t_end=T)
    assert abs(oracle.piston_disp(m, 0.0)) < 1e-15
    assert abs(oracle.piston_disp(m, T / 2) - S / 2) < 1e-12
    assert abs(oracle.piston_disp(m, T) - S) < 1e-12     # the full stroke at the end of the signal
    assert oracle.piston_disp(m, 2 * T) == oracle.piston_disp(m, T)


def test_flume_width_periodicity_and_particle_size():
    for w in (WL.wave_tank_small(),):
        p = w.params
        assert p["periodic"] == 2                                      # the cross-tank (y) axis
        assert abs(p["box_hi"][1] - p["box_lo"][1] - 0.06) < 1e-12     # the small stand-in is narrower
        assert p["dx"] in G["flume_particle_sizes"]
    import inspect
    sig = inspect.signature(WL.wave_tank)
    assert sig.parameters["width"].default == G["flume_width"]
    assert sig.parameters["dx"].default in G["flume_particle_sizes"]
