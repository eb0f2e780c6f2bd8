"""Conditioning of the per-particle acceleration sums, for the error bounds of
the FP32 force sweep.

The acceleration of particle i is a sum over its neighbours of pair terms
(pressure, Eq. dist_p_1; viscosity, Eq. visc_2 or visc_1; surface tension,
F_s/rho) plus g.  Evaluated in FP32, every rounding is relative to the size of
the quantity rounded, so the error of a_i scales with

    S_i = sum_j (|p_ij| + |v_ij| + |s_ij|) + |g|,

the sum of the magnitudes of its terms, not with |a_i|.  In a hydrostatic
column the pressure terms are of order rho g H / (rho h) per neighbour and
cancel to about g, so S_i / max(|a_i|, |g|) (the condition number of the sum)
is 50 to 400 on the parity states.  Each pair term carries at most
ROUNDINGS_PER_TERM FP32 roundings before it enters its running sum (pair
vector, squared distance, distance, 1 - q/2, its cube, the pair factor and the
product), and a running sum of k terms adds at most k - 1 more, so with the
unit roundoff u = 2^-24 (Higham, Accuracy and Stability of Numerical
Algorithms, ch. 3-4):

    |a_gpu,i - a_i| <= (k_i + ROUNDINGS_PER_TERM) u S_i  (first order in u).

Test infrastructure: this module restates the magnitudes of the terms from
the oracle's outputs to size the bound; it computes no result that a test
compares against.
"""
import numpy as np

import oracle

U32 = 2.0 ** -24
ROUNDINGS_PER_TERM = 8


def term_magnitudes(p, x, u, rho, P, T, phase, wall):
    """(S_i, k_i): the sum of the magnitudes of particle i's pair terms plus
    |g|, and its number of neighbours within 2h (oracle state: the density and
    pressure after renormalisation, the surface stress tensor)."""
    d = int(p["dim"])
    x = np.asarray(x, np.float64)
    u = np.asarray(u, np.float64)
    rho = np.asarray(rho, np.float64)
    start, lst = oracle.neighbours(p, x, "cells")
    n = len(x)
    h = p["h"]
    al = 7 / (4 * np.pi * h * h) if d == 2 else 21 / (16 * np.pi * h ** 3)
    mass = np.asarray(p["mass"])[phase]
    Q = np.abs(np.asarray(P) / rho ** 2)
    mu = np.asarray(p["mu"])
    rho0 = np.asarray(p["rho0"])
    kin = int(p.get("visc_form", 0)) == 1
    visc_ph = mu / rho0 if kin else mu
    Tn = np.linalg.norm(np.asarray(T).reshape(n, -1), axis=1)
    sig = rho / mass
    per = int(p.get("periodic", 0))
    S = np.zeros(n)
    step = 1 << 17
    for c0 in range(0, n, step):
        c1 = min(n, c0 + step)
        I = np.repeat(np.arange(c0, c1), np.diff(start[c0:c1 + 1]))
        J = lst[start[c0]:start[c1]].astype(np.int64)
        r = x[I] - x[J]
        for a in range(d):
            if (per >> a) & 1:
                L = p["box_hi"][a] - p["box_lo"][a]
                r[:, a] -= L * np.round(r[:, a] / L)
        rn = np.linalg.norm(r, axis=1)
        q = rn / h
        dwdr = np.abs(al * (-5 * q / h) * np.maximum(1 - 0.5 * q, 0.0) ** 3)   # |grad_i W_ij|
        pres = mass[J] * (Q[I] + Q[J]) * dwdr
        a_, b_ = visc_ph[phase[I]], visc_ph[phase[J]]
        kij = 2 * a_ * b_ / np.maximum(a_ + b_, 1e-300)
        pref = 1.0 if kin else 1.0 / rho[I]
        uij = np.linalg.norm(u[I] - u[J], axis=1)
        visc = pref * 2 * kij * (mass[J] / rho[J]) * rn * dwdr / (rn ** 2 + p["delta"] ** 2) * uij
        st = (Tn[I] / sig[I] ** 2 + Tn[J] / sig[J] ** 2) * dwdr / mass[I]
        S[c0:c1] = np.bincount(I - c0, weights=pres + visc + st, minlength=c1 - c0)
    S += np.linalg.norm(p["g"])
    k = np.diff(start)
    return S, k


def acc_error_report(p, x, u, ref, got_acc, phase, wall):
    """Per-particle errors of the fluid accelerations: (max over fluid
    particles of |da_i| / ((k_i + ROUNDINGS_PER_TERM) u S_i), the same with
    the bare u S_i, and the per-particle error against max(|a_i|, |g|))."""
    S, k = term_magnitudes(p, x, u, ref["rho"], ref["P"], ref["T"], phase, wall)
    fl = np.asarray(wall) == 0
    da = np.linalg.norm(got_acc[fl] - ref["a"][fl], axis=1)
    bound = (k[fl] + ROUNDINGS_PER_TERM) * U32 * S[fl]
    floor = np.maximum(np.linalg.norm(ref["a"][fl], axis=1), np.linalg.norm(p["g"]))
    return float((da / bound).max()), float((da / (U32 * S[fl])).max()), float((da / floor).max())
