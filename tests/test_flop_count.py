"""Algorithmic flops per neighbour pair of the force sweep (the roofline's
numerator in bench.py), counted on a restatement of the pair terms.

The restatement evaluates, for one ordered pair (i, j) within 2h, the terms
of Sec. II that the force sweep sums: the pressure term (Eq. dist_p_1), the
dynamic-form viscous term (Eq. visc_2) and the continuity term
(Eq. ct_dist_2), with grad_i W_ij = (dW/dr) r_ij / r of the Wendland C2
kernel.  Quantities that depend on one particle only (P/rho^2, m/rho, the
harmonic-mean viscosity of a phase pair, the kernel's constant factor) are
per-particle or per-phase values, not pair work, and enter as plain numbers;
the pair factor m_j (P_i/rho_i^2 + P_j/rho_j^2) is counted as written (an
add and a multiply).
Every +, -, * and / and the square root count one flop (a fused
multiply-add counts two).  Surface-tension pairs (a few per cent, at the
interface only) are not counted.
"""
import math

import bench


class Counted:
    """A float that counts the arithmetic done on it."""
    ops = 0

    def __init__(self, v):
        self.v = float(v)

    @staticmethod
    def _v(o):
        return o.v if isinstance(o, Counted) else float(o)

    def _op(self, r):
        Counted.ops += 1
        return Counted(r)

    def __add__(self, o): return self._op(self.v + self._v(o))
    def __radd__(self, o): return self._op(self._v(o) + self.v)
    def __sub__(self, o): return self._op(self.v - self._v(o))
    def __rsub__(self, o): return self._op(self._v(o) - self.v)
    def __mul__(self, o): return self._op(self.v * self._v(o))
    def __rmul__(self, o): return self._op(self._v(o) * self.v)
    def __truediv__(self, o): return self._op(self.v / self._v(o))

    def sqrt(self):
        return self._op(math.sqrt(self.v))


def pair_terms(dim, xi, xj, ui, uj, Q_i, Q_j, m_j, V_j, k_ij, inv_2h, delta2, acc, visc, div):
    """Adds pair (i, j)'s terms to the running sums: pressure
    m_j (P_i/rho_i^2 + P_j/rho_j^2) grad W, viscous k_ij V_j (r.grad W)/(r^2 +
    delta^2) u_ij (the 1/rho_i of Eq. visc_2 and the kernel's constant factor
    are applied once per particle), continuity V_j u_ij . grad W."""
    r = [xi[c] - xj[c] for c in range(dim)]
    r2 = r[0] * r[0]
    for c in range(1, dim):
        r2 = r2 + r[c] * r[c]
    rr = r2.sqrt()
    t = 1.0 - rr * inv_2h
    t3 = t * t * t                                  # (dW/dr) / r up to the constant factor
    pt = (Q_i + Q_j) * m_j * t3
    for c in range(dim):
        acc[c] = acc[c] + pt * r[c]
    u = [ui[c] - uj[c] for c in range(dim)]
    vt = V_j * t3
    s = k_ij * vt * r2 / (r2 + delta2)
    for c in range(dim):
        visc[c] = visc[c] + s * u[c]
    ur = u[0] * r[0]
    for c in range(1, dim):
        ur = ur + u[c] * r[c]
    return div + vt * ur


def continuity_terms(dim, xi, xj, ui, uj, V_j, inv_2h, div):
    """The continuity term alone, V_j u_ij . grad W (what a boundary particle
    takes from a pair with a moving particle)."""
    r = [xi[c] - xj[c] for c in range(dim)]
    r2 = r[0] * r[0]
    for c in range(1, dim):
        r2 = r2 + r[c] * r[c]
    rr = r2.sqrt()
    t = 1.0 - rr * inv_2h
    t3 = t * t * t
    vt = V_j * t3
    u = [ui[c] - uj[c] for c in range(dim)]
    ur = u[0] * r[0]
    for c in range(1, dim):
        ur = ur + u[c] * r[c]
    return div + vt * ur


def count_continuity(dim):
    C = Counted
    xi, xj = [C(0.1 * (c + 1)) for c in range(dim)], [C(0.05 * c) for c in range(dim)]
    ui, uj = [C(0.0)] * dim, [C(-0.02 * c) for c in range(dim)]
    Counted.ops = 0
    continuity_terms(dim, xi, xj, ui, uj, 1e-11, 1.0 / 0.65, C(0.0))
    return Counted.ops


def count(dim):
    C = Counted
    xi, xj = [C(0.1 * (c + 1)) for c in range(dim)], [C(0.05 * c) for c in range(dim)]
    ui, uj = [C(0.01 * c) for c in range(dim)], [C(-0.02 * c) for c in range(dim)]
    acc, visc = [C(0.0)] * dim, [C(0.0)] * dim
    Counted.ops = 0
    pair_terms(dim, xi, xj, ui, uj, C(2e-4), C(3e-4), 1e-8, 1e-11, 2e-3, 1.0 / 0.65, 1e-3, acc, visc, C(0.0))
    return Counted.ops


def test_force_sweep_flops_per_pair_match_bench():
    for dim in (2, 3):
        assert count(dim) == bench.SWEEP_B_FLOPS_PER_PAIR[dim], (dim, count(dim))


def test_continuity_only_flops_per_pair_match_bench():
    for dim in (2, 3):
        assert count_continuity(dim) == bench.SWEEP_B_FLOPS_CONTINUITY[dim], (dim, count_continuity(dim))
