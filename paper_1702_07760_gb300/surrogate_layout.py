"""Parameter layout and seeded initial weights of the learned k-step surrogate.

This module holds the storage format only (which tensors, in which order and
shape, and the seeded random initial values); none of the network's
arithmetic.  The CUDA library and the FP64 oracle both read weights in this
format, so a weight file trained by one can be evaluated by the other.

Network (message passing over the particle graph, width H = 128; the paper
has no learned component, the architecture is this library's):

* node input, 2d + 4 channels: velocity u (d), density deviation
  (rho - rho0) / rho0, oil flag, wall flag, and the explicit increments of
  the plain method's rates at the current state over the jump T = k dt:
  T a (d) and T (Drho/Dt) / rho0; each normalised as (raw - mu_in) / sd_in;
* edge input for the pair (receiver i, sender j), |r_ij| < 2h, 2d + 3
  channels: r_ij / 2h (d), |r_ij| / 2h, 1 when i and j are of different
  phase, (u_i - u_j) / sd_edge_u (d) and the difference of the density
  deviations ((rho_i - rho0_i)/rho0_i - (rho_j - rho0_j)/rho0_j) / sd_edge_rho;
* encoder ``enc1`` (d+3 -> H), SiLU, ``enc2`` (H -> H);
* two rounds r of: edge MLP on [h_i, h_j, e_ij] whose first layer is stored
  split as ``w1`` (acting on h_i, with bias ``b1``), ``w2`` (on h_j) and
  ``w3`` (on e_ij), SiLU, second layer ``we2`` / ``be2``; messages summed
  over j and scaled by 1 / k_ref; node MLP ``n1`` (on [h, M], 2H -> H), SiLU,
  ``n2`` (H -> H), added to h;
* decoder ``dec1`` (H -> H), SiLU, ``dec2`` (H -> 2d + 1): normalised
  outputs de-normalised as D = y * sd_out + mu_out, corrections to the
  explicit jump: velocity increment du = T a + D[d:2d], density deviation
  increment T (Drho/Dt) / rho0 + D[2d] (times rho0 for drho), position
  increment dx = T (u + du / 2) + D[:d] (the trapezoid rule plus a
  correction).

Flat order: the tensors below in list order, each row-major (weights
[out, in]).  The normalisation block is a separate array of
6 d + 14 values: mu_in (2d+4), sd_in (2d+4), mu_out (2d+1), sd_out (2d+1),
k_ref, T, sd_edge_u, sd_edge_rho.
"""
from __future__ import annotations

import numpy as np

H = 128
ROUNDS = 2


def n_in(dim: int) -> int:
    return 2 * dim + 4


def n_edge(dim: int) -> int:
    return 2 * dim + 3


def n_out(dim: int) -> int:
    return 2 * dim + 1


def layout(dim: int, width: int = H):
    """[(name, shape)] of every parameter tensor, in storage order."""
    L = [("enc1.w", (width, n_in(dim))), ("enc1.b", (width,)),
         ("enc2.w", (width, width)), ("enc2.b", (width,))]
    for r in range(ROUNDS):
        L += [(f"r{r}.w1", (width, width)), (f"r{r}.b1", (width,)),
              (f"r{r}.w2", (width, width)),
              (f"r{r}.w3", (width, n_edge(dim))),
              (f"r{r}.we2", (width, width)), (f"r{r}.be2", (width,)),
              (f"r{r}.n1", (width, 2 * width)), (f"r{r}.n1b", (width,)),
              (f"r{r}.n2", (width, width)), (f"r{r}.n2b", (width,))]
    L += [("dec1.w", (width, width)), ("dec1.b", (width,)),
          ("dec2.w", (n_out(dim), width)), ("dec2.b", (n_out(dim),))]
    return L


def size(dim: int, width: int = H) -> int:
    return int(sum(np.prod(s) for _, s in layout(dim, width)))


def unflatten(flat: np.ndarray, dim: int, width: int = H) -> dict:
    """Views of the flat parameter vector, by name."""
    out, o = {}, 0
    for name, shape in layout(dim, width):
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    assert o == len(flat)
    return out


def offsets(dim: int, width: int = H) -> dict:
    """Element offset of every tensor in the flat vector."""
    out, o = {}, 0
    for name, shape in layout(dim, width):
        out[name] = o
        o += int(np.prod(shape))
    return out


def init_weights(dim: int, seed: int = 0, width: int = H, out_scale: float = 0.1) -> np.ndarray:
    """Seeded initial parameters (float64): weights N(0, 1/fan_in), biases 0,
    the decoder's last layer scaled by out_scale.  Drawn from
    Generator(PCG64(seed)) in storage order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, shape in layout(dim, width):
        if len(shape) == 1:
            parts.append(np.zeros(shape))
            continue
        fan_in = shape[1]
        if name.endswith(".w1") or name.endswith(".w2") or name.endswith(".w3"):
            fan_in = 2 * width + n_edge(dim)   # the three parts form one layer
        w = rng.standard_normal(shape) / np.sqrt(fan_in)
        if name == "dec2.w":
            w *= out_scale
        parts.append(w)
    return np.concatenate([p.ravel() for p in parts])


def norm_size(dim: int) -> int:
    return 2 * n_in(dim) + 2 * n_out(dim) + 4


def make_norm(dim: int, mu_in, sd_in, mu_out, sd_out, k_ref: float, t_jump: float, sd_edge_u: float,
              sd_edge_rho: float) -> np.ndarray:
    """Pack the normalisation block."""
    v = np.concatenate([np.asarray(mu_in, float), np.asarray(sd_in, float), np.asarray(mu_out, float),
                        np.asarray(sd_out, float), [float(k_ref), float(t_jump), float(sd_edge_u),
                                                    float(sd_edge_rho)]])
    assert len(v) == norm_size(dim)
    return v


def split_norm(norm: np.ndarray, dim: int):
    """(mu_in, sd_in, mu_out, sd_out, k_ref, t_jump, sd_edge_u, sd_edge_rho)."""
    a, b = n_in(dim), n_out(dim)
    o = 2 * a + 2 * b
    return (norm[:a], norm[a:2 * a], norm[2 * a:2 * a + b], norm[2 * a + b:o], float(norm[o]),
            float(norm[o + 1]), float(norm[o + 2]), float(norm[o + 3]))
