"""FP64 CPU oracle of the learned k-step surrogate (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg use this module; the CUDA library never does.

The paper (Wei et al., two-phase SPH) has no learned component.  The network
is a message-passing neural network in the sense of Gilmer et al. (2017,
"Neural message passing for quantum chemistry"): an encoder, two rounds of
edge messages summed at the receiver followed by a residual node update, and
a decoder, with SiLU activations (Elfwing et al. 2018) and the Adam optimiser
(Kingma & Ba 2015).  The parameter format and the feature definitions are in
``paper_1702_07760_gb300/surrogate_layout.py``; this file restates the
arithmetic in plain numpy:

* forward: the edge MLP's first layer acts on the concatenation
  [h_i, h_j, e_ij]; written as W1 h_i + W2 h_j + W3 e_ij it is the same
  matrix product split by blocks.  Its second layer is linear, so the sum of
  messages over j equals the second layer applied to the sum of the hidden
  activations plus deg_i times its bias; this oracle uses that exact
  identity (the tests check it against the per-edge textbook form).
* backward: reverse-mode differentiation of the forward, by hand.
* loss: masked mean squared error of normalised increments.
* adam: one Adam step with bias correction.
"""
from __future__ import annotations

import numpy as np

import oracle as SPH
from paper_1702_07760_gb300 import surrogate_layout as SL


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def graph(p: dict, x: np.ndarray, phase: np.ndarray, u=None, rho=None, norm=None):
    """Edges (receiver i, sender j), j != i, |x_i - x_j| < 2h, sorted by
    (i, j), by brute force over all pairs; edge features
    [r_ij / 2h, |r_ij| / 2h, phase_i != phase_j, (u_i - u_j) / sd_edge_u,
    (delta_i - delta_j) / sd_edge_rho] with delta = (rho - rho0) / rho0.
    Without u, rho and norm the state-difference channels are zero."""
    x = np.asarray(x, float)
    n = len(x)
    two_h = 2.0 * p["h"]
    recv, send = [], []
    for i in range(n):
        r = x[i] - x
        d2 = np.einsum("ij,ij->i", r, r)
        js = np.nonzero(d2 < two_h * two_h)[0]
        js = js[js != i]
        recv.append(np.full(len(js), i))
        send.append(js)
    recv = np.concatenate(recv).astype(np.int64) if n else np.zeros(0, np.int64)
    send = np.concatenate(send).astype(np.int64) if n else np.zeros(0, np.int64)
    r = x[recv] - x[send]
    dist = np.sqrt(np.einsum("ij,ij->i", r, r))
    diff = (phase[recv] != phase[send]).astype(float)
    dim = x.shape[1]
    if u is None:
        du = np.zeros((len(recv), dim))
        dd = np.zeros(len(recv))
    else:
        _, _, _, _, _, _, su, sr = SL.split_norm(norm, dim)
        delta = (rho - np.asarray(p["rho0"], float)[phase]) / np.asarray(p["rho0"], float)[phase]
        du = (u[recv] - u[send]) / su
        dd = (delta[recv] - delta[send]) / sr
    E = np.concatenate([r / two_h, (dist / two_h)[:, None], diff[:, None], du, dd[:, None]], axis=1)
    return recv, send, E


def rates(p: dict, x, u, rho, phase, wall):
    """The plain method's acceleration and density rate at the state (the
    FP64 SPH oracle, with the density renormalisation of stage 1)."""
    ref = SPH.evaluate(p, x, u, rho, phase, wall, renorm=True)
    return ref["a"], ref["drho"]


def node_features(p: dict, u, rho, phase, wall, norm: np.ndarray, a, drho_dt):
    """Normalised node inputs [u, (rho - rho0)/rho0, oil, wall, T a,
    T (Drho/Dt) / rho0]."""
    dim = int(p["dim"])
    mu_in, sd_in, _, _, _, T, _, _ = SL.split_norm(norm, dim)
    rho0 = np.asarray(p["rho0"], float)[phase]
    raw = np.concatenate([np.asarray(u, float), ((rho - rho0) / rho0)[:, None],
                          phase[:, None].astype(float), wall[:, None].astype(float),
                          T * np.asarray(a, float), (T * np.asarray(drho_dt, float) / rho0)[:, None]], axis=1)
    return (raw - mu_in) / sd_in


def forward(flat: np.ndarray, dim: int, X, E, recv, send, k_ref: float, width: int = SL.H):
    """Normalised outputs y (N, 2d+1) and the activations the backward needs."""
    W = SL.unflatten(np.asarray(flat, float), dim, width)
    N = len(X)
    deg = np.bincount(recv, minlength=N).astype(float)
    c = {"X": X, "E": E, "recv": recv, "send": send, "deg": deg, "k_ref": k_ref, "rounds": [], "width": width}
    z0 = X @ W["enc1.w"].T + W["enc1.b"]
    a0 = silu(z0)
    h = a0 @ W["enc2.w"].T + W["enc2.b"]
    c["z0"], c["a0"] = z0, a0
    for r in range(SL.ROUNDS):
        P = h @ W[f"r{r}.w1"].T + W[f"r{r}.b1"]
        Q = h @ W[f"r{r}.w2"].T
        Z = P[recv] + Q[send] + E @ W[f"r{r}.w3"].T
        S = np.zeros_like(h)
        np.add.at(S, recv, silu(Z))
        S /= k_ref
        M = S @ W[f"r{r}.we2"].T + (deg / k_ref)[:, None] * W[f"r{r}.be2"]
        A1 = np.concatenate([h, M], axis=1)
        Z1 = A1 @ W[f"r{r}.n1"].T + W[f"r{r}.n1b"]
        G1 = silu(Z1)
        h_new = h + G1 @ W[f"r{r}.n2"].T + W[f"r{r}.n2b"]
        c["rounds"].append({"h": h, "Z": Z, "S": S, "A1": A1, "Z1": Z1, "G1": G1})
        h = h_new
    z2 = h @ W["dec1.w"].T + W["dec1.b"]
    a2 = silu(z2)
    y = a2 @ W["dec2.w"].T + W["dec2.b"]
    c["hL"], c["z2"], c["a2"] = h, z2, a2
    return y, c


def loss(y, t, mask):
    """Masked mean squared error and its gradient dL/dy."""
    cnt = mask.sum()
    d = (y - t) * mask
    return float((d * d).sum() / cnt), 2.0 * d / cnt


def output_mask(dim: int, wall):
    """1 for every (node, channel) that enters the loss: all channels of
    fluid nodes, only the density channel of wall nodes."""
    m = np.ones((len(wall), SL.n_out(dim)))
    m[wall.astype(bool), :2 * dim] = 0.0
    return m


def backward(flat: np.ndarray, dim: int, cache, dy):
    """Gradient of the loss with respect to every parameter (flat vector)."""
    width = cache["width"]
    W = SL.unflatten(np.asarray(flat, float), dim, width)
    G = {k: np.zeros_like(v) for k, v in W.items()}
    recv, send, E, deg, k_ref = cache["recv"], cache["send"], cache["E"], cache["deg"], cache["k_ref"]
    # decoder
    G["dec2.w"] = dy.T @ cache["a2"]
    G["dec2.b"] = dy.sum(0)
    dz2 = (dy @ W["dec2.w"]) * dsilu(cache["z2"])
    G["dec1.w"] = dz2.T @ cache["hL"]
    G["dec1.b"] = dz2.sum(0)
    dh = dz2 @ W["dec1.w"]
    # rounds in reverse
    for r in reversed(range(SL.ROUNDS)):
        R = cache["rounds"][r]
        Hd = R["h"].shape[1]
        G[f"r{r}.n2"] = dh.T @ R["G1"]
        G[f"r{r}.n2b"] = dh.sum(0)
        dZ1 = (dh @ W[f"r{r}.n2"]) * dsilu(R["Z1"])
        G[f"r{r}.n1"] = dZ1.T @ R["A1"]
        G[f"r{r}.n1b"] = dZ1.sum(0)
        dA1 = dZ1 @ W[f"r{r}.n1"]
        dh_next = dh + dA1[:, :Hd]
        dM = dA1[:, Hd:]
        G[f"r{r}.we2"] = dM.T @ R["S"]
        G[f"r{r}.be2"] = ((deg / k_ref)[:, None] * dM).sum(0)
        dS = dM @ W[f"r{r}.we2"]
        dZ = dS[recv] * dsilu(R["Z"]) / k_ref
        dP = np.zeros_like(dS)
        dQ = np.zeros_like(dS)
        np.add.at(dP, recv, dZ)
        np.add.at(dQ, send, dZ)
        G[f"r{r}.w3"] = dZ.T @ E
        G[f"r{r}.w1"] = dP.T @ R["h"]
        G[f"r{r}.b1"] = dP.sum(0)
        G[f"r{r}.w2"] = dQ.T @ R["h"]
        dh = dh_next + dP @ W[f"r{r}.w1"] + dQ @ W[f"r{r}.w2"]
    # encoder
    G["enc2.w"] = dh.T @ cache["a0"]
    G["enc2.b"] = dh.sum(0)
    dz0 = (dh @ W["enc2.w"]) * dsilu(cache["z0"])
    G["enc1.w"] = dz0.T @ cache["X"]
    G["enc1.b"] = dz0.sum(0)
    return np.concatenate([G[name].ravel() for name, _ in SL.layout(dim, width)])


def adam(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1); step counts from 1.
    Returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def targets(p: dict, x0, u0, rho0_state, x1, u1, rho1, phase, norm, a, drho_dt):
    """Normalised training targets between two states T apart: the position
    increment's departure from the trapezoid rule T (u0 + u1) / 2, and the
    velocity and density deviation increments' departures from the explicit
    jump T a and T (Drho/Dt) / rho0."""
    dim = int(p["dim"])
    _, _, mu_out, sd_out, _, T, _, _ = SL.split_norm(norm, dim)
    ref = np.asarray(p["rho0"], float)[phase]
    D = np.concatenate([(x1 - x0) - T * 0.5 * (u0 + u1), u1 - u0 - T * np.asarray(a, float),
                        ((rho1 - rho0_state) / ref - T * np.asarray(drho_dt, float) / ref)[:, None]], axis=1)
    return (D - mu_out) / sd_out


def predict(flat, p: dict, x, u, rho, phase, wall, norm):
    """De-normalised increments over k plain steps for the state (x, u, rho):
    (dx (N, d), du (N, d), drho (N,)); walls get zero dx and du."""
    dim = int(p["dim"])
    a, drho_dt = rates(p, x, u, rho, phase, wall)
    recv, send, E = graph(p, x, phase, u, rho, norm)
    X = node_features(p, u, rho, phase, wall, norm, a, drho_dt)
    _, _, mu_out, sd_out, k_ref, T, _, _ = SL.split_norm(norm, dim)
    y, _ = forward(flat, dim, X, E, recv, send, k_ref)
    D = y * sd_out + mu_out
    ref = np.asarray(p["rho0"], float)[phase]
    du = T * np.asarray(a, float) + D[:, dim:2 * dim]
    dx = T * (np.asarray(u, float) + 0.5 * du) + D[:, :dim]
    drel = T * np.asarray(drho_dt, float) / ref + D[:, 2 * dim]
    dx[wall.astype(bool)] = 0.0
    du[wall.astype(bool)] = 0.0
    return dx, du, drel * ref
