"""Pins of the FP64 surrogate oracle (oracle/mpnn.py), CPU only.

* The split first layer (W1 h_i + W2 h_j + W3 e_ij) and the second layer
  applied after the sum are checked against the textbook per-edge form
  (one matrix on the concatenation [h_i, h_j, e_ij], the two-layer message
  computed for every edge, then summed), written with torch.
* The hand-written backward is checked against torch autograd of that
  textbook form, and against central finite differences on a narrow net.
* Translation invariance, permutation equivariance, the all-zero-weight
  special case, the edge set against the oracle's cell-list neighbour
  search, and Adam against torch.optim.Adam.
"""
import numpy as np
import pytest

import oracle
from oracle import mpnn as O
from paper_1702_07760_gb300 import surrogate_layout as SL
from paper_1702_07760_gb300 import workloads as WL

torch = pytest.importorskip("torch")


def _case(dim=2, seed=3):
    if dim == 2:
        w = WL.drop_tank(2, (7, 9), drop_d_dx=4, seed=seed, perturb=True, wall_layers=2)
    else:
        w = WL.drop_tank(3, (4, 4, 5), drop_d_dx=3, seed=seed, perturb=True, wall_layers=1)
    rng = np.random.Generator(np.random.PCG64(seed))
    n_in, n_out = SL.n_in(dim), SL.n_out(dim)
    norm = SL.make_norm(dim, rng.normal(0, 0.1, n_in), rng.uniform(0.5, 2, n_in),
                        rng.normal(0, 0.1, n_out), rng.uniform(0.5, 2, n_out), k_ref=10.0, t_jump=8e-5,
                        sd_edge_u=0.02 * w.params["c0"], sd_edge_rho=1e-3)
    return w, norm


def _textbook(flat, dim, X, E, recv, send, k_ref, width=SL.H):
    """Per-edge two-layer message on [h_i, h_j, e_ij], summed at i (torch)."""
    W = {k: torch.tensor(v) for k, v in SL.unflatten(flat, dim, width).items()}
    X, E = torch.tensor(X), torch.tensor(E)
    recv_t, send_t = torch.tensor(recv), torch.tensor(send)
    act = torch.nn.functional.silu
    h = act(X @ W["enc1.w"].T + W["enc1.b"]) @ W["enc2.w"].T + W["enc2.b"]
    for r in range(SL.ROUNDS):
        full = torch.cat([W[f"r{r}.w1"], W[f"r{r}.w2"], W[f"r{r}.w3"]], dim=1)
        inp = torch.cat([h[recv_t], h[send_t], E], dim=1)
        msg = act(inp @ full.T + W[f"r{r}.b1"]) @ W[f"r{r}.we2"].T + W[f"r{r}.be2"]
        M = torch.zeros_like(h).index_add(0, recv_t, msg) / k_ref
        h = h + act(torch.cat([h, M], 1) @ W[f"r{r}.n1"].T + W[f"r{r}.n1b"]) @ W[f"r{r}.n2"].T + W[f"r{r}.n2b"]
    return act(h @ W["dec1.w"].T + W["dec1.b"]) @ W["dec2.w"].T + W["dec2.b"]


@pytest.mark.parametrize("dim", [2, 3])
def test_forward_equals_textbook_edge_mlp(dim):
    w, norm = _case(dim)
    flat = SL.init_weights(dim, seed=5, out_scale=1.0)
    recv, send, E = O.graph(w.params, w.x, w.phase, w.u, w.rho, norm)
    X = O.node_features(w.params, w.u, w.rho, w.phase, w.wall, norm, *O.rates(w.params, w.x, w.u, w.rho, w.phase, w.wall))
    y, _ = O.forward(flat, dim, X, E, recv, send, 10.0)
    yt = _textbook(flat, dim, X, E, recv, send, 10.0).numpy()
    assert len(recv) > 10 * len(X)
    assert np.abs(y - yt).max() <= 1e-12 * np.abs(yt).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_backward_equals_autograd_of_textbook_form(dim):
    w, norm = _case(dim, seed=4)
    flat = SL.init_weights(dim, seed=6, out_scale=1.0)
    recv, send, E = O.graph(w.params, w.x, w.phase, w.u, w.rho, norm)
    X = O.node_features(w.params, w.u, w.rho, w.phase, w.wall, norm, *O.rates(w.params, w.x, w.u, w.rho, w.phase, w.wall))
    rng = np.random.Generator(np.random.PCG64(9))
    t = rng.normal(size=(len(X), SL.n_out(dim)))
    mask = O.output_mask(dim, w.wall)
    y, cache = O.forward(flat, dim, X, E, recv, send, 10.0)
    L, dy = O.loss(y, t, mask)
    g = O.backward(flat, dim, cache, dy)
    th = torch.tensor(flat, requires_grad=True)
    # rebuild the textbook graph on the differentiable flat vector
    names = SL.layout(dim)
    offs = SL.offsets(dim)

    def textbook_from(theta):
        W = {n: theta[offs[n]:offs[n] + int(np.prod(s))].reshape(s) for n, s in names}
        act = torch.nn.functional.silu
        Xt, Et = torch.tensor(X), torch.tensor(E)
        rt, st = torch.tensor(recv), torch.tensor(send)
        h = act(Xt @ W["enc1.w"].T + W["enc1.b"]) @ W["enc2.w"].T + W["enc2.b"]
        for r in range(SL.ROUNDS):
            full = torch.cat([W[f"r{r}.w1"], W[f"r{r}.w2"], W[f"r{r}.w3"]], dim=1)
            msg = act(torch.cat([h[rt], h[st], Et], 1) @ full.T + W[f"r{r}.b1"]) @ W[f"r{r}.we2"].T + W[f"r{r}.be2"]
            M = torch.zeros_like(h).index_add(0, rt, msg) / 10.0
            h = h + act(torch.cat([h, M], 1) @ W[f"r{r}.n1"].T + W[f"r{r}.n1b"]) @ W[f"r{r}.n2"].T + W[f"r{r}.n2b"]
        return act(h @ W["dec1.w"].T + W["dec1.b"]) @ W["dec2.w"].T + W["dec2.b"]

    yt = textbook_from(th)
    mt = torch.tensor(mask)
    Lt = (((yt - torch.tensor(t)) * mt) ** 2).sum() / mt.sum()
    Lt.backward()
    gt = th.grad.numpy()
    assert abs(L - Lt.item()) <= 1e-12 * abs(L)
    assert np.abs(g - gt).max() <= 1e-10 * np.abs(gt).max()
    # every tensor receives a gradient
    for name, _ in names:
        o = offs[name]
        assert np.any(gt[o:o + 1] != 0) or np.any(gt[o:o + 4] != 0), name


def test_backward_matches_central_differences():
    dim, width = 2, 6
    w, norm = _case(2, seed=7)
    flat = SL.init_weights(dim, seed=8, width=width, out_scale=1.0)
    recv, send, E = O.graph(w.params, w.x, w.phase, w.u, w.rho, norm)
    X = O.node_features(w.params, w.u, w.rho, w.phase, w.wall, norm, *O.rates(w.params, w.x, w.u, w.rho, w.phase, w.wall))
    rng = np.random.Generator(np.random.PCG64(10))
    t = rng.normal(size=(len(X), SL.n_out(dim)))
    mask = O.output_mask(dim, w.wall)

    def f(theta):
        return O.loss(O.forward(theta, dim, X, E, recv, send, 10.0, width)[0], t, mask)[0]

    y, cache = O.forward(flat, dim, X, E, recv, send, 10.0, width)
    _, dy = O.loss(y, t, mask)
    g = O.backward(flat, dim, cache, dy)
    # central differences with Richardson extrapolation (truncation error O(eps^4))
    eps = 1e-5
    idx = rng.choice(len(flat), size=120, replace=False)
    for k in idx:
        e = np.zeros_like(flat)
        e[k] = 1.0

        def cd(h):
            return (f(flat + h * e) - f(flat - h * e)) / (2 * h)

        fd = (4.0 * cd(eps / 2) - cd(eps)) / 3.0
        assert abs(fd - g[k]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (k, fd, g[k])


def test_translation_invariance_and_permutation_equivariance():
    dim = 2
    w, norm = _case(dim, seed=11)
    flat = SL.init_weights(dim, seed=12, out_scale=1.0)
    dx, du, dr = O.predict(flat, w.params, w.x, w.u, w.rho, w.phase, w.wall, norm)
    shift = np.array([3.7e-3, -1.1e-3])
    p2 = dict(w.params, box_lo=[w.params["box_lo"][0] + shift[0], w.params["box_lo"][1] + shift[1], 0.0],
              box_hi=[w.params["box_hi"][0] + shift[0], w.params["box_hi"][1] + shift[1], 0.0])
    dx2, du2, dr2 = O.predict(flat, p2, w.x + shift, w.u, w.rho, w.phase, w.wall, norm)
    assert np.allclose(dx, dx2, rtol=0, atol=1e-9 * np.abs(dx).max())
    assert np.allclose(dr, dr2, rtol=0, atol=1e-9 * np.abs(dr).max())
    perm = np.random.Generator(np.random.PCG64(13)).permutation(w.n)
    dx3, du3, dr3 = O.predict(flat, w.params, w.x[perm], w.u[perm], w.rho[perm], w.phase[perm], w.wall[perm], norm)
    assert np.allclose(dx3, dx[perm], rtol=0, atol=1e-12 * np.abs(dx).max())
    assert np.allclose(du3, du[perm], rtol=0, atol=1e-12 * np.abs(du).max())
    assert np.all(dx[w.wall == 1] == 0) and np.all(du[w.wall == 1] == 0)


def test_zero_weights_give_the_output_bias():
    dim = 3
    w, norm = _case(dim, seed=14)
    flat = np.zeros(SL.size(dim))
    b = np.arange(1, SL.n_out(dim) + 1, dtype=float)
    flat[SL.offsets(dim)["dec2.b"]:SL.offsets(dim)["dec2.b"] + len(b)] = b
    recv, send, E = O.graph(w.params, w.x, w.phase, w.u, w.rho, norm)
    X = O.node_features(w.params, w.u, w.rho, w.phase, w.wall, norm, *O.rates(w.params, w.x, w.u, w.rho, w.phase, w.wall))
    y, _ = O.forward(flat, dim, X, E, recv, send, 10.0)
    assert np.all(y == b)


@pytest.mark.parametrize("dim", [2, 3])
def test_graph_equals_cell_list_neighbours(dim):
    w, norm = _case(dim, seed=15)
    recv, send, E = O.graph(w.params, w.x, w.phase, w.u, w.rho, norm)
    start, lst = oracle.neighbours(w.params, w.x, "cells")
    r2 = np.repeat(np.arange(w.n), np.diff(start))
    assert np.array_equal(recv, r2) and np.array_equal(send, lst)
    assert np.all(E[:, dim] < 1.0) and np.all(E[:, dim] > 0.0)
    assert np.allclose(np.linalg.norm(E[:, :dim], axis=1), E[:, dim], rtol=1e-14)
    # the state-difference channels are antisymmetric in (i, j)
    key = {(a, b): k for k, (a, b) in enumerate(zip(recv, send))}
    rev = np.array([key[(b, a)] for a, b in zip(recv, send)])
    flip = np.r_[np.arange(dim), np.arange(dim + 2, 2 * dim + 3)]
    keep = np.array([dim, dim + 1])
    assert np.array_equal(E[rev][:, flip], -E[:, flip]) and np.array_equal(E[rev][:, keep], E[:, keep])


def test_adam_matches_torch():
    rng = np.random.Generator(np.random.PCG64(16))
    theta = rng.normal(size=50)
    th = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([th], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 6):
        g = rng.normal(size=50)
        theta, m, v = O.adam(theta, g, m, v, step, 3e-3)
        opt.zero_grad()
        th.grad = torch.tensor(g)
        opt.step()
        assert np.allclose(theta, th.detach().numpy(), rtol=0, atol=1e-15)
