"""Pins of the second-order references the GPU tests use, on the FP64 oracle (no GPU).

The exact Hessian-vector product of the misfit is the directional derivative of its gradient,
H v = d/dC g(C) . v. With J = dM/dC and w = 2 (M - M_obs) it splits into
H v = 2 J^T (J v) + d/dC[J^T w] . v (w held fixed). The references are central differences of the
oracle's pinned gradient and of its vector-Jacobian product (the misfit gradient with
M_obs = M - w/2). These tests check that the differences are converged in h, that the split
holds, and that the Hessian they give is symmetric."""
import numpy as np
import pytest

import oracle
from paper_2603_04070_gb300 import inputs


def _setup(seed, order=8):
    wl = inputs.make_workload("full_shot_set", seed=seed, nx=40, nz=36, nt=220, n_elem=10, n_tx=2, fd_order=order)
    p = oracle.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml=wl.pml, pml_R=wl.pml_R,
                       pml_cref=wl.pml_cref, fd_order=wl.fd_order)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    w = wl.wavelet.astype(np.float64)

    def traces(C):
        return np.stack([oracle.forward(p, C, (tix[k], tiz[k]), w, rix[k], riz[k]) for k in range(wl.n_tx)])

    def grad(C, M_obs):
        return oracle.misfit_gradient(p, C, tix, tiz, w, rix, riz, M_obs)[1]

    def vjp(C, q):
        return grad(C, traces(C) - 0.5 * q)

    rng = np.random.default_rng(seed)
    C = wl.sos_start[0].astype(np.float64)
    M_obs = traces(wl.sos_true[0].astype(np.float64))
    return C, M_obs, traces, grad, vjp, rng


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("order", [8, 4])
def test_hessian_split_and_convergence(order):
    C, M_obs, traces, grad, vjp, rng = _setup(70 + order, order)
    v = rng.standard_normal(C.shape) * 5.0

    def hv(h):
        return (grad(C + h * v, M_obs) - grad(C - h * v, M_obs)) / (2 * h)

    H1, H2 = hv(0.05), hv(0.025)
    assert _rel(H1, H2) <= 1e-5                              # O(h^2) differences have converged
    w = 2.0 * (traces(C) - M_obs)
    S = (vjp(C + 0.05 * v, w) - vjp(C - 0.05 * v, w)) / 0.1
    Jv = (traces(C + 0.05 * v) - traces(C - 0.05 * v)) / 0.1
    GN = vjp(C, 2.0 * Jv)
    assert _rel(S + GN, H1) <= 1e-5                          # H v = 2 J^T J v + d/dC[J^T w] . v
    assert _rel(GN, H1) >= 1e-2                              # the residual term is not negligible here


def test_hessian_is_symmetric():
    C, M_obs, traces, grad, vjp, rng = _setup(79)
    u = rng.standard_normal(C.shape) * 5.0
    v = rng.standard_normal(C.shape) * 5.0
    h = 0.05
    Hv = (grad(C + h * v, M_obs) - grad(C - h * v, M_obs)) / (2 * h)
    Hu = (grad(C + h * u, M_obs) - grad(C - h * u, M_obs)) / (2 * h)
    a, b = float(np.sum(u * Hv)), float(np.sum(v * Hu))
    assert abs(a - b) <= 1e-6 * max(abs(a), abs(b))
