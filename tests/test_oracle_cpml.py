"""Pins of the oracle's convolutional PML (the alternative to the damping term D of Eq. 1).

* coefficient tables: identity (a = 0, b = 1) off the layer, a decaying recursion inside it,
  mirror symmetry of the profiles, and a = b - 1 when alpha = 0 (the classical PML limit);
* with a vanishing damping maximum the CPML reduces to the plain staggered operator;
* the border return is below twice the design reflection R = 1e-3 and over ten times smaller
  than that of the damping layer of the same thickness;
* the adjoint dot-product identity and central finite differences of the misfit (the discrete
  adjoint is the transpose of the forward recursion, memory variables included).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_04070_gb300 import inputs


def _cpml(n=30, nz=None, nt=200, pml=10, alpha=2 * math.pi * 1e6, **kw):
    return oracle.Problem(nx=n, nz=nz or n, dx=1e-4, dt=1e-8, nt=nt, pml=pml, pml_cref=1540.0, fd_order=8,
                          boundary=1, pml_alpha=alpha, **kw)


def test_cpml_coefficients():
    p = _cpml(n=20, pml=8)
    c = oracle.cpml_coeffs(p)
    P, n = p.pml, p.nx
    inner = slice(P, P + n)                      # physical nodes
    assert np.all(c["a_node_x"][inner] == 0.0) and np.all(c["b_node_x"][inner] == 1.0)
    assert np.all(c["a_half_x"][P:P + n - 1] == 0.0) and np.all(c["b_half_x"][P:P + n - 1] == 1.0)
    lay = np.r_[0:P, P + n:p.nxp]
    assert np.all((c["b_node_x"][lay] > 0) & (c["b_node_x"][lay] < 1)) and np.all(c["a_node_x"][lay] < 0)
    # mirror symmetry: node i <-> nxp-1-i, half point j <-> nxp-2-j
    assert np.allclose(c["a_node_x"], c["a_node_x"][::-1], rtol=0, atol=1e-15)
    assert np.allclose(c["a_half_x"][:-1], c["a_half_x"][:-1][::-1], rtol=0, atol=1e-15)
    # deeper is stronger (d grows faster than alpha shrinks for these settings)
    assert np.all(np.diff(c["b_node_x"][:P + 1]) > 0)
    # classical PML limit
    c0 = oracle.cpml_coeffs(_cpml(n=20, pml=8, alpha=0.0))
    assert np.allclose(c0["a_node_x"], c0["b_node_x"] - 1.0, rtol=0, atol=1e-15)


def test_cpml_without_damping_is_the_plain_staggered_operator():
    """pml_R -> 1 makes d0 -> 0: the memory variables stay ~0 and the traces are those of the
    staggered operator (unit density) with no absorbing term."""
    rng = np.random.default_rng(0)
    C = 1540.0 + 30.0 * rng.standard_normal((26, 30))
    w = inputs.ricker(260, 1e-8, 2e6).astype(np.float64)
    kw = dict(nx=30, nz=26, dx=1e-4, dt=1e-8, nt=260, pml=8, pml_R=1.0 - 1e-14, pml_cref=1540.0, fd_order=8)
    a = oracle.forward(oracle.Problem(boundary=1, pml_alpha=0.0, **kw), C, (4, 3), w, np.array([20, 2]),
                       np.array([15, 20]))
    b = oracle.forward(oracle.Problem(**kw), C, (4, 3), w, np.array([20, 2]), np.array([15, 20]),
                       rho=np.ones((26, 30)))
    assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b))


def test_cpml_reflection_below_design_and_damping_layer():
    c, dx, dt, f0 = 1540.0, 1e-4, 1e-8, 2e6
    nt = 700
    w = inputs.ricker(nt, dt, f0).astype(np.float64)
    for P in (10, 20):
        refl = {}
        for bnd in (0, 1):
            kw = dict(dx=dx, dt=dt, nt=nt, pml=P, pml_cref=c, fd_order=8, boundary=bnd, pml_alpha=math.pi * f0)
            small = oracle.Problem(nx=60, nz=60, **kw)
            big = oracle.Problem(nx=180, nz=180, **kw)
            tr_s = oracle.forward(small, np.full((60, 60), c), (30, 30), w, np.array([52]), np.array([30]))[:, 0]
            tr_b = oracle.forward(big, np.full((180, 180), c), (90, 90), w, np.array([112]), np.array([90]))[:, 0]
            refl[bnd] = np.max(np.abs(tr_s - tr_b)) / np.max(np.abs(tr_b))
        assert refl[1] < 2e-3, (P, refl)
        assert refl[1] < 0.1 * refl[0], (P, refl)


@pytest.mark.parametrize("with_density", [False, True])
def test_cpml_adjoint_dot_product(with_density):
    rng = np.random.default_rng(4)
    p = _cpml(n=26, nz=22, nt=200, pml=8)
    C = 1540.0 + 40.0 * rng.standard_normal((22, 26))
    rho = 1000.0 + 800.0 * rng.uniform(size=(22, 26)) if with_density else None
    rx_ix = np.array([2, 9, 20, 25, 13], dtype=np.int32)
    rx_iz = np.array([0, 5, 21, 11, 13], dtype=np.int32)
    src = (7, 15)
    w = rng.standard_normal(p.nt)
    q = rng.standard_normal((p.nt, rx_ix.size))
    Fw = oracle.forward(p, C, src, w, rx_ix, rx_iz, rho=rho)
    lam = oracle.adjoint_probe(p, C, rx_ix, rx_iz, q, src, rho=rho)
    lhs = np.sum(Fw * q)
    rhs = p.dt ** 2 / p.dx ** 2 * np.sum(w[:-1] * lam[1:])
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(Fw * q))


@pytest.mark.parametrize("with_density", [False, True])
def test_cpml_gradient_finite_differences(with_density):
    rng = np.random.default_rng(5)
    n, nt = 18, 180
    p = _cpml(n=n, nt=nt, pml=6)
    rho = 1000.0 + 600.0 * rng.uniform(size=(n, n)) if with_density else None
    C_true = 1540.0 + 40.0 * rng.standard_normal((n, n))
    C0 = 1540.0 + 5.0 * rng.standard_normal((n, n))
    tx_ix, tx_iz = np.array([3, 12], np.int32), np.array([0, 0], np.int32)
    rx_ix = np.tile(np.array([0, 4, 8, 12, 17], np.int32), (2, 1))
    rx_iz = np.tile(np.array([0, 0, 17, 0, 7], np.int32), (2, 1))
    w = inputs.ricker(nt, p.dt, 2e6).astype(np.float64)
    M_obs = np.stack([oracle.forward(p, C_true, (tx_ix[k], tx_iz[k]), w, rx_ix[k], rx_iz[k], rho=rho)
                      for k in range(2)])
    J, g, M = oracle.misfit_gradient(p, C0, tx_ix, tx_iz, w, rx_ix, rx_iz, M_obs, rho=rho, return_traces=True)
    M0 = np.stack([oracle.forward(p, C0, (tx_ix[k], tx_iz[k]), w, rx_ix[k], rx_iz[k], rho=rho) for k in range(2)])
    assert np.array_equal(M, M0)
    assert J == pytest.approx(np.sum((M0 - M_obs) ** 2), rel=1e-12)
    d = rng.standard_normal((n, n))
    h = 1e-2
    Jp, _ = oracle.misfit_gradient(p, C0 + h * d, tx_ix, tx_iz, w, rx_ix, rx_iz, M_obs, rho=rho)
    Jm, _ = oracle.misfit_gradient(p, C0 - h * d, tx_ix, tx_iz, w, rx_ix, rx_iz, M_obs, rho=rho)
    fd = (Jp - Jm) / (2 * h)
    assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)
