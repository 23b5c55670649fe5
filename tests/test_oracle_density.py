"""Pins of the oracle's variable-density operator (Eq. 1 with rho(x, z)), on the CPU.

The density term rho div((1/rho) grad u) is discretised with staggered first differences and
half-point buoyancies. It is pinned to facts fixed by the mathematics and the physics:

* the moment conditions that define the staggered weights;
* exact divergence of b grad u for polynomial u and b;
* symmetry and definiteness of the operator (the discrete adjoint relies on it);
* the analytic 2-D Green's function at constant density;
* the normal-incidence reflection coefficient (rho2 - rho1)/(rho2 + rho1) of a density step
  at equal speed, which holds at every angle, so a point source sees an exact mirror image;
* invariance of the traces under a global scaling of the density;
* reciprocity, the adjoint dot-product identity and finite differences of the misfit.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_04070_gb300 import inputs


def _ricker(t, f0, delay):
    a = (math.pi * f0 * (t - delay)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def _green_trace(r, c, times, f0, delay, n_gl=3000):
    """u_tt - c^2 lap u = w(t) delta(x) in 2-D, by Gauss-Legendre quadrature of
    (1/(2 pi c^2)) int_0^acosh(ct/r) w(t - r cosh(s)/c) ds."""
    xg, wg = np.polynomial.legendre.leggauss(n_gl)
    out = np.zeros(times.size)
    for i, t in enumerate(times):
        if c * t <= r:
            continue
        smax = math.acosh(c * t / r)
        s = 0.5 * smax * (xg + 1.0)
        out[i] = 0.5 * smax * np.sum(wg * _ricker(t - (r / c) * np.cosh(s), f0, delay)) / (2 * math.pi * c * c)
    return out


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_staggered_moment_conditions(order):
    """sum_k s_k (2k-1)^(2m+1) = 1 for m = 0 and 0 for m = 1..M-1 (exact derivative of odd
    monomials from samples at +-(k - 1/2) dx)."""
    s = oracle.stagger_coeffs(order)
    k = np.arange(1, s.size + 1)
    for m in range(s.size):
        want = 1.0 if m == 0 else 0.0
        assert abs(np.sum(s * (2 * k - 1.0) ** (2 * m + 1)) - want) < 1e-13


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_div_b_grad_exact_on_polynomials(order):
    """D-(b D+u) = d/dx(b du/dx) + d/dz(b du/dz) exactly for u of degree order and b linear,
    at nodes whose whole stencil lies inside the grid (dx = 1)."""
    M = order // 2
    p = oracle.Problem(nx=6, nz=6, dx=1.0, dt=1.0, nt=1, pml=2 * M + 2, fd_order=order)
    X, Z = np.meshgrid(np.arange(p.nxp, dtype=np.float64), np.arange(p.nzp, dtype=np.float64))
    cx, cz, L = (p.nxp - 1) / 2, (p.nzp - 1) / 2, 8.0
    bfun = lambda x, z: 1.0 + 0.05 * (x - cx) - 0.03 * (z - cz)
    deg = order
    ux = ((X - cx) / L) ** deg
    uz = ((Z - cz) / L) ** deg
    u = ux + 0.5 * uz + 0.25 * ((X - cx) / L) * ((Z - cz) / L) ** (deg - 1)
    bx = bfun(X + 0.5, Z)
    bz = bfun(X, Z + 0.5)
    out = oracle.div_b_grad(p, bx, bz, u)
    # analytic: d/dx(b u_x) + d/dz(b u_z) with b_x = 0.05, b_z = -0.03
    xs, zs = (X - cx) / L, (Z - cz) / L
    u_x = deg * xs ** (deg - 1) / L + 0.25 * zs ** (deg - 1) / L
    u_xx = deg * (deg - 1) * xs ** (deg - 2) / L ** 2
    u_z = 0.5 * deg * zs ** (deg - 1) / L + 0.25 * xs * (deg - 1) * zs ** (deg - 2) / L
    u_zz = 0.5 * deg * (deg - 1) * zs ** (deg - 2) / L ** 2 + 0.25 * xs * (deg - 1) * (deg - 2) * zs ** max(deg - 3, 0) / L ** 2 * (deg > 2)
    b = bfun(X, Z)
    want = 0.05 * u_x + b * u_xx - 0.03 * u_z + b * u_zz
    h = 2 * M - 1
    sl = (slice(h, p.nzp - h), slice(h, p.nxp - h))
    assert np.max(np.abs(out[sl] - want[sl])) <= 1e-11 * np.max(np.abs(want[sl]))


def test_div_b_grad_symmetric_negative_and_zero_on_constants():
    rng = np.random.default_rng(0)
    p = oracle.Problem(nx=14, nz=11, dx=1e-4, dt=1e-8, nt=1, pml=5, fd_order=8)
    rho = np.exp(rng.uniform(np.log(500.0), np.log(3000.0), size=(p.nzp, p.nxp)))
    bx, bz = oracle.buoyancy(p, rho)
    assert np.all(bx[:, -1] == 0.0) and np.all(bz[-1, :] == 0.0)
    assert bx[3, 4] == pytest.approx(2.0 / (rho[3, 4] + rho[3, 5]), rel=1e-15)
    u, v = rng.standard_normal((2, p.nzp, p.nxp))
    Lu, Lv = oracle.div_b_grad(p, bx, bz, u), oracle.div_b_grad(p, bx, bz, v)
    assert abs(np.sum(Lu * v) - np.sum(u * Lv)) <= 1e-12 * np.sum(np.abs(Lu * v))
    assert np.sum(Lu * u) < 0.0
    c = np.full((p.nzp, p.nxp), 3.7)
    Lc = oracle.div_b_grad(p, bx, bz, c)
    h = 7                                   # nodes whose stencil stays inside the grid
    assert np.all(Lc[h:-h, h:-h] == 0.0)


def test_constant_density_green_function():
    """At constant density the staggered operator is an 8th-order Laplacian: the homogeneous
    trace matches the analytic Green's function like the compact one does."""
    c, dx, dt, f0, n = 1500.0, 1e-4, 5e-9, 1.0e6, 161
    nt = 1400
    p = oracle.Problem(nx=n, nz=n, dx=dx, dt=dt, nt=nt, pml=20, pml_cref=c, fd_order=8)
    w = _ricker(np.arange(nt) * dt, f0, 1.5 / f0)
    rxs = [(105, 80), (80, 45)]
    rho = np.full((n, n), 1000.0)
    tr = oracle.forward(p, np.full((n, n), c), (80, 80), w, np.array([r[0] for r in rxs]),
                        np.array([r[1] for r in rxs]), rho=rho)
    for k, r in enumerate(rxs):
        ref = _green_trace(math.hypot(r[0] - 80, r[1] - 80) * dx, c, np.arange(nt) * dt, f0, 1.5 / f0)
        assert np.linalg.norm(tr[:, k] - ref) / np.linalg.norm(ref) < 2e-3


def _step_reflection_error(f0, nt, rho2, rho1=1000.0):
    """Relative L2 error of the simulated reflection against R times the homogeneous field at the
    receiver's mirror image, for a density step below row 90 (interface at z = 90.5)."""
    c, dx, dt, n = 1500.0, 1e-4, 5e-9, 161
    p = oracle.Problem(nx=n, nz=n, dx=dx, dt=dt, nt=nt, pml=20, pml_cref=c, fd_order=8)
    w = _ricker(np.arange(nt) * dt, f0, 1.5 / f0)
    C = np.full((n, n), c)
    rho = np.full((n, n), rho1)
    rho[91:, :] = rho2
    src, rec, mirror = (80, 70), (80, 62), (80, 119)            # 119 = 2 * 90.5 - 62
    tr = oracle.forward(p, C, src, w, np.array([rec[0]]), np.array([rec[1]]), rho=rho)[:, 0]
    hom = oracle.forward(p, C, src, w, np.array([rec[0], mirror[0]]), np.array([rec[1], mirror[1]]),
                         rho=np.full((n, n), rho1))
    R = (rho2 - rho1) / (rho2 + rho1)
    want = R * hom[:, 1]
    return np.linalg.norm(tr - hom[:, 0] - want) / np.linalg.norm(want), p, C, src, rec, w, hom[:, 0]


@pytest.mark.parametrize("rho2", [2000.0, 400.0])
def test_density_step_reflection_coefficient(rho2):
    """Equal speed, density rho1 above the interface and rho2 below: the reflected field equals
    R = (rho2 - rho1)/(rho2 + rho1) times the homogeneous field at the receiver's mirror image
    (exact for a point source, since R does not depend on the angle at equal speed). The
    discrete interface leaves an error of second order in frequency: about 0.9% at 0.7 MHz,
    twice that at 1 MHz (15 cells per wavelength)."""
    e07, p, C, src, rec, w, direct = _step_reflection_error(0.7e6, 1700, rho2)
    e10 = _step_reflection_error(1.0e6, 1500, rho2)[0]
    assert e07 < 1.2e-2, e07
    assert 1.7 < e10 / e07 < 2.5, (e10, e07)
    # control: the compact constant-density path (no density map) gives the direct field only
    tr_c = oracle.forward(p, C, src, w, np.array([rec[0]]), np.array([rec[1]]))[:, 0]
    assert np.linalg.norm(tr_c - direct) <= 5e-3 * np.linalg.norm(direct)


def test_density_scaling_leaves_traces_unchanged():
    rng = np.random.default_rng(1)
    p = oracle.Problem(nx=24, nz=20, dx=1e-4, dt=1e-8, nt=200, pml=8, fd_order=8)
    C = 1540.0 + 40.0 * rng.standard_normal((20, 24))
    rho = 1000.0 + 300.0 * rng.uniform(size=(20, 24))
    w = inputs.ricker(p.nt, p.dt, 2e6).astype(np.float64)
    a = oracle.forward(p, C, (5, 3), w, np.array([18, 2]), np.array([15, 19]), rho=rho)
    b = oracle.forward(p, C, (5, 3), w, np.array([18, 2]), np.array([15, 19]), rho=7.5 * rho)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
    c = oracle.forward(p, C, (5, 3), w, np.array([18, 2]), np.array([15, 19]))
    assert np.max(np.abs(a - c)) > 1e-2 * np.max(np.abs(a))     # the density matters


def test_density_reciprocity():
    """trace(s->r) kappa_s = trace(r->s) kappa_r with kappa = rho C^2 dt^2 at physical nodes."""
    rng = np.random.default_rng(2)
    p = oracle.Problem(nx=30, nz=30, dx=1e-4, dt=1e-8, nt=300, pml=10, fd_order=8)
    C = 1540.0 + 40.0 * rng.standard_normal((30, 30))
    rho = 1000.0 + 500.0 * rng.uniform(size=(30, 30))
    w = inputs.ricker(p.nt, p.dt, 2e6).astype(np.float64)
    s, r = (5, 3), (22, 17)
    t_sr = oracle.forward(p, C, s, w, np.array([r[0]]), np.array([r[1]]), rho=rho)[:, 0]
    t_rs = oracle.forward(p, C, r, w, np.array([s[0]]), np.array([s[1]]), rho=rho)[:, 0]
    ks = rho[s[1], s[0]] * C[s[1], s[0]] ** 2
    kr = rho[r[1], r[0]] * C[r[1], r[0]] ** 2
    assert np.max(np.abs(t_sr * ks - t_rs * kr)) <= 1e-11 * np.max(np.abs(t_sr * ks))


def test_density_adjoint_dot_product():
    rng = np.random.default_rng(4)
    p = oracle.Problem(nx=26, nz=22, dx=1e-4, dt=1e-8, nt=200, pml=8, fd_order=8)
    C = 1540.0 + 40.0 * rng.standard_normal((22, 26))
    rho = 1000.0 + 800.0 * rng.uniform(size=(22, 26))
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


def test_density_gradient_finite_differences():
    rng = np.random.default_rng(5)
    n, nt = 18, 180
    p = oracle.Problem(nx=n, nz=n, dx=1e-4, dt=1e-8, nt=nt, pml=6, fd_order=8)
    rho = 1000.0 + 600.0 * rng.uniform(size=(n, n))
    C_true = 1540.0 + 40.0 * rng.standard_normal((n, n))
    C0 = 1540.0 + 5.0 * rng.standard_normal((n, n))
    tx_ix, tx_iz = np.array([3, 12], np.int32), np.array([0, 0], np.int32)
    rx_ix = np.tile(np.array([0, 4, 8, 12, 17], np.int32), (2, 1))
    rx_iz = np.tile(np.array([0, 0, 17, 0, 7], np.int32), (2, 1))
    w = inputs.ricker(nt, p.dt, 2e6).astype(np.float64)
    M_obs = np.stack([oracle.forward(p, C_true, (tx_ix[k], tx_iz[k]), w, rx_ix[k], rx_iz[k], rho=rho)
                      for k in range(2)])
    J, g = oracle.misfit_gradient(p, C0, tx_ix, tx_iz, w, rx_ix, rx_iz, M_obs, rho=rho)
    Jc, gc = oracle.misfit_gradient(p, C0, tx_ix, tx_iz, w, rx_ix, rx_iz, M_obs, ckpt=37, rho=rho)
    assert Jc == J and np.array_equal(gc, g)
    d = rng.standard_normal((n, n))
    h = 1e-2
    Jp, _ = oracle.misfit_gradient(p, C0 + h * d, tx_ix, tx_iz, w, rx_ix, rx_iz, M_obs, rho=rho)
    Jm, _ = oracle.misfit_gradient(p, C0 - h * d, tx_ix, tx_iz, w, rx_ix, rx_iz, M_obs, rho=rho)
    fd = (Jp - Jm) / (2 * h)
    assert abs(fd - np.sum(g * d)) <= 1e-6 * abs(fd)
