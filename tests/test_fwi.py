"""Classical FWI loop (Eq. 7) and the ring-phantom inputs, on the CPU.

The L-BFGS recursion is pinned to the dense BFGS inverse-Hessian update and to the secant
condition. Both loops are run on convex quadratics with known minimisers, and on a tiny
ring problem with the oracle as the misfit/gradient callback."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_04070_gb300 import fwi, inputs


def _pairs(n, m, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)                    # SPD: every pair has s^T y > 0
    S = [torch.from_numpy(rng.standard_normal(n)) for _ in range(m)]
    Y = [torch.from_numpy(A @ s.numpy()) for s in S]
    return S, Y


def _dense_bfgs_inverse(S, Y):
    """H from H0 = (s^T y / y^T y) I (newest pair) by the BFGS inverse update, oldest pair first."""
    n = S[0].numel()
    s_, y_ = S[-1].numpy(), Y[-1].numpy()
    H = (s_ @ y_) / (y_ @ y_) * np.eye(n)
    for s, y in zip(S, Y):
        s, y = s.numpy(), y.numpy()
        r = 1.0 / (y @ s)
        V = np.eye(n) - r * np.outer(y, s)
        H = V.T @ H @ V + r * np.outer(s, s)
    return H


@pytest.mark.parametrize("m", [1, 3, 5])
def test_two_loop_equals_dense_bfgs_inverse(m):
    S, Y = _pairs(12, m, seed=m)
    g = torch.from_numpy(np.random.default_rng(99).standard_normal(12))
    want = _dense_bfgs_inverse(S, Y) @ g.numpy()
    got = fwi.two_loop(g, S, Y).numpy()
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)


def test_two_loop_secant_condition_and_empty_memory():
    S, Y = _pairs(10, 4, seed=7)
    assert torch.allclose(fwi.two_loop(Y[-1], S, Y), S[-1], rtol=1e-10, atol=1e-12)   # H y_k = s_k
    g = torch.arange(6, dtype=torch.float64)
    assert torch.equal(fwi.two_loop(g, [], []), g)


def _quadratic(n_maps=2, n=64, seed=0):
    rng = np.random.default_rng(seed)
    w = torch.from_numpy(np.logspace(0, 2, n).reshape(1, 8, n // 8).repeat(n_maps, 0))
    cstar = torch.from_numpy(1500.0 + rng.uniform(-50, 50, size=(n_maps, 8, n // 8)))

    def evaluate(c, need_grad):
        r = c.to(torch.float64) - cstar
        J = (w * r * r).flatten(1).sum(1)
        return J, (2.0 * w * r).to(c.dtype) if need_grad else None
    return evaluate, cstar


def _quadratic_hessvec(n_maps=2, n=64):
    w = torch.from_numpy(np.logspace(0, 2, n).reshape(1, 8, n // 8).repeat(n_maps, 0))
    return lambda c, v: (2.0 * w * v.to(torch.float64)).to(v.dtype)


def test_cg_direction_solves_newton_system_exactly():
    """CG on H = diag(2w) (64 distinct eigenvalues, condition number 100): with enough steps
    d = -H^-1 g to rounding, and the residual test, not the step cap, ends it (finite-precision
    CG needs somewhat more than the 64 steps of exact arithmetic)."""
    rng = np.random.default_rng(3)
    g = torch.from_numpy(rng.standard_normal((2, 8, 8)))
    hv = _quadratic_hessvec()
    d, steps = fwi.cg_newton_direction(g, hv, torch.zeros_like(g), 200, 1e-12)
    w = torch.from_numpy(np.logspace(0, 2, 64).reshape(8, 8))
    assert torch.allclose(d, -g / (2.0 * w), rtol=1e-8, atol=1e-12)
    assert torch.all(steps < 200)


def test_newton_cg_converges_in_one_step_on_quadratic():
    evaluate, cstar = _quadratic()
    c0 = torch.full(cstar.shape, 1500.0, dtype=torch.float64)
    res = fwi.newton_cg(evaluate, _quadratic_hessvec(), c0, 2, cg_iters=100, cg_tol=1e-12, sync=False)
    J = torch.stack(res.misfits)
    assert torch.all(J[1] <= 1e-16 * J[0])
    assert torch.allclose(res.sos, cstar, atol=1e-6)
    assert torch.all(res.steps[0] == 1.0)                      # the unit Newton step is accepted


def test_truncated_newton_is_monotone_and_handles_negative_curvature():
    evaluate, cstar = _quadratic(seed=4)
    c0 = torch.full(cstar.shape, 1500.0, dtype=torch.float64)
    res = fwi.newton_cg(evaluate, _quadratic_hessvec(), c0, 8, cg_iters=3, cg_tol=1e-3, sync=False)
    J = torch.stack(res.misfits)
    assert torch.all(J[1:] <= J[:-1]) and J[-1].max() <= 1e-3 * J[0].min()
    # a Hessian that reports negative curvature: no CG step, steepest descent of alpha m/s instead
    bad = fwi.newton_cg(evaluate, lambda c, v: -v, c0, 3, cg_iters=5, sync=False)
    assert all(int(s.max()) == 0 for s in bad.cg_steps)
    Jb = torch.stack(bad.misfits)
    assert torch.all(Jb[1:] < Jb[:-1])


def test_lbfgs_converges_on_quadratic():
    evaluate, cstar = _quadratic()
    c0 = torch.full(cstar.shape, 1500.0, dtype=torch.float64)
    res = fwi.lbfgs(evaluate, c0, 60, memory=5, alpha=20.0, sync=False)
    J = torch.stack(res.misfits)
    assert torch.all(J[1:] <= J[:-1])
    assert torch.all(J[-1] <= 1e-8 * J[0])
    assert torch.allclose(res.sos, cstar, atol=1e-3)


def test_steepest_descent_monotone_on_quadratic():
    evaluate, cstar = _quadratic(seed=1)
    c0 = torch.full(cstar.shape, 1500.0, dtype=torch.float64)
    res = fwi.steepest_descent(evaluate, c0, 30, alpha=20.0, sync=False)
    J = torch.stack(res.misfits)
    assert torch.all(J[1:] < J[:-1])
    assert torch.all(J[-1] < 0.05 * J[0])
    for k, st in enumerate(res.steps):
        assert torch.all(st > 0), k


def test_line_search_respects_bounds():
    evaluate, cstar = _quadratic(seed=2)
    c0 = torch.full(cstar.shape, 1500.0, dtype=torch.float64)
    res = fwi.steepest_descent(evaluate, c0, 5, alpha=500.0, c_lo=1480.0, c_hi=1520.0, sync=False)
    assert res.sos.min() >= 1480.0 and res.sos.max() <= 1520.0


# ------------------------------------------------------------------ ring-phantom inputs
def test_ring_phantom_geometry():
    wl = inputs.ring_phantom(seed=0, n_maps=3)
    assert (wl.nx, wl.nz, wl.nt) == (188, 188, 1034)
    assert wl.dx == pytest.approx(0.1 / 188) and wl.dt == pytest.approx(90.243e-9)
    assert wl.elem_ix.min() >= 0 and wl.elem_ix.max() <= 187 and wl.elem_iz.min() >= 0 and wl.elem_iz.max() <= 187
    c = 93.5
    r = np.hypot(wl.elem_ix - c, wl.elem_iz - c)
    assert np.all(np.abs(r - 93.5) <= 0.75)                       # on the inscribed 10 cm ring
    assert wl.n_tx == 16 and wl.n_rx == 3
    for j in range(16):                                           # opposite element and its neighbours
        assert sorted(wl.rx_elem[j]) == sorted([(j + 7) % 16, (j + 8) % 16, (j + 9) % 16])
    vals = set(np.unique(wl.sos_true).tolist())
    assert 1500.0 in vals and vals <= {1500.0, 1588.0, 2700.0} and len(vals) >= 2
    # printed maximum damping of the 20-cell layer at this grid (Sec. IV)
    p = oracle.Problem(nx=188, nz=188, dx=wl.dx, dt=wl.dt, nt=10, pml_cref=wl.pml_cref)
    assert oracle.d0(p) == pytest.approx(1.46e6, rel=1e-3)
    c8 = oracle.fd_coeffs(8)                                      # leapfrog stability limit in 2-D
    nyq = abs(c8[0] + 2 * sum(c8[k] * (-1) ** k for k in range(1, c8.size)))
    assert wl.c_max * wl.dt / wl.dx < 2.0 / math.sqrt(2.0 * nyq)


def test_rods_inside_ring_and_disjoint():
    rng = inputs.rng_for(5)
    dx = 0.1 / 188
    for _ in range(20):
        m = inputs.phantom_rods_map(rng, 188, dx, 93.5)
        inside = np.argwhere(m != 1500.0)
        rr = np.hypot(inside[:, 1] - 93.5, inside[:, 0] - 93.5)
        assert rr.max() * dx <= 93.5 * dx - 5e-3 + 1.5 * dx       # a rod radius clear of the ring


def test_awgn_snr():
    rng = inputs.rng_for(3)
    cd = rng.standard_normal((2, 16, 1034, 3)).astype(np.float32) * np.array([1.0, 5.0]).reshape(2, 1, 1, 1)
    noisy = inputs.add_awgn(inputs.rng_for(4), cd, 30.0)
    for b in range(2):
        snr = 10 * math.log10(np.mean(cd[b].astype(np.float64) ** 2) / np.mean((noisy[b] - cd[b]).astype(np.float64) ** 2))
        assert abs(snr - 30.0) < 0.15


# ------------------------------------------------------------------ FWI with the oracle
def test_fwi_loops_with_oracle_decrease_misfit():
    """Both loops on a 40 x 40 ring problem (8 elements, 300 steps) with oracle gradients."""
    wl = inputs.ring_phantom(seed=1, n_maps=1, n=40, nt=300, n_elem=8, width_m=40 * 0.1 / 188,
                             rod_diameter_m=4e-3)
    p = oracle.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml=wl.pml, pml_R=wl.pml_R,
                       pml_cref=wl.pml_cref, fd_order=wl.fd_order)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    w = wl.wavelet.astype(np.float64)
    obs = np.stack([oracle.forward(p, wl.sos_true[0].astype(np.float64), (tix[k], tiz[k]), w, rix[k], riz[k])
                    for k in range(wl.n_tx)])

    def evaluate(c, need_grad):
        J, g = oracle.misfit_gradient(p, c[0].numpy().astype(np.float64), tix, tiz, w, rix, riz, obs)
        return torch.tensor([J], dtype=torch.float64), torch.from_numpy(g[None]) if need_grad else None

    c0 = torch.from_numpy(wl.sos_start.astype(np.float64))
    for loop in (fwi.steepest_descent, fwi.lbfgs):
        res = loop(evaluate, c0, 3, alpha=20.0, sync=False)
        J = torch.stack(res.misfits)[:, 0]
        assert torch.all(J[1:] < J[:-1]), (loop.__name__, J)
        assert J[-1] < 0.9 * J[0], (loop.__name__, J)
        assert res.gradients == 4 and res.evaluations >= 3
