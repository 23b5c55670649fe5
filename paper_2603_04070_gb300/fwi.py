"""Classical FWI around the GPU misfit and gradient (Sec. II-B, Eqs. 5-7).

Eq. 7 updates the SoS map along the data-fidelity gradient, C_{k+1} = C_k + gamma_k g_k, with
gamma_k < 0 for a descent step. Three ways to choose the step are provided:

* ``steepest_descent``: the direction is -g_k. The trial step is scaled so that its largest
  change is ``alpha`` m/s, and ``alpha`` is halved until the misfit falls by the Armijo margin
  (sufficient decrease, c1 = 1e-4). The next iteration starts from twice the accepted ``alpha``.
* ``lbfgs``: the direction is -H_k g_k, with H_k the limited-memory BFGS inverse Hessian built
  from the last ``memory`` pairs (s, y) by the two-loop recursion (Nocedal and Wright, Numerical
  Optimization, Algorithm 7.4), with H_0 = (s^T y / y^T y) I. A unit step is tried first, then
  halved under the same Armijo test. The first iteration, with no pairs yet, is a steepest-descent
  step of ``alpha`` m/s. Pairs with s^T y <= 0 are skipped.
* ``newton_cg``: truncated Newton. The direction approximately solves H_k d = -g_k by conjugate
  gradients with exact Hessian-vector products (``dufwi_hvp``), stopped when the residual falls
  below ``cg_tol`` |g_k| or at the first direction of non-positive curvature (Nocedal and
  Wright, Algorithm 7.1; with no CG step taken the direction is -g_k, scaled to ``alpha`` m/s).
  A unit step is tried first, then halved under the Armijo test.

Each map of a batch is an independent problem: its own step sizes and curvature pairs. Maps are
evaluated together in one library call per trial step. A line search needs misfits only, so
it uses ``dufwi.misfit``, one forward sweep costing about a third of a gradient.

The SoS is clamped to [c_lo, c_hi] after every step, which keeps it physical and below the
stability limit of the time step. The paper's own FWI baseline adds total-variation
regularisation through ADMM (Sec. V); that comparison system is not reproduced here.

The ``evaluate`` callback ``(sos, need_grad) -> (J [B] float64, g [B, nz, nx] or None)``
defaults to the CUDA library. Tests can pass any other function with the same contract.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Callable

import torch

ARMIJO_C1 = 1e-4


@dataclass
class FWIResult:
    sos: torch.Tensor                                   # [B, nz, nx] final estimate
    misfits: list = field(default_factory=list)         # per iteration: J [B] (float64, host) at C_k
    steps: list = field(default_factory=list)           # per iteration: accepted step scale per map
    evaluations: int = 0                                # misfit-only calls
    gradients: int = 0                                  # gradient calls
    seconds: list = field(default_factory=list)         # wall time per iteration (device synchronised)
    cg_steps: list = field(default_factory=list)        # newton_cg: CG steps per map and iteration


def cuda_evaluator(problem, wavelet, geom, cd_obs, *, workspace=None):
    """(sos, need_grad) -> (J, g) through the library; one workspace reused by every call."""
    from . import dufwi
    n_maps = cd_obs.shape[0]
    if workspace is None:
        nbytes = dufwi.workspace_size(problem, geom, n_maps, gradient=True)
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=cd_obs.device)

    def evaluate(sos, need_grad):
        if need_grad:
            J, g = dufwi.misfit_gradient(problem, sos, wavelet, geom, cd_obs, workspace=workspace)
            return J, g
        return dufwi.misfit(problem, sos, wavelet, geom, cd_obs, workspace=workspace), None
    return evaluate


def _per_map(v: torch.Tensor, like: torch.Tensor) -> torch.Tensor:
    return v.reshape((-1,) + (1,) * (like.dim() - 1)).to(like.dtype)


def _dot(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Per-map inner products in FP64."""
    return (a.to(torch.float64) * b.to(torch.float64)).flatten(1).sum(1)


def _line_search(evaluate, c, J, g, d, scale, c_lo, c_hi, max_halvings, res):
    """Armijo backtracking per map along d with initial step scale[b] (d already a descent
    direction). Returns (new sos, new J, accepted scale); a map with no acceptable step keeps C_k
    and reports scale 0."""
    slope = _dot(g, d)                                   # < 0 for a descent direction
    accepted = torch.zeros_like(scale)
    c_new, J_new = c.clone(), J.clone()
    todo = torch.ones_like(scale, dtype=torch.bool)
    t = scale.clone()
    for _ in range(max_halvings + 1):
        trial = torch.clamp(c + _per_map(t, c) * d, c_lo, c_hi)
        Jt, _ = evaluate(trial, False)
        res.evaluations += 1
        ok = todo & (Jt <= J + ARMIJO_C1 * t * slope)
        if ok.any():
            c_new[ok] = trial[ok]
            J_new[ok] = Jt[ok]
            accepted[ok] = t[ok]
            todo &= ~ok
        if not todo.any():
            break
        t = torch.where(todo, 0.5 * t, t)
    return c_new, J_new, accepted


def steepest_descent(evaluate: Callable, sos0: torch.Tensor, iters: int, *, alpha: float = 20.0,
                     c_lo: float = 1300.0, c_hi: float = 3000.0, max_halvings: int = 6,
                     sync: bool = True) -> FWIResult:
    """Eq. 7 with gamma_k = -alpha_k / max|g_k| (per map), alpha_k by Armijo backtracking."""
    c = sos0.clone()
    res = FWIResult(sos=c)
    a = torch.full((c.shape[0],), float(alpha), dtype=torch.float64, device=c.device)
    J, g = evaluate(c, True)
    res.gradients += 1
    for _ in range(iters):
        t0 = time.perf_counter()
        res.misfits.append(J.detach().cpu().clone())
        gmax = g.abs().flatten(1).amax(1).to(torch.float64).clamp_min(1e-30)
        d = -g
        c, J_acc, step = _line_search(evaluate, c, J, g, d, a / gmax, c_lo, c_hi, max_halvings, res)
        res.steps.append((step * gmax).cpu())           # accepted alpha in m/s
        a = torch.where(step > 0, 2.0 * step * gmax, 0.25 * a)
        J, g = evaluate(c, True)
        res.gradients += 1
        if sync and c.is_cuda:
            torch.cuda.synchronize()
        res.seconds.append(time.perf_counter() - t0)
    res.misfits.append(J.detach().cpu().clone())
    res.sos = c
    return res


def cuda_hessvec(problem, wavelet, geom, cd_obs, *, workspace=None):
    """(sos, v) -> H v [B, nz, nx], the exact Hessian-vector product of the misfit (``dufwi_hvp``)."""
    from . import dufwi
    n_maps = cd_obs.shape[0]
    if workspace is None:
        nbytes = dufwi.second_order_workspace_size(problem, geom, n_maps)
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=cd_obs.device)

    def hessvec(sos, v):
        return dufwi.hvp(problem, sos, wavelet, geom, cd_obs, v.contiguous(), workspace=workspace)
    return hessvec


def cg_newton_direction(g: torch.Tensor, hessvec, sos: torch.Tensor, cg_iters: int, cg_tol: float):
    """Per map, an approximate solution d of H d = -g by conjugate gradients (all maps advance
    together: one Hessian-vector call per CG iteration, on directions scaled to unit max-norm).
    Returns (d, cg steps taken per map). A map stops at |r| <= cg_tol |g| or at the first
    direction p with p^T H p <= 0."""
    B = g.shape[0]
    gd = g.to(torch.float64)
    d = torch.zeros_like(gd)
    r = -gd.clone()                                   # residual of H d = -g at d = 0
    p = r.clone()
    rr = _dot(r, r)
    stop = rr.sqrt() <= cg_tol * _dot(gd, gd).sqrt()
    steps = torch.zeros(B, dtype=torch.int64, device=g.device)
    for _ in range(cg_iters):
        if bool(stop.all()):
            break
        # H p = |p|_inf H (p / |p|_inf): the product is linear, and a unit-scale direction keeps
        # the FP32 sweeps far from underflow (p has the scale of the gradient, ~1e-17 here)
        pm = p.abs().flatten(1).amax(1).clamp_min(1e-300)
        Hp = hessvec(sos, (p / _per_map(pm, p)).to(sos.dtype)).to(torch.float64) * _per_map(pm, p)
        pHp = _dot(p, Hp)
        neg = ~stop & (pHp <= 0)
        stop |= neg
        act = ~stop
        a = torch.where(act, rr / torch.where(pHp > 0, pHp, torch.ones_like(pHp)), torch.zeros_like(rr))
        d = d + _per_map(a, d) * p
        r = r - _per_map(a, r) * Hp
        rr_new = _dot(r, r)
        steps = steps + act.to(torch.int64)
        stop |= act & (rr_new.sqrt() <= cg_tol * _dot(gd, gd).sqrt())
        beta = torch.where(act, rr_new / torch.where(rr > 0, rr, torch.ones_like(rr)), torch.zeros_like(rr))
        p = torch.where(_per_map(act, p).bool(), r + _per_map(beta, p) * p, p)
        rr = torch.where(act, rr_new, rr)
    return d, steps


def newton_cg(evaluate: Callable, hessvec: Callable, sos0: torch.Tensor, iters: int, *, cg_iters: int = 10,
              cg_tol: float = 0.1, alpha: float = 20.0, c_lo: float = 1300.0, c_hi: float = 3000.0,
              max_halvings: int = 6, sync: bool = True) -> FWIResult:
    """Eq. 7 with gamma_k g_k replaced by the truncated-Newton step t_k d_k, H_k d_k ~ -g_k."""
    c = sos0.clone()
    res = FWIResult(sos=c)
    J, g = evaluate(c, True)
    res.gradients += 1
    for _ in range(iters):
        t0 = time.perf_counter()
        res.misfits.append(J.detach().cpu().clone())
        d, steps = cg_newton_direction(g, hessvec, c, cg_iters, cg_tol)
        res.cg_steps.append(steps.cpu())
        scale = torch.ones(c.shape[0], dtype=torch.float64, device=c.device)
        for b in range(c.shape[0]):
            if int(steps[b]) == 0:             # no CG step: steepest descent of alpha m/s
                d[b] = -g[b].to(torch.float64)
                scale[b] = alpha / float(g[b].abs().max().clamp_min(1e-30))
        c, _, step = _line_search(evaluate, c, J, g, d.to(c.dtype), scale, c_lo, c_hi, max_halvings, res)
        res.steps.append(step.cpu())
        J, g = evaluate(c, True)
        res.gradients += 1
        if sync and c.is_cuda:
            torch.cuda.synchronize()
        res.seconds.append(time.perf_counter() - t0)
    res.misfits.append(J.detach().cpu().clone())
    res.sos = c
    return res


def two_loop(g: torch.Tensor, S: list, Y: list) -> torch.Tensor:
    """H_k g for one map by the L-BFGS two-loop recursion; S, Y hold the pairs oldest first.
    H_0 = (s^T y / y^T y) I from the newest pair (identity with no pairs)."""
    q = g.to(torch.float64).flatten().clone()
    rho = [1.0 / float(torch.dot(y, s)) for s, y in zip(S, Y)]
    al = [0.0] * len(S)
    for i in range(len(S) - 1, -1, -1):
        al[i] = rho[i] * float(torch.dot(S[i], q))
        q -= al[i] * Y[i]
    if S:
        q *= float(torch.dot(S[-1], Y[-1])) / float(torch.dot(Y[-1], Y[-1]))
    for i in range(len(S)):
        b = rho[i] * float(torch.dot(Y[i], q))
        q += (al[i] - b) * S[i]
    return q.reshape(g.shape)


def lbfgs(evaluate: Callable, sos0: torch.Tensor, iters: int, *, memory: int = 5, alpha: float = 20.0,
          c_lo: float = 1300.0, c_hi: float = 3000.0, max_halvings: int = 6, sync: bool = True) -> FWIResult:
    """Eq. 7 with gamma_k g_k replaced by the L-BFGS step -t_k H_k g_k (unit step first)."""
    c = sos0.clone()
    res = FWIResult(sos=c)
    B = c.shape[0]
    S = [[] for _ in range(B)]
    Y = [[] for _ in range(B)]
    J, g = evaluate(c, True)
    res.gradients += 1
    for _ in range(iters):
        t0 = time.perf_counter()
        res.misfits.append(J.detach().cpu().clone())
        d = torch.empty_like(g, dtype=torch.float64)
        scale = torch.ones(B, dtype=torch.float64, device=c.device)
        for b in range(B):
            if S[b]:
                d[b] = -two_loop(g[b], S[b], Y[b])
            else:
                d[b] = -g[b].to(torch.float64)
                scale[b] = alpha / float(g[b].abs().max().clamp_min(1e-30))
        c_prev, g_prev = c, g
        c, J_new, step = _line_search(evaluate, c, J, g, d.to(c.dtype), scale, c_lo, c_hi, max_halvings, res)
        res.steps.append(step.cpu())
        J, g = evaluate(c, True)
        res.gradients += 1
        for b in range(B):
            s = (c[b] - c_prev[b]).to(torch.float64).flatten()
            y = (g[b] - g_prev[b]).to(torch.float64).flatten()
            if float(torch.dot(s, y)) > 0.0:
                S[b].append(s)
                Y[b].append(y)
                if len(S[b]) > memory:
                    S[b].pop(0)
                    Y[b].pop(0)
        if sync and c.is_cuda:
            torch.cuda.synchronize()
        res.seconds.append(time.perf_counter() - t0)
    res.misfits.append(J.detach().cpu().clone())
    res.sos = c
    return res
