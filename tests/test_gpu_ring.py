"""The paper's ring geometry (Sec. IV, VII) on the GPU: parity with the oracle at full size, the
misfit-only entry point, and the classical FWI loop (Eq. 7) driven by the CUDA library."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_04070_gb300 import inputs

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def d():
    from paper_2603_04070_gb300 import build_lib
    build_lib.build()
    from paper_2603_04070_gb300 import dufwi
    return dufwi


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _oracle_problem(wl):
    return oracle.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml=wl.pml, pml_R=wl.pml_R,
                          pml_cref=wl.pml_cref, fd_order=wl.fd_order)


def _noisy_observed(wl, seed=11):
    """Oracle traces of the true maps plus 30 dB white noise, as FP32 (both sides see these)."""
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    w = wl.wavelet.astype(np.float64)
    clean = np.stack([np.stack([oracle.forward(p, wl.sos_true[b].astype(np.float64), (tix[k], tiz[k]), w,
                                               rix[k], riz[k]) for k in range(wl.n_tx)])
                      for b in range(wl.n_maps)])
    return inputs.add_awgn(inputs.rng_for(seed), clean, 30.0)


def _setup(d, wl, **kw):
    pb = d.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml_cells=wl.pml, pml_R=wl.pml_R,
                   pml_cref=wl.pml_cref, fd_order=wl.fd_order, c_max=wl.c_max, **kw)
    return pb, d.Geometry.from_workload(wl)


@pytest.mark.parametrize("ckpt", [0, 100])
def test_ring_phantom_full_size_gradient(d, ckpt):
    """188 x 188, 16 transmits x 3 receivers, 1034 steps, noisy data: traces, misfit and gradient
    against the oracle, with histories stored for every step and with checkpoints every 100."""
    wl = inputs.ring_phantom(seed=2, n_maps=1)
    obs = _noisy_observed(wl)
    pb, geom = _setup(d, wl, ckpt_interval=ckpt)
    sos = torch.from_numpy(wl.sos_start).cuda()
    J, g, cd = d.misfit_gradient(pb, sos, torch.from_numpy(wl.wavelet).cuda(), geom, torch.from_numpy(obs).cuda(),
                                 return_cd=True, check=True)
    torch.cuda.synchronize()
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    Jr, gr, Mr = oracle.misfit_gradient(p, wl.sos_start[0].astype(np.float64), tix, tiz,
                                        wl.wavelet.astype(np.float64), rix, riz, obs[0].astype(np.float64),
                                        return_traces=True)
    assert rel_l2(cd[0].cpu().numpy(), Mr) <= TRACE_TOL
    assert abs(float(J[0]) - Jr) <= 1e-4 * Jr
    assert rel_l2(g[0].cpu().numpy(), gr) <= GRAD_TOL


def test_misfit_only_matches_gradient_call_and_oracle(d):
    """dufwi_misfit gives the misfit of dufwi_misfit_gradient bit for bit, and its simulated data."""
    wl = inputs.ring_phantom(seed=3, n_maps=3, n=72, nt=500, n_elem=12, width_m=72 * 0.1 / 188,
                             rod_diameter_m=6e-3)
    obs = _noisy_observed(wl)
    pb, geom = _setup(d, wl, ckpt_interval=50)
    sos = torch.from_numpy(wl.sos_start).cuda()
    sos[1] += 12.0                                  # three different maps
    sos[2] = torch.from_numpy(wl.sos_true[2]).cuda()
    wav = torch.from_numpy(wl.wavelet).cuda()
    o = torch.from_numpy(obs).cuda()
    J1, _, cd1 = d.misfit_gradient(pb, sos, wav, geom, o, return_cd=True, check=True)
    cd2 = torch.empty_like(cd1)
    J2 = d.misfit(pb, sos, wav, geom, o, cd_sim=cd2, check=True)
    torch.cuda.synchronize()
    assert torch.equal(J1, J2)
    assert torch.equal(cd1, cd2)
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    for b in range(3):
        Jr, _ = oracle.misfit_gradient(p, sos[b].cpu().numpy().astype(np.float64), tix, tiz,
                                       wl.wavelet.astype(np.float64), rix, riz, obs[b].astype(np.float64))
        assert abs(float(J2[b]) - Jr) <= 1e-4 * Jr


def test_classical_fwi_on_gpu(d):
    """Three L-BFGS and three steepest-descent iterations of Eq. 7 at full ring size: the misfit
    falls every iteration, the estimate stays finite and within the bounds."""
    from paper_2603_04070_gb300 import fwi
    wl = inputs.ring_phantom(seed=4, n_maps=2)
    pb, geom = _setup(d, wl)
    wav = torch.from_numpy(wl.wavelet).cuda()
    clean = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), wav, geom)
    obs = torch.from_numpy(inputs.add_awgn(inputs.rng_for(5), clean.cpu().numpy(), 30.0)).cuda()
    ev = fwi.cuda_evaluator(pb, wav, geom, obs)
    c0 = torch.from_numpy(wl.sos_start).cuda()
    for loop in (fwi.lbfgs, fwi.steepest_descent):
        res = loop(ev, c0, 3)
        J = torch.stack(res.misfits)
        assert torch.all(J[1:] < J[:-1]), (loop.__name__, J)
        assert torch.isfinite(res.sos).all()
        assert res.sos.min() >= 1300.0 and res.sos.max() <= 3000.0


def test_autotune_gradient_probe_bit_identical(d):
    """The gradient-mode tuner times every launch-option candidate on a short misfit gradient and
    keeps one of them; the options change speed only, so the full gradient under the chosen set
    equals the gradient under the default set bit for bit. A second call hits the cache."""
    from paper_2603_04070_gb300 import autotune
    wl = inputs.ring_phantom(seed=5, n_maps=1)
    pb, geom = _setup(d, wl, ckpt_interval=0)
    sos = torch.from_numpy(wl.sos_start).cuda()
    wav = torch.from_numpy(wl.wavelet).cuda()
    obs = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), wav, geom)
    try:
        autotune.apply(autotune.CANDIDATES[0])
        J0, g0 = d.misfit_gradient(pb, sos, wav, geom, obs)
        best = autotune.tune(pb, sos, wav, geom, gradient=True, cd_obs=obs, steps=120, repeats=1)
        picked = {k: best[k] for k in autotune.KNOBS}
        assert picked in [dict(c) for c in autotune.CANDIDATES]
        # every candidate gives the default gradient bit for bit
        for cand in autotune.CANDIDATES:
            autotune.apply(cand)
            Jc, gc = d.misfit_gradient(pb, sos, wav, geom, obs)
            assert torch.equal(J0, Jc) and torch.equal(g0, gc), cand
        autotune.apply(picked)
        assert len(best["candidates_ms_per_step"]) == len(autotune.CANDIDATES)
        assert all(t is None or t > 0 for t in best["candidates_ms_per_step"])
        assert best["candidates_ms_per_step"][0] > 0
        J1, g1 = d.misfit_gradient(pb, sos, wav, geom, obs)
        torch.cuda.synchronize()
        assert torch.equal(J0, J1)
        assert torch.equal(g0, g1)
        again = autotune.tune(pb, sos, wav, geom, gradient=True, cd_obs=obs)
        assert again == best
    finally:
        autotune.apply(autotune.CANDIDATES[0])
