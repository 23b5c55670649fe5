"""Second-order products on the GPU (``dufwi_second_order`` and the autograd double backward)
against central differences of the FP64 oracle's first-order products, which the oracle pins
pin in turn (finite-difference gradients, adjoint dot-product test)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_04070_gb300 import inputs

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4
SO_TOL = 1e-3     # FP32 second-order sums against an FP64 central difference (h = 0.05 m/s)


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


def _traces(wl, C):
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    return np.stack([oracle.forward(p, np.asarray(C, np.float64), (tix[k], tiz[k]), wl.wavelet.astype(np.float64),
                                    rix[k], riz[k]) for k in range(wl.n_tx)])


def _grad(wl, C, M_obs):
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    return oracle.misfit_gradient(p, np.asarray(C, np.float64), tix, tiz, wl.wavelet.astype(np.float64), rix, riz,
                                  np.asarray(M_obs, np.float64))[1]


def _vjp(wl, C, w):
    """(dM/dC)^T w of one map: the oracle misfit gradient with M_obs = M(C) - w/2."""
    return _grad(wl, C, _traces(wl, C) - 0.5 * w)


def _case(seed, nx=56, nz=50, nt=300, n_tx=2, order=8):
    wl = inputs.make_workload("full_shot_set", seed=seed, nx=nx, nz=nz, nt=nt, n_elem=14, n_tx=n_tx,
                              fd_order=order)
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(wl.sos_start.shape) * 5.0
    return wl, v


def _problem(d, wl, **kw):
    return d.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml_cells=wl.pml, pml_R=wl.pml_R,
                     pml_cref=wl.pml_cref, fd_order=wl.fd_order, c_max=wl.c_max, **kw)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("ckpt,order", [(0, 8), (37, 8), (0, 4)])
def test_second_order_matches_oracle_differences(d, ckpt, order):
    """so = d/dC[(dM/dC)^T w] . v for the residual cotangent w = 2 (M(C) - M_obs), against the
    central difference of the oracle's (dM/dC)^T w along v with w held fixed; the returned
    first-order products against the oracle too."""
    wl, v = _case(40 + order, order=order)
    C = wl.sos_start[0].astype(np.float64)
    M_obs = _traces(wl, wl.sos_true[0])
    w = 2.0 * (_traces(wl, C) - M_obs)
    h = 0.05
    ref = (_vjp(wl, C + h * v[0], w) - _vjp(wl, C - h * v[0], w)) / (2 * h)
    pb = _problem(d, wl, ckpt_interval=ckpt)
    geom = d.Geometry.from_workload(wl)
    so, dcd, g = d.second_order(pb, _cuda(wl.sos_start), _cuda(wl.wavelet), geom, _cuda(w[None]), _cuda(v),
                                return_grad=True, check=True)
    torch.cuda.synchronize()
    assert rel_l2(so.cpu().numpy()[0], ref) <= SO_TOL
    assert rel_l2(g.cpu().numpy()[0], _vjp(wl, C, w)) <= GRAD_TOL
    jv_ref = (_traces(wl, C + h * v[0]) - _traces(wl, C - h * v[0])) / (2 * h)
    assert rel_l2(dcd.cpu().numpy()[0], jv_ref) <= 1e-4


def test_second_order_first_order_outputs_agree_with_jvp_and_backward(d):
    """The Born data and the vector-Jacobian product returned by the second-order call are the
    ones of dufwi_jvp and dufwi_backward (same tile arithmetic, to FP32 rounding), on two maps."""
    wl = inputs.make_workload("linear_disk", seed=9, nx=70, nz=54, nt=240, n_elem=16, n_tx=2, n_maps=2)
    rng = np.random.default_rng(9)
    v = _cuda(rng.standard_normal(wl.sos_true.shape) * 4.0)
    w = _cuda(rng.standard_normal((2, wl.n_tx, wl.nt, wl.n_rx)) * 1e-9)
    pb = _problem(d, wl, ckpt_interval=50)
    geom = d.Geometry.from_workload(wl)
    sos, wav = _cuda(wl.sos_true), _cuda(wl.wavelet)
    so, dcd, g = d.second_order(pb, sos, wav, geom, w, v, return_grad=True, check=True)
    jv = d.jvp(pb, sos, wav, geom, v)
    _, ws = d.forward_save(pb, sos, wav, geom)
    g1 = d.backward(pb, sos, wav, geom, w, ws)
    torch.cuda.synchronize()
    assert rel_l2(dcd.cpu().numpy(), jv.cpu().numpy()) <= 1e-6
    assert rel_l2(g.cpu().numpy(), g1.cpu().numpy()) <= 1e-6
    assert float(so.abs().max()) > 0


def test_second_order_checkpointed_is_bit_identical_to_store_all(d):
    """Recomputing each segment's two histories from FP32 snapshots reproduces them exactly."""
    wl, v = _case(50, nt=260)
    rng = np.random.default_rng(50)
    w = _cuda(rng.standard_normal((1, wl.n_tx, wl.nt, wl.n_rx)) * 1e-9)
    geom = d.Geometry.from_workload(wl)
    sos, wav, vv = _cuda(wl.sos_start), _cuda(wl.wavelet), _cuda(v)
    out = []
    for ckpt in (0, 25, 100):
        so, dcd, g = d.second_order(_problem(d, wl, ckpt_interval=ckpt), sos, wav, geom, w, vv, return_grad=True,
                                    check=True)
        torch.cuda.synchronize()
        out.append((so.cpu(), dcd.cpu(), g.cpu()))
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert torch.equal(a, b)


def test_exact_hvp_by_double_backward_matches_oracle(d):
    """H v of the misfit at a nonzero residual (start map against data of the true map), through
    torch.autograd.grad twice, against the central difference of the oracle gradient with M_obs
    held fixed. The Gauss-Newton product alone misses the residual term by far more than the
    tolerance."""
    from paper_2603_04070_gb300 import autograd
    wl, v = _case(60)
    C = wl.sos_start[0].astype(np.float64)
    M_obs = _traces(wl, wl.sos_true[0])
    h = 0.05
    ref = (_grad(wl, C + h * v[0], M_obs) - _grad(wl, C - h * v[0], M_obs)) / (2 * h)
    pb = _problem(d, wl, ckpt_interval=40)
    geom = d.Geometry.from_workload(wl)
    sos, wav, obs, vv = _cuda(wl.sos_start), _cuda(wl.wavelet), _cuda(M_obs[None]), _cuda(v)
    Hv = autograd.hvp(pb, sos, wav, geom, obs, vv)
    gn = autograd.hvp_gauss_newton(pb, sos, wav, geom, vv)
    torch.cuda.synchronize()
    assert rel_l2(Hv.cpu().numpy()[0], ref) <= SO_TOL
    assert rel_l2(gn.cpu().numpy()[0], ref) > 10 * SO_TOL


def test_exact_hvp_is_symmetric(d):
    """<u, H v> = <v, H u> for the exact Hessian (two maps, each its own product)."""
    from paper_2603_04070_gb300 import autograd
    wl = inputs.make_workload("linear_disk", seed=61, nx=60, nz=52, nt=280, n_elem=14, n_tx=2, n_maps=2)
    rng = np.random.default_rng(61)
    u = _cuda(rng.standard_normal(wl.sos_true.shape) * 5.0)
    v = _cuda(rng.standard_normal(wl.sos_true.shape) * 5.0)
    pb = _problem(d, wl)
    geom = d.Geometry.from_workload(wl)
    sos, wav = _cuda(wl.sos_start), _cuda(wl.wavelet)
    obs = d.simulate(pb, _cuda(wl.sos_true), wav, geom)
    Hv = autograd.hvp(pb, sos, wav, geom, obs, v).double()
    Hu = autograd.hvp(pb, sos, wav, geom, obs, u).double()
    a = (u.double() * Hv).flatten(1).sum(1)
    b = (v.double() * Hu).flatten(1).sum(1)
    assert torch.all((a - b).abs() <= 1e-4 * torch.maximum(a.abs(), b.abs()))


def test_second_order_rejects_third_derivatives(d):
    from paper_2603_04070_gb300 import autograd
    wl, v = _case(62, nt=120)
    pb = _problem(d, wl)
    geom = d.Geometry.from_workload(wl)
    sos, wav = _cuda(wl.sos_start), _cuda(wl.wavelet)
    c = sos.clone().requires_grad_(True)
    J = autograd.misfit(pb, c, wav, geom, d.simulate(pb, _cuda(wl.sos_true), wav, geom)).sum()
    (g,) = torch.autograd.grad(J, c, create_graph=True)
    with pytest.raises(RuntimeError, match="third derivatives"):
        torch.autograd.grad(g, c, grad_outputs=_cuda(v), create_graph=True)


@pytest.mark.parametrize("ckpt", [0, 40])
def test_fused_hvp_matches_double_backward_and_oracle(d, ckpt):
    """dufwi_hvp (the adjoint of 2 J v carried by dmu's receiver source) against the double
    backward of the autograd wrapper (separate sweeps) and the oracle's central differences; its
    misfit and gradient against dufwi_misfit_gradient."""
    from paper_2603_04070_gb300 import autograd
    wl, v = _case(63)
    C = wl.sos_start[0].astype(np.float64)
    M_obs = _traces(wl, wl.sos_true[0])
    h = 0.05
    ref = (_grad(wl, C + h * v[0], M_obs) - _grad(wl, C - h * v[0], M_obs)) / (2 * h)
    pb = _problem(d, wl, ckpt_interval=ckpt)
    geom = d.Geometry.from_workload(wl)
    sos, wav, obs, vv = _cuda(wl.sos_start), _cuda(wl.wavelet), _cuda(M_obs[None]), _cuda(v)
    hv, J, g = d.hvp(pb, sos, wav, geom, obs, vv, return_all=True, check=True)
    Hv2 = autograd.hvp(pb, sos, wav, geom, obs, vv)
    J1, g1 = d.misfit_gradient(pb, sos, wav, geom, obs)
    torch.cuda.synchronize()
    assert rel_l2(hv.cpu().numpy()[0], ref) <= SO_TOL
    assert rel_l2(hv.cpu().numpy(), Hv2.cpu().numpy()) <= 1e-5
    assert torch.equal(J, J1)
    assert rel_l2(g.cpu().numpy(), g1.cpu().numpy()) <= 1e-6


def test_newton_cg_fwi_with_exact_hvp(d):
    """Truncated Newton (CG on dufwi_hvp products) lowers the misfit monotonically, by more than an
    order of magnitude in its first iteration on this case (the FP64 oracle with differenced
    Hessian products gives 20x), and further than L-BFGS after the same number of iterations."""
    from paper_2603_04070_gb300 import fwi
    wl, _ = _case(64)
    pb = _problem(d, wl)
    geom = d.Geometry.from_workload(wl)
    wav = _cuda(wl.wavelet)
    obs = d.simulate(pb, _cuda(wl.sos_true), wav, geom)
    ev = fwi.cuda_evaluator(pb, wav, geom, obs)
    hv = fwi.cuda_hessvec(pb, wav, geom, obs)
    c0 = _cuda(wl.sos_start)
    res = fwi.newton_cg(ev, hv, c0, 3, cg_iters=4)
    J = torch.stack(res.misfits)[:, 0]
    assert torch.all(J[1:] < J[:-1])
    assert float(J[1]) < 0.1 * float(J[0])
    lb = fwi.lbfgs(ev, c0, 3)
    assert float(J[-1]) < float(torch.stack(lb.misfits)[-1, 0])


def test_exact_hvp_full_shot_set_properties(d):
    """Full shot set (512 x 512 + 20, 16 transmits x 128 receivers, 6000 steps, checkpoint
    interval 100), where the oracle would take minutes per product: properties that hold at any
    size. The Hessian is symmetric; dufwi_hvp agrees with the composed form (dufwi_second_order
    plus the VJP of 2 J v); its misfit equals dufwi_misfit_gradient's and its gradient agrees."""
    wl = inputs.make_workload("full_shot_set", seed=0)
    pb = _problem(d, wl, ckpt_interval=100)
    geom = d.Geometry.from_workload(wl)
    sos, wav = _cuda(wl.sos_start), _cuda(wl.wavelet)
    obs = d.simulate(pb, _cuda(wl.sos_true), wav, geom)
    rng = np.random.default_rng(0)
    v = _cuda(rng.standard_normal(wl.sos_start.shape) * 5.0)
    u = _cuda(rng.standard_normal(wl.sos_start.shape) * 5.0)
    ws = torch.empty(d.second_order_workspace_size(pb, geom, 1), dtype=torch.uint8, device="cuda")
    Hv, J, g = d.hvp(pb, sos, wav, geom, obs, v, return_all=True, workspace=ws, check=True)
    Hv, J, g = Hv.clone(), J.clone(), g.clone()
    Hu = d.hvp(pb, sos, wav, geom, obs, u, workspace=ws, check=True).clone()
    a, b = float((u.double() * Hv.double()).sum()), float((v.double() * Hu.double()).sum())
    assert abs(a - b) <= 1e-4 * max(abs(a), abs(b))
    J1, g1 = d.misfit_gradient(pb, sos, wav, geom, obs)
    cd = d.simulate(pb, sos, wav, geom)
    so, dcd = d.second_order(pb, sos, wav, geom, 2.0 * (cd - obs), v, workspace=ws, check=True)
    _, wsg = d.forward_save(pb, sos, wav, geom)
    gn = d.backward(pb, sos, wav, geom, 2.0 * dcd, wsg)
    torch.cuda.synchronize()
    assert torch.equal(J, J1)
    assert rel_l2(g.cpu().numpy(), g1.cpu().numpy()) <= 1e-6
    assert rel_l2(Hv.cpu().numpy(), (so + gn).cpu().numpy()) <= 1e-5


def test_differentiable_data_gradient_applies_exact_hessian(d):
    """Backpropagating through g = dJ/dC (the unfolded loop's data gradient) applies the exact
    Hessian: equal to dufwi_hvp and to the double backward of the autograd wrapper."""
    from paper_2603_04070_gb300 import autograd, unfolded
    wl = inputs.make_workload("linear_disk", seed=80, nx=56, nz=48, nt=260, n_elem=14, n_tx=2, n_maps=3)
    pb = _problem(d, wl, ckpt_interval=50)
    geom = d.Geometry.from_workload(wl)
    wav = _cuda(wl.wavelet)
    phys = unfolded.Physics(pb, wav, geom)
    obs = d.simulate(pb, _cuda(wl.sos_true), wav, geom)
    c = _cuda(wl.sos_start).requires_grad_(True)
    v = _cuda(np.random.default_rng(80).standard_normal(wl.sos_start.shape) * 3e-18)   # gradient-sized cotangent
    g = unfolded.data_gradient_differentiable(phys, c, obs, chunk=2)
    (Hv,) = torch.autograd.grad(g, c, grad_outputs=v)
    s = v.abs().amax(dim=(-2, -1), keepdim=True)
    ref = d.hvp(pb, c.detach(), wav, geom, obs, (v / s).contiguous()) * s
    Hv2 = autograd.hvp(pb, c.detach(), wav, geom, obs, (v / s).contiguous()) * s
    torch.cuda.synchronize()
    assert rel_l2(Hv.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    assert rel_l2(Hv.cpu().numpy(), Hv2.cpu().numpy()) <= 1e-5


def test_unfolded_end_to_end_gradient_matches_loss_differences(d):
    """End-to-end gradient of the SoS MSE of C_K for K = 2 unfolded iterations, through both
    nets and both data gradients (exact Hessian-vector products): its projection on its own
    direction d equals the central difference of the loss along d, computed by running the loop
    forward (physics included) at theta +- h d, closer than the truncated gradient that treats
    the data gradients as constants (the Hessian term is a few percent here). The nets run in
    FP64 with deterministic cuDNN algorithms: TF32 or FP32 rounding, and run-to-run differences
    in the nets' training, would put noise of up to ~1e-3 on the loss. Training then lowers the
    loss."""
    from paper_2603_04070_gb300 import unfolded
    torch.manual_seed(0)
    wl = inputs.make_workload("linear_disk", seed=81, nx=48, nz=48, nt=260, n_elem=14, n_tx=3, n_maps=4)
    pb = _problem(d, wl, ckpt_interval=50)
    geom = d.Geometry.from_workload(wl)
    phys = unfolded.Physics(pb, _cuda(wl.wavelet), geom)
    gt = _cuda(wl.sos_true)
    obs = d.simulate(pb, gt, phys.wavelet, geom)
    c0 = _cuda(wl.sos_start)
    flags = (torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32,
             torch.backends.cudnn.deterministic, torch.backends.cudnn.benchmark)
    torch.backends.cudnn.allow_tf32 = False
    torch.backends.cuda.matmul.allow_tf32 = False
    torch.backends.cudnn.deterministic = True
    torch.backends.cudnn.benchmark = False
    try:
        model = unfolded.UnfoldedFWI(K=2).cuda().double()
        model.train_blockwise(phys, c0, obs, gt, epochs=20, batch=4, lrs=(3e-3, 1e-3))
        params = list(model.parameters())

        def loss_value():
            with torch.no_grad():
                return float(((model.infer(phys, c0, obs)[-1] - gt) ** 2).double().mean())

        def loss_graph(exact):
            c = c0
            for net in model.nets:
                g = unfolded.data_gradient_differentiable(phys, c, obs) if exact else \
                    unfolded.data_gradient(phys, c.detach(), obs)[1]
                c = c + net(c, g)
            return ((c - gt) ** 2).mean()

        loss = loss_graph(True)
        grads = torch.autograd.grad(loss, params)
        gnorm = float(torch.sqrt(sum((g.double() ** 2).sum() for g in grads)))
        dirs = [g / gnorm for g in grads]
        grads_t = torch.autograd.grad(loss_graph(False), params)
        proj_t = float(sum((a.double() * b.double()).sum() for a, b in zip(grads_t, dirs)))
        h = 1e-3 * float(loss.detach()) / gnorm
        with torch.no_grad():
            for p_, d_ in zip(params, dirs):
                p_.add_(h * d_)
        Lp = loss_value()
        with torch.no_grad():
            for p_, d_ in zip(params, dirs):
                p_.sub_(2 * h * d_)
        Lm = loss_value()
        with torch.no_grad():
            for p_, d_ in zip(params, dirs):
                p_.add_(h * d_)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gnorm) <= 5e-3 * gnorm
        assert abs(fd - gnorm) < abs(fd - proj_t)
        losses = model.train_end_to_end(phys, c0, obs, gt, epochs=8, batch=4, lr=1e-4)
        assert all(np.isfinite(losses))
        assert losses[-1] < losses[0]
    finally:
        (torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32,
         torch.backends.cudnn.deterministic, torch.backends.cudnn.benchmark) = flags


# ------------------------------------------------------------------------------ density maps
def _density_case(seed, nt=280):
    wl, v = _case(seed, nt=nt)
    rho = inputs.density_map(inputs.rng_for(seed + 300), wl.nx, wl.nz, wl.dx)
    return wl, v, rho


def _traces_rho(wl, C, rho):
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    return np.stack([oracle.forward(p, np.asarray(C, np.float64), (tix[k], tiz[k]), wl.wavelet.astype(np.float64),
                                    rix[k], riz[k], rho=rho) for k in range(wl.n_tx)])


def _grad_rho(wl, C, M_obs, rho):
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    return oracle.misfit_gradient(p, np.asarray(C, np.float64), tix, tiz, wl.wavelet.astype(np.float64), rix, riz,
                                  np.asarray(M_obs, np.float64), rho=rho)[1]


@pytest.mark.parametrize("ckpt", [0, 40])
def test_second_order_with_density_matches_oracle_differences(d, ckpt):
    """With a density map (the staggered operator of Eq. 1 in all three fields): the second-order
    term against the central difference of the oracle's vector-Jacobian product with density, and
    the Born data and the VJP against the oracle."""
    wl, v, rho = _density_case(70)
    C = wl.sos_start[0].astype(np.float64)
    M_obs = _traces_rho(wl, wl.sos_true[0], rho)
    w = 2.0 * (_traces_rho(wl, C, rho) - M_obs)
    h = 0.05

    def vjp(Cx):
        return _grad_rho(wl, Cx, _traces_rho(wl, Cx, rho) - 0.5 * w, rho)

    ref = (vjp(C + h * v[0]) - vjp(C - h * v[0])) / (2 * h)
    pb = _problem(d, wl, ckpt_interval=ckpt)
    pb.c_max = 2000.0
    geom = d.Geometry.from_workload(wl)
    so, dcd, g = d.second_order(pb, _cuda(wl.sos_start), _cuda(wl.wavelet), geom, _cuda(w[None]), _cuda(v),
                                return_grad=True, check=True, density=_cuda(rho[None]))
    torch.cuda.synchronize()
    assert rel_l2(so.cpu().numpy()[0], ref) <= SO_TOL
    assert rel_l2(g.cpu().numpy()[0], vjp(C)) <= GRAD_TOL
    jv_ref = (_traces_rho(wl, C + h * v[0], rho) - _traces_rho(wl, C - h * v[0], rho)) / (2 * h)
    assert rel_l2(dcd.cpu().numpy()[0], jv_ref) <= 1e-4


def test_exact_hvp_with_density_matches_oracle_and_is_symmetric(d):
    """dufwi_hvp with a density map against the central difference of the oracle gradient with
    density (M_obs fixed), its misfit and gradient against dufwi_misfit_gradient with the same map,
    and <u, H v> = <v, H u>."""
    wl, v, rho = _density_case(71)
    C = wl.sos_start[0].astype(np.float64)
    M_obs = _traces_rho(wl, wl.sos_true[0], rho)
    h = 0.05
    ref = (_grad_rho(wl, C + h * v[0], M_obs, rho) - _grad_rho(wl, C - h * v[0], M_obs, rho)) / (2 * h)
    pb = _problem(d, wl, ckpt_interval=35)
    pb.c_max = 2000.0
    geom = d.Geometry.from_workload(wl)
    sos, wav, obs, r = _cuda(wl.sos_start), _cuda(wl.wavelet), _cuda(M_obs[None]), _cuda(rho[None])
    hv, J, g = d.hvp(pb, sos, wav, geom, obs, _cuda(v), return_all=True, check=True, density=r)
    J1, g1 = d.misfit_gradient(pb, sos, wav, geom, obs, density=r)
    torch.cuda.synchronize()
    assert rel_l2(hv.cpu().numpy()[0], ref) <= SO_TOL
    assert torch.equal(J, J1)
    assert rel_l2(g.cpu().numpy(), g1.cpu().numpy()) <= 1e-6
    u = _cuda(np.random.default_rng(72).standard_normal(wl.sos_start.shape) * 5.0)
    hu = d.hvp(pb, sos, wav, geom, obs, u, density=r)
    a = float((u.double() * hv.double()).sum())
    b = float((_cuda(v).double() * hu.double()).sum())
    assert abs(a - b) <= 1e-4 * max(abs(a), abs(b))


@pytest.mark.parametrize("with_density", [False, True])
def test_second_order_calls_are_bit_identical_across_shot_groups(d, with_density):
    """The Born JVP, the second-order call and dufwi_hvp step their rings per shot group on
    concurrent streams; 1, 2 and 4 groups (4 shots here) give the same results bit for bit."""
    wl, v = _case(73, nt=200, n_tx=4)
    pb = _problem(d, wl, ckpt_interval=45)
    pb.c_max = 2000.0
    geom = d.Geometry.from_workload(wl)
    sos, wav, vv = _cuda(wl.sos_start), _cuda(wl.wavelet), _cuda(v)
    rho = _cuda(inputs.density_map(inputs.rng_for(75), wl.nx, wl.nz, wl.dx)[None]) if with_density else None
    obs = d.simulate(pb, _cuda(wl.sos_true), wav, geom, density=rho)
    w = torch.randn(obs.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(5)) * 1e-6
    before = d.get_option(d.OPT_SHOT_GROUPS)
    outs = []
    try:
        for groups in (1, 2, 4):
            d.set_option(d.OPT_SHOT_GROUPS, groups)
            dcd, cd = d.jvp(pb, sos, wav, geom, vv, density=rho, return_cd=True)
            so, dcd2, g = d.second_order(pb, sos, wav, geom, w, vv, return_grad=True, check=True, density=rho)
            hv, J, g2 = d.hvp(pb, sos, wav, geom, obs, vv, return_all=True, check=True, density=rho)
            torch.cuda.synchronize()
            outs.append((dcd, cd, so, dcd2, g, hv, J, g2))
    finally:
        d.set_option(d.OPT_SHOT_GROUPS, before)
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert torch.equal(a, b)
    assert float(outs[0][2].abs().max()) > 0.0 and float(outs[0][5].abs().max()) > 0.0
