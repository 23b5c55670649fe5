"""Convolutional PML (the alternative absorbing layer) on the GPU against the oracle.

Same tolerances as the other paths: traces rel-L2 <= 1e-5, gradient rel-L2 <= 1e-4, misfit
relative error <= 1e-4. Checkpointed gradients snapshot the forward memory variables with the
fields at each segment start and keep the adjoint's memory variables apart."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2603_04070_gb300 import inputs

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-5
GRAD_TOL = 1e-4
C_MAX = 2000.0


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


def _case(seed, nx, nz, nt, n_elem, n_tx, n_maps=1, order=8, density=False):
    wl = inputs.make_workload("linear_disk", seed=seed, nx=nx, nz=nz, nt=nt, n_elem=n_elem, n_tx=n_tx,
                              n_maps=n_maps, fd_order=order)
    r2 = inputs.rng_for(seed + 900)
    wl.sos_true = np.stack([inputs.grf_rods_map(r2, nx, nz, wl.dx) for _ in range(n_maps)])
    rho = None
    if density:
        rng = inputs.rng_for(seed + 500)
        rho = np.stack([inputs.density_map(rng, nx, nz, wl.dx) for _ in range(n_maps)])
    return wl, rho


ALPHA = math.pi * 2e6


def _op(wl):
    return oracle.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml=wl.pml, pml_R=wl.pml_R,
                          pml_cref=wl.pml_cref, fd_order=wl.fd_order, boundary=1, pml_alpha=ALPHA)


def _pb(d, wl, **kw):
    return d.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml_cells=wl.pml, pml_R=wl.pml_R,
                     pml_cref=wl.pml_cref, fd_order=wl.fd_order, c_max=C_MAX, boundary="cpml", pml_alpha=ALPHA, **kw)


def _oracle_traces(wl, C, rho):
    p = _op(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    return np.stack([oracle.forward(p, np.asarray(C, np.float64), (tix[k], tiz[k]), wl.wavelet.astype(np.float64),
                                    rix[k], riz[k], rho=rho) for k in range(wl.n_tx)])


def _t(a):
    return None if a is None else torch.from_numpy(a).cuda()


@pytest.mark.parametrize("order,density", [(8, False), (8, True), (4, False), (2, True)])
def test_cpml_simulate_matches_oracle(d, order, density):
    wl, rho = _case(order + 3 * density, 97, 71, 500, 24, 3, order=order, density=density)
    geom = d.Geometry.from_workload(wl)
    cd = d.simulate(_pb(d, wl), _t(wl.sos_true), _t(wl.wavelet), geom, density=_t(rho), check=True).cpu().numpy()
    ref = _oracle_traces(wl, wl.sos_true[0], None if rho is None else rho[0])
    assert rel_l2(cd[0], ref) <= TRACE_TOL


@pytest.mark.parametrize("density", [False, True])
def test_cpml_gradient_matches_oracle(d, density):
    wl, rho = _case(21, 72, 60, 600, 20, 2, n_maps=2, density=density)
    obs = np.stack([_oracle_traces(wl, wl.sos_true[b], None if rho is None else rho[b])
                    for b in range(2)]).astype(np.float32)
    geom = d.Geometry.from_workload(wl)
    pb = _pb(d, wl)
    J, g, cd = d.misfit_gradient(pb, _t(wl.sos_start), _t(wl.wavelet), geom, _t(obs), density=_t(rho),
                                 return_cd=True, check=True)
    J2 = d.misfit(pb, _t(wl.sos_start), _t(wl.wavelet), geom, _t(obs), density=_t(rho), check=True)
    torch.cuda.synchronize()
    assert torch.equal(J, J2)
    p = _op(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    for b in range(2):
        Jr, gr, Mr = oracle.misfit_gradient(p, wl.sos_start[b].astype(np.float64), tix, tiz,
                                            wl.wavelet.astype(np.float64), rix, riz, obs[b].astype(np.float64),
                                            return_traces=True, rho=None if rho is None else rho[b])
        assert np.linalg.norm(Mr - obs[b]) >= 0.03 * np.linalg.norm(Mr)
        assert rel_l2(cd[b].cpu().numpy(), Mr) <= TRACE_TOL
        assert abs(float(J[b]) - Jr) <= 1e-4 * Jr
        assert rel_l2(g[b].cpu().numpy(), gr) <= GRAD_TOL


def test_cpml_backward_equals_misfit_gradient(d):
    """dufwi_backward with the cotangent 2 (M - M_obs) gives the gradient of the misfit call."""
    wl, _ = _case(22, 64, 56, 300, 16, 2)
    geom = d.Geometry.from_workload(wl)
    pb = _pb(d, wl)
    obs = d.simulate(pb, _t(wl.sos_true), _t(wl.wavelet), geom)
    J, g = d.misfit_gradient(pb, _t(wl.sos_start), _t(wl.wavelet), geom, obs, check=True)
    cd, ws = d.forward_save(pb, _t(wl.sos_start), _t(wl.wavelet), geom)
    g2 = d.backward(pb, _t(wl.sos_start), _t(wl.wavelet), geom, (2.0 * (cd - obs)).contiguous(), ws)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)


def test_cpml_absorbs_better_than_the_damping_layer(d):
    """Border return against a domain three times as large, both layers 20 cells thick."""
    c, dx, dt, f0, nt = 1540.0, 1e-4, 1e-8, 2e6, 700
    w = _t(inputs.ricker(nt, dt, f0))
    refl = {}
    for boundary in ("damping", "cpml"):
        tr = []
        for n, src, rec in ((60, 30, 52), (180, 90, 112)):
            pb = d.Problem(nx=n, nz=n, dx=dx, dt=dt, nt=nt, pml_cells=20, pml_cref=c, c_max=C_MAX, boundary=boundary,
                           pml_alpha=math.pi * f0)
            geom = d.Geometry(np.array([src, rec], np.int32), np.array([src, src], np.int32), np.array([0], np.int32),
                              np.array([[1]], np.int32))
            cd = d.simulate(pb, torch.full((1, n, n), c, device="cuda"), w, geom, check=True)
            tr.append(cd[0, 0, :, 0].cpu().numpy().astype(np.float64))
        refl[boundary] = np.max(np.abs(tr[0] - tr[1])) / np.max(np.abs(tr[1]))
    assert refl["cpml"] < 2e-3 and refl["cpml"] < 0.1 * refl["damping"], refl


@pytest.mark.parametrize("ckpt,kept,density", [(1, 0, False), (7, 0, True), (64, 0, False), (25, 3, True)])
def test_cpml_checkpointed_gradient_is_bit_identical_to_store_all(d, ckpt, kept, density):
    """Snapshots of (U^t, U^{t-1}) and of the four forward memory fields read at step t restore
    the exact forward state, and the adjoint's memory variables live in sets of their own, so the
    checkpointed gradient (with or without kept segments) equals the store-all one bit for bit."""
    wl, rho = _case(24, 64, 56, 300, 16, 2, n_maps=2, density=density)
    geom = d.Geometry.from_workload(wl)
    sos, w = _t(wl.sos_start), _t(wl.wavelet)
    obs = d.simulate(_pb(d, wl), _t(wl.sos_true), w, geom, density=_t(rho))
    J0, g0 = d.misfit_gradient(_pb(d, wl), sos, w, geom, obs, density=_t(rho), check=True)
    J1, g1 = d.misfit_gradient(_pb(d, wl, ckpt_interval=ckpt, kept_segments=kept), sos, w, geom, obs,
                               density=_t(rho), check=True)
    assert torch.equal(J0, J1) and torch.equal(g0, g1)
    cd, ws = d.forward_save(_pb(d, wl, ckpt_interval=ckpt), sos, w, geom, density=_t(rho))
    g2 = d.backward(_pb(d, wl, ckpt_interval=ckpt), sos, w, geom, (2.0 * (cd - obs)).contiguous(), ws,
                    density=_t(rho))
    assert torch.equal(g0, g2)


def test_cpml_checkpointed_gradient_matches_oracle(d):
    """Checkpoints every 50 steps on the CPML, against the oracle's gradient."""
    wl, _ = _case(25, 80, 70, 700, 20, 2)
    obs = _oracle_traces(wl, wl.sos_true[0], None)[None].astype(np.float32)
    geom = d.Geometry.from_workload(wl)
    J, g = d.misfit_gradient(_pb(d, wl, ckpt_interval=50), _t(wl.sos_start), _t(wl.wavelet), geom, _t(obs),
                             check=True)
    p = _op(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    Jr, gr = oracle.misfit_gradient(p, wl.sos_start[0].astype(np.float64), tix, tiz, wl.wavelet.astype(np.float64),
                                    rix, riz, obs[0].astype(np.float64), ckpt=50)[:2]
    assert abs(float(J[0]) - Jr) <= 1e-4 * Jr
    assert rel_l2(g[0].cpu().numpy(), gr) <= GRAD_TOL


def test_cpml_unsupported_combinations(d):
    wl, _ = _case(23, 40, 40, 60, 8, 1)
    geom = d.Geometry.from_workload(wl)
    sos, w = _t(wl.sos_true), _t(wl.wavelet)
    with pytest.raises(d.DufwiError) as e:                      # maps of different sizes
        d.simulate(_pb(d, wl), sos, w, geom, sizes=[(40, 40)])
    assert e.value.status == d.ERR_UNSUPPORTED


# ------------------------------------------------------------------------ second-order products
SO_TOL = 1e-3     # FP32 second-order sums against an FP64 central difference (h = 0.05 m/s)


def _so_case(seed, density):
    # 124 x 60 keeps tiles that run the staggered kernel (x0 = 64, z0 = 32) beside the layer tiles
    wl, rho = _case(seed, 124, 60, 300, 20, 2, density=density)
    v = np.random.default_rng(seed).standard_normal(wl.sos_start.shape) * 5.0
    return wl, (None if rho is None else rho[0]), v


def _grad_o(wl, C, M_obs, rho):
    p = _op(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    return oracle.misfit_gradient(p, np.asarray(C, np.float64), tix, tiz, wl.wavelet.astype(np.float64), rix, riz,
                                  np.asarray(M_obs, np.float64), rho=rho)[1]


@pytest.mark.parametrize("ckpt,density", [(0, False), (40, False), (40, True)])
def test_cpml_second_order_matches_oracle_differences(d, ckpt, density):
    """dufwi_second_order with the CPML: the second-order term against the central difference of
    the oracle's vector-Jacobian product with the CPML, the Born data against central differences
    of the oracle traces, and the VJP against the oracle."""
    wl, rho, v = _so_case(90, density)
    C = wl.sos_start[0].astype(np.float64)
    M_obs = _oracle_traces(wl, wl.sos_true[0], rho)
    w = 2.0 * (_oracle_traces(wl, C, rho) - M_obs)
    h = 0.05

    def vjp(Cx):
        return _grad_o(wl, Cx, _oracle_traces(wl, Cx, rho) - 0.5 * w, rho)

    ref = (vjp(C + h * v[0]) - vjp(C - h * v[0])) / (2 * h)
    pb = _pb(d, wl, ckpt_interval=ckpt)
    geom = d.Geometry.from_workload(wl)
    r = None if rho is None else _t(rho[None].astype(np.float32))
    so, dcd, g = d.second_order(pb, _t(wl.sos_start), _t(wl.wavelet), geom, _t(w[None].astype(np.float32)),
                                _t(v.astype(np.float32)), return_grad=True, check=True, density=r)
    torch.cuda.synchronize()
    assert rel_l2(so.cpu().numpy()[0], ref) <= SO_TOL
    assert rel_l2(g.cpu().numpy()[0], vjp(C)) <= GRAD_TOL
    jv_ref = (_oracle_traces(wl, C + h * v[0], rho) - _oracle_traces(wl, C - h * v[0], rho)) / (2 * h)
    assert rel_l2(dcd.cpu().numpy()[0], jv_ref) <= 1e-4


def test_cpml_exact_hvp_matches_oracle_and_is_symmetric(d):
    """dufwi_hvp with the CPML against the central difference of the oracle gradient (M_obs fixed),
    its misfit and gradient against dufwi_misfit_gradient, <u, H v> = <v, H u>, and the checkpointed
    form (memory variables of U and dU snapshotted with the fields) against keeping every step."""
    wl, rho, v = _so_case(91, False)
    C = wl.sos_start[0].astype(np.float64)
    M_obs = _oracle_traces(wl, wl.sos_true[0], rho)
    h = 0.05
    ref = (_grad_o(wl, C + h * v[0], M_obs, rho) - _grad_o(wl, C - h * v[0], M_obs, rho)) / (2 * h)
    geom = d.Geometry.from_workload(wl)
    sos, wav, obs, vv = _t(wl.sos_start), _t(wl.wavelet), _t(M_obs[None].astype(np.float32)), _t(v.astype(np.float32))
    pb = _pb(d, wl, ckpt_interval=35)
    hv, J, g = d.hvp(pb, sos, wav, geom, obs, vv, return_all=True, check=True)
    hv0 = d.hvp(_pb(d, wl), sos, wav, geom, obs, vv, check=True)
    J1, g1 = d.misfit_gradient(pb, sos, wav, geom, obs)
    torch.cuda.synchronize()
    assert rel_l2(hv.cpu().numpy()[0], ref) <= SO_TOL
    assert torch.equal(hv, hv0)
    assert torch.equal(J, J1)
    assert rel_l2(g.cpu().numpy(), g1.cpu().numpy()) <= 1e-6
    u = _t(np.random.default_rng(92).standard_normal(wl.sos_start.shape).astype(np.float32) * 5.0)
    hu = d.hvp(pb, sos, wav, geom, obs, u)
    a = float((u.double() * hv.double()).sum())
    b = float((vv.double() * hu.double()).sum())
    assert abs(a - b) <= 1e-4 * max(abs(a), abs(b))


@pytest.mark.parametrize("density", [False, True])
def test_cpml_born_jvp_matches_oracle_differences(d, density):
    """dufwi_jvp with the CPML (the Born field with its own memory variables, through the CPML
    kernel's Born kind on the layer tiles) against central differences of the oracle traces, and
    its background data against the oracle; the JVP and the VJP are transposes."""
    wl, rho, v = _so_case(93, density)
    C = wl.sos_true[0].astype(np.float64)
    h = 0.05
    ref = (_oracle_traces(wl, C + h * v[0], rho) - _oracle_traces(wl, C - h * v[0], rho)) / (2 * h)
    pb = _pb(d, wl)
    geom = d.Geometry.from_workload(wl)
    r = None if rho is None else _t(rho[None].astype(np.float32))
    sos, wav, vv = _t(wl.sos_true), _t(wl.wavelet), _t(v.astype(np.float32))
    dcd, cd = d.jvp(pb, sos, wav, geom, vv, density=r, return_cd=True, check=True)
    torch.cuda.synchronize()
    assert rel_l2(dcd.cpu().numpy()[0], ref) <= 1e-4
    assert rel_l2(cd.cpu().numpy()[0], _oracle_traces(wl, C, rho)) <= TRACE_TOL
    q = torch.randn(dcd.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(4)) * 1e-9
    _, ws = d.forward_save(pb, sos, wav, geom, density=r)
    JTq = d.backward(pb, sos, wav, geom, q, ws, density=r)
    lhs = float((dcd.double() * q.double()).sum())
    rhs = float((vv.double() * JTq.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
