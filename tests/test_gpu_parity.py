"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on identical seeded inputs.

Tolerances (FP32 stencil arithmetic against the FP64 oracle):
  traces    rel-L2 <= 1e-5
  gradient  rel-L2 <= 1e-4
  misfit    relative error <= 1e-4
Compressed checkpoint snapshots (BF16 or FP16) leave the traces and the misfit untouched,
since both come from the uncompressed first sweep. Their gradient errors are measured and
bounded separately.
"""
import functools

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


def _dufwi_problem(d, wl, **kw):
    return d.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml_cells=wl.pml, pml_R=wl.pml_R,
                     pml_cref=wl.pml_cref, fd_order=wl.fd_order, c_max=wl.c_max, **kw)


def _oracle_traces(wl, C, tx=None):
    """Oracle channel data [n_tx][nt][n_rx] of one map."""
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    txs = range(wl.n_tx) if tx is None else tx
    return np.stack([oracle.forward(p, np.asarray(C, np.float64), (tix[k], tiz[k]),
                                    wl.wavelet.astype(np.float64), rix[k], riz[k]) for k in txs])


def _observed(wl):
    """Observed data of the true maps, from the oracle, rounded to FP32 (both sides see these)."""
    return np.stack([_oracle_traces(wl, wl.sos_true[b]) for b in range(wl.n_maps)]).astype(np.float32)


def _oracle_grad(wl, C, M_obs, ckpt=0):
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    return oracle.misfit_gradient(p, np.asarray(C, np.float64), tix, tiz, wl.wavelet.astype(np.float64), rix, riz,
                                  M_obs.astype(np.float64), ckpt=ckpt, return_traces=True)


def _gpu_grad(d, wl, M_obs, **kw):
    pb = _dufwi_problem(d, wl, **kw)
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_start).cuda()
    w = torch.from_numpy(wl.wavelet).cuda()
    obs = torch.from_numpy(M_obs).cuda()
    J, g, cd = d.misfit_gradient(pb, sos, w, geom, obs, return_cd=True, check=True)
    torch.cuda.synchronize()
    return J.cpu().numpy(), g.cpu().numpy(), cd.cpu().numpy()


# ----------------------------------------------------------------------------- forward
@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_simulate_matches_oracle_ragged_grid(d, order):
    """Ragged grids: several tiles and a partial last tile in both axes, pitch padding in x."""
    wl = inputs.make_workload("linear_disk", seed=order, nx=97, nz=71, nt=500, n_elem=24, n_tx=3)
    geom = d.Geometry.from_workload(wl)
    wl.fd_order = order
    pb = _dufwi_problem(d, wl)
    cd = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda(), geom,
                    check=True).cpu().numpy()
    ref = _oracle_traces(wl, wl.sos_true[0])
    assert np.all(cd[0, :, 0, :] == 0.0)
    assert rel_l2(cd[0], ref) <= TRACE_TOL


def test_simulate_linear_disk_full_size(d):
    """128 x 128, 2000 steps, 32 elements, centre transmit (the linear-disk workload)."""
    wl = inputs.make_workload("linear_disk", seed=0)
    geom = d.Geometry.from_workload(wl)
    pb = _dufwi_problem(d, wl)
    cd = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda(), geom,
                    check=True).cpu().numpy()
    assert rel_l2(cd[0], _oracle_traces(wl, wl.sos_true[0])) <= TRACE_TOL


def test_simulate_batched_maps_and_per_tx_wavelets(d):
    wl = inputs.make_workload("linear_disk", seed=3, nx=80, nz=66, nt=400, n_elem=20, n_tx=4, n_maps=3)
    rng = np.random.default_rng(0)
    wav = np.stack([inputs.ricker(wl.nt, wl.dt, 2e6, delay=0.75e-6 + 0.1e-6 * k) for k in range(wl.n_tx)])
    wav *= rng.uniform(0.5, 1.5, size=(wl.n_tx, 1)).astype(np.float32)
    geom = d.Geometry(wl.elem_ix, wl.elem_iz, wl.tx_elem, wl.rx_elem, wavelet_per_tx=True)
    pb = _dufwi_problem(d, wl)
    cd = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wav).cuda(), geom,
                    check=True).cpu().numpy()
    p = _oracle_problem(wl)
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    for b in range(wl.n_maps):
        for k in range(wl.n_tx):
            ref = oracle.forward(p, wl.sos_true[b].astype(np.float64), (tix[k], tiz[k]), wav[k].astype(np.float64),
                                 rix[k], riz[k])
            assert rel_l2(cd[b, k], ref) <= TRACE_TOL


def test_simulate_edge_cases(d):
    """Elements on the grid corners, a transmitter that also receives (listed twice), a
    receive subset that changes per transmit, and the shortest time axes."""
    nx, nz = 40, 33
    elem_ix = np.array([0, nx - 1, 0, nx - 1, 17], np.int32)
    elem_iz = np.array([0, 0, nz - 1, nz - 1, 16], np.int32)
    tx = np.array([4, 0], np.int32)
    rx = np.array([[4, 4, 0, 1], [2, 3, 0, 4]], np.int32)
    rng = np.random.default_rng(1)
    C = (1540.0 + 30.0 * rng.standard_normal((1, nz, nx))).astype(np.float32)
    for nt in (1, 2, 3, 150):
        w = inputs.ricker(nt, 1e-8, 2e6)
        pb = d.Problem(nx=nx, nz=nz, dx=1e-4, dt=1e-8, nt=nt, c_max=1800.0)
        geom = d.Geometry(elem_ix, elem_iz, tx, rx)
        cd = d.simulate(pb, torch.from_numpy(C).cuda(), torch.from_numpy(w).cuda(), geom, check=True).cpu().numpy()
        p = oracle.Problem(nx=nx, nz=nz, dx=1e-4, dt=1e-8, nt=nt, pml=20, pml_cref=1540.0, fd_order=8)
        for k in range(2):
            ref = oracle.forward(p, C[0].astype(np.float64), (elem_ix[tx[k]], elem_iz[tx[k]]), w.astype(np.float64),
                                 elem_ix[rx[k]], elem_iz[rx[k]])
            if nt <= 2:
                # U[0] = 0 and U[1] is the scaled first wavelet sample at the transmitter
                assert np.allclose(cd[0, k], ref, rtol=1e-6, atol=0)
            else:
                assert rel_l2(cd[0, k], ref) <= TRACE_TOL
        assert np.array_equal(cd[0, 0, :, 0], cd[0, 0, :, 1])


def test_simulate_no_receivers(d):
    pb = d.Problem(nx=30, nz=30, dx=1e-4, dt=1e-8, nt=50)
    geom = d.Geometry(np.array([5, 9], np.int32), np.array([0, 0], np.int32), np.array([0]), np.zeros((1, 0), np.int32))
    cd = d.simulate(pb, torch.full((1, 30, 30), 1540.0, device="cuda"),
                    torch.from_numpy(inputs.ricker(50, 1e-8, 2e6)).cuda(), geom, check=True)
    assert cd.shape == (1, 1, 50, 0)
    obs = torch.zeros((1, 1, 50, 0), device="cuda")
    J, g = d.misfit_gradient(d.Problem(nx=30, nz=30, dx=1e-4, dt=1e-8, nt=50, ckpt_interval=7),
                             torch.full((1, 30, 30), 1540.0, device="cuda"),
                             torch.from_numpy(inputs.ricker(50, 1e-8, 2e6)).cuda(), geom, obs, check=True)
    assert float(J[0]) == 0.0 and torch.count_nonzero(g).item() == 0


def test_device_status_word(d):
    """Out-of-range SoS and non-finite observed data are reported through the workspace status
    word (density checks: tests/test_gpu_density.py)."""
    wl = inputs.make_workload("linear_disk", seed=2, nx=40, nz=40, nt=60, n_elem=8)
    geom = d.Geometry.from_workload(wl)
    pb = _dufwi_problem(d, wl)
    w = torch.from_numpy(wl.wavelet).cuda()
    bad = torch.from_numpy(wl.sos_true).cuda().clone()
    bad[0, 5, 5] = 2500.0            # above c_max = 1700
    ws = torch.empty(d.workspace_size(pb, geom, 1, gradient=False), dtype=torch.uint8, device="cuda")
    d.simulate(pb, bad, w, geom, workspace=ws)
    assert d.workspace_status(ws) == d.ERR_CFL
    bad[0, 5, 5] = float("nan")
    d.simulate(pb, bad, w, geom, workspace=ws)
    assert d.workspace_status(ws) == d.ERR_NONFINITE
    good = torch.from_numpy(wl.sos_true).cuda()
    d.simulate(pb, good, w, geom, workspace=ws)
    assert d.workspace_status(ws) == d.OK
    obs = torch.zeros((1, wl.n_tx, wl.nt, wl.n_rx), device="cuda")
    obs[0, 0, 10, 2] = float("inf")
    with pytest.raises(d.DufwiError) as e:
        d.misfit_gradient(pb, good, w, geom, obs, check=True)
    assert e.value.status == d.ERR_NONFINITE


# ----------------------------------------------------------------------------- gradient
def test_gradient_matches_oracle_store_all(d):
    wl = inputs.make_workload("linear_disk", seed=5, nx=72, nz=60, nt=600, n_elem=20, n_tx=2)
    M_obs = _observed(wl)
    J_ref, g_ref, cd_ref = _oracle_grad(wl, wl.sos_start[0], M_obs[0])
    J, g, cd = _gpu_grad(d, wl, M_obs)
    assert rel_l2(cd[0], cd_ref) <= TRACE_TOL
    assert abs(J[0] - J_ref) <= 1e-4 * J_ref
    assert rel_l2(g[0], g_ref) <= GRAD_TOL


@pytest.mark.parametrize("ckpt", [1, 7, 64])
def test_checkpointed_gradient_is_bit_identical_to_store_all(d, ckpt):
    """FP32 snapshots restore the exact fields, and the recompute runs the same kernels, so the
    gradient is bit-identical to the store-all gradient."""
    wl = inputs.make_workload("linear_disk", seed=6, nx=64, nz=64, nt=300, n_elem=16, n_tx=2, n_maps=2)
    M_obs = _observed(wl)
    J0, g0, _ = _gpu_grad(d, wl, M_obs)
    J1, g1, _ = _gpu_grad(d, wl, M_obs, ckpt_interval=ckpt)
    assert np.array_equal(J0, J1) and np.array_equal(g0, g1)


@pytest.mark.parametrize("kept,precision", [(1, "fp32"), (3, "fp32"), (8, "fp32"), (99, "fp32"), (2, "compensated")])
def test_hybrid_history_is_bit_identical_to_store_all(d, kept, precision):
    """The last `kept` checkpoint segments keep their history from the forward sweep; the earlier
    ones are recomputed into the slots the kept ones freed. Every split gives the store-all
    gradient bit for bit (8 segments of 37 steps here; 99 keeps them all)."""
    wl = inputs.make_workload("linear_disk", seed=6, nx=64, nz=64, nt=290, n_elem=16, n_tx=2, n_maps=2)
    M_obs = _observed(wl)
    J0, g0, c0 = _gpu_grad(d, wl, M_obs, forward_precision=precision)
    J1, g1, c1 = _gpu_grad(d, wl, M_obs, ckpt_interval=37, kept_segments=kept, forward_precision=precision)
    assert np.array_equal(J0, J1) and np.array_equal(g0, g1) and np.array_equal(c0, c1)


def test_hybrid_history_with_compressed_snapshots(d):
    """With FP16 snapshots only the recomputed segments carry the snapshot error: keeping every
    segment gives the store-all gradient exactly, keeping some lands between the two."""
    wl = inputs.make_workload("linear_disk", seed=8, nx=80, nz=80, nt=801, n_elem=24, n_tx=2)
    M_obs = _observed(wl)
    _, g_all, _ = _gpu_grad(d, wl, M_obs)
    errs = []
    for kept in (0, 8, 16):
        _, g, _ = _gpu_grad(d, wl, M_obs, ckpt_interval=50, snapshot_dtype="fp16", kept_segments=kept)
        errs.append(rel_l2(g[0], g_all[0]))
    assert errs[2] == 0.0
    assert 0.0 < errs[1] <= errs[0]


@pytest.mark.parametrize("kw", [dict(kept_segments=0), dict(kept_segments=3), dict(snapshot_dtype="fp16"),
                                dict(forward_precision="compensated"), dict(boundary="cpml", pml_alpha=6e6)])
def test_backward_repeats_after_one_forward_save(d, kw):
    """dufwi_backward can run any number of times on one dufwi_forward_save workspace: a reverse
    sweep recomputes earlier segments into the first kept segment's history slots, so each
    backward recomputes that segment from its own snapshot. Repeated products are bit-identical,
    and the misfit cotangent gives dufwi_misfit_gradient's gradient bit for bit."""
    wl = inputs.make_workload("linear_disk", seed=9, nx=64, nz=64, nt=290, n_elem=16, n_tx=2, n_maps=2)
    M_obs = _observed(wl)
    pb = _dufwi_problem(d, wl, ckpt_interval=37, **kw)        # 8 segments
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_start).cuda()
    wav = torch.from_numpy(wl.wavelet).cuda()
    obs = torch.from_numpy(M_obs).cuda()
    cd, ws = d.forward_save(pb, sos, wav, geom)
    q = torch.randn(cd.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(3)) * 1e-9
    w = 2.0 * (cd - obs)
    gq1 = d.backward(pb, sos, wav, geom, q, ws, check=True)
    gw1 = d.backward(pb, sos, wav, geom, w, ws, check=True)
    gq2 = d.backward(pb, sos, wav, geom, q, ws, check=True)
    gw2 = d.backward(pb, sos, wav, geom, w, ws, check=True)
    J, g = d.misfit_gradient(pb, sos, wav, geom, obs)
    torch.cuda.synchronize()
    assert torch.equal(gq1, gq2) and torch.equal(gw1, gw2)
    if kw.get("forward_precision") != "compensated":          # the residual then adds the traces' low parts
        assert torch.equal(gw1, g)
    assert float(gq1.abs().max()) > 0.0


def test_gradient_batched_maps(d):
    wl = inputs.make_workload("linear_disk", seed=7, nx=70, nz=58, nt=500, n_elem=22, n_tx=3, n_maps=2)
    wl.sos_start = (wl.sos_start + np.random.default_rng(1).uniform(-5, 5, wl.sos_start.shape)).astype(np.float32)
    M_obs = _observed(wl)
    J, g, _ = _gpu_grad(d, wl, M_obs, ckpt_interval=50)
    for b in range(wl.n_maps):
        J_ref, g_ref, _ = _oracle_grad(wl, wl.sos_start[b], M_obs[b])
        assert abs(J[b] - J_ref) <= 1e-4 * J_ref
        assert rel_l2(g[b], g_ref) <= GRAD_TOL


def test_fp64_gradient_output(d):
    """dufwi_misfit_gradient_fp64 skips only the final rounding: its gradient rounded to FP32 is the
    FP32 call's gradient bit for bit, its misfit is the same, and it matches the oracle."""
    wl = inputs.make_workload("linear_disk", seed=10, nx=70, nz=58, nt=400, n_elem=18, n_tx=3, n_maps=2)
    M_obs = _observed(wl)
    pb = _dufwi_problem(d, wl, ckpt_interval=40)
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_start).cuda()
    w = torch.from_numpy(wl.wavelet).cuda()
    obs = torch.from_numpy(M_obs).cuda()
    J32, g32 = d.misfit_gradient(pb, sos, w, geom, obs, check=True)
    g64 = torch.empty(sos.shape, dtype=torch.float64, device="cuda")
    J64, g64 = d.misfit_gradient(pb, sos, w, geom, obs, grad=g64, check=True)
    assert g64.dtype == torch.float64
    assert torch.equal(J32, J64)
    assert torch.equal(g64.float(), g32)
    for b in range(wl.n_maps):
        _, g_ref, _ = _oracle_grad(wl, wl.sos_start[b], M_obs[b])
        assert rel_l2(g64[b].cpu().numpy(), g_ref) <= GRAD_TOL


@pytest.mark.parametrize("dtype,tol", [("fp16", 6e-3), ("bf16", 6e-2)])
def test_compressed_snapshots(d, dtype, tol):
    """BF16/FP16 snapshots with per-snapshot power-of-two max-abs scaling: traces and misfit are
    unchanged; the gradient error against the oracle is bounded per dtype."""
    wl = inputs.make_workload("linear_disk", seed=8, nx=80, nz=80, nt=800, n_elem=24, n_tx=2)
    M_obs = _observed(wl)
    J_ref, g_ref, cd_ref = _oracle_grad(wl, wl.sos_start[0], M_obs[0])
    J, g, cd = _gpu_grad(d, wl, M_obs, ckpt_interval=50, snapshot_dtype=dtype)
    assert rel_l2(cd[0], cd_ref) <= TRACE_TOL
    assert abs(J[0] - J_ref) <= 1e-4 * J_ref
    err = rel_l2(g[0], g_ref)
    print("snapshot %s gradient rel-L2 vs oracle: %.3e" % (dtype, err))
    assert err <= tol


@functools.lru_cache(maxsize=1)
def _cropped_scale_case():
    """The cropped 256 x 256 sub-problem of the 1024 x 1024 configuration (central 64 elements,
    8 transmits, 3500 steps) with its oracle observed data and oracle gradient (checkpoints every
    100 steps), computed once for the snapshot-precision cases."""
    wl = inputs.make_workload("scale", seed=0, nx=256, nz=256, nt=3500, n_elem=64, n_tx=8)
    M_obs = _observed(wl)
    return wl, M_obs, _oracle_grad(wl, wl.sos_start[0], M_obs[0], ckpt=100)


@pytest.mark.parametrize("dtype,grad_tol", [("fp32", GRAD_TOL), ("fp16", GRAD_TOL), ("bf16", 1e-3)])
def test_snapshot_precision_at_scale_vs_oracle(d, dtype, grad_tol):
    """The snapshot-precision study against the oracle at a paper-scale size (the cropped case
    above, checkpoints every 100 steps). FP32 and FP16 snapshots stay within the FP32 bounds
    (traces 1e-5, gradient 1e-4); BF16 snapshots, measured at about 2e-4, are held to 1e-3. The
    errors are printed (pytest -s) for the precision summary."""
    wl, M_obs, (J_ref, g_ref, cd_ref) = _cropped_scale_case()
    J, g, cd = _gpu_grad(d, wl, M_obs, ckpt_interval=100, snapshot_dtype=dtype)
    errs = (rel_l2(cd[0], cd_ref), abs(float(J[0]) - J_ref) / J_ref, rel_l2(g[0], g_ref))
    print("snapshots %s at 256x256x8x3500 vs oracle: traces %.3e misfit %.3e gradient %.3e" % ((dtype,) + errs))
    assert errs[0] <= TRACE_TOL
    assert errs[1] <= 1e-4
    assert errs[2] <= grad_tol


def test_zero_residual_gives_zero_gradient(d):
    """Observed data equal to the GPU's own simulation at the start map: J = 0 and g = 0."""
    wl = inputs.make_workload("linear_disk", seed=9, nx=50, nz=50, nt=200, n_elem=12, n_tx=2)
    geom = d.Geometry.from_workload(wl)
    pb = _dufwi_problem(d, wl, ckpt_interval=20)
    sos = torch.from_numpy(wl.sos_start).cuda()
    w = torch.from_numpy(wl.wavelet).cuda()
    obs = d.simulate(pb, sos, w, geom)
    J, g = d.misfit_gradient(pb, sos, w, geom, obs, check=True)
    assert float(J[0]) == 0.0 and torch.count_nonzero(g).item() == 0


def test_gradient_full_shot_set_grid_single_transmit(d):
    """512 x 512, 6000 steps, 128 receivers, checkpoint interval 100: the grid, time axis and
    launch shape of the full shot set, with one transmit so the FP64 oracle finishes."""
    wl = inputs.make_workload("full_shot_set", seed=0, n_tx=1)
    M_obs = _observed(wl)
    J_ref, g_ref, cd_ref = _oracle_grad(wl, wl.sos_start[0], M_obs[0], ckpt=100)
    J, g, cd = _gpu_grad(d, wl, M_obs, ckpt_interval=100)
    assert rel_l2(cd[0], cd_ref) <= TRACE_TOL
    assert abs(J[0] - J_ref) <= 1e-4 * J_ref
    assert rel_l2(g[0], g_ref) <= GRAD_TOL


def test_gradient_full_shot_set_all_transmits(d):
    """The headline launch exactly: 512 x 512, 6000 steps, all 16 transmits and 128 receivers in one
    call, checkpoint interval 100, FP32 snapshots; the FP64 cross-transmit reduction (Eqs. 4-6)
    against the oracle's gradient over the same 16 transmits (about 4 min of host time)."""
    wl = inputs.make_workload("full_shot_set", seed=0)
    assert (wl.n_tx, wl.n_rx, wl.nt) == (16, 128, 6000)
    M_obs = _observed(wl)
    J_ref, g_ref, cd_ref = _oracle_grad(wl, wl.sos_start[0], M_obs[0], ckpt=100)
    J, g, cd = _gpu_grad(d, wl, M_obs, ckpt_interval=100)
    errs = (rel_l2(cd[0], cd_ref), abs(float(J[0]) - J_ref) / J_ref, rel_l2(g[0], g_ref))
    print("full shot set, 16 transmits: traces %.2e misfit %.2e gradient %.2e" % errs)
    assert errs[0] <= TRACE_TOL
    assert errs[1] <= 1e-4
    assert errs[2] <= GRAD_TOL


@pytest.mark.parametrize("precision", ["fp32", "compensated"])
def test_gradient_cell_by_cell_on_a_tiny_grid(d, precision):
    """Every cell of a 14 x 12 gradient against the oracle, not only the field norm: the edge cells
    carry the fold of the 20-cell absorbing layer (and the corners that of two strips), so an error
    confined to the layer or the fold would show there. Bound: max |g - g_ref| <= 1e-4 max |g_ref|,
    over the interior, the edge rows and columns, and the corners separately."""
    wl = inputs.make_workload("linear_disk", seed=21, nx=14, nz=12, nt=260, n_elem=4, n_tx=2)
    wl.sos_start = (wl.sos_start + np.random.default_rng(2).uniform(-20, 20, wl.sos_start.shape)).astype(np.float32)
    M_obs = _observed(wl)
    _, g_ref, _ = _oracle_grad(wl, wl.sos_start[0], M_obs[0])
    _, g, _ = _gpu_grad(d, wl, M_obs, ckpt_interval=31, forward_precision=precision)
    err = np.abs(g[0].astype(np.float64) - g_ref)
    scale = np.abs(g_ref).max()
    edge = np.zeros(g_ref.shape, bool)
    edge[0, :] = edge[-1, :] = edge[:, 0] = edge[:, -1] = True
    corners = np.zeros(g_ref.shape, bool)
    corners[0, 0] = corners[0, -1] = corners[-1, 0] = corners[-1, -1] = True
    for name, mask in (("interior", ~edge), ("edges", edge & ~corners), ("corners", corners)):
        worst = err[mask].max() / scale
        print("%s %s: max cell error / max |g| = %.2e" % (precision, name, worst))
        assert worst <= 1e-4, name


def test_simulate_full_shot_set_sampled_transmits(d):
    """All 16 transmits of the 512 x 512, 6000-step workload in one call (the benchmark's launch
    configuration); two sampled transmits are recomputed by the oracle."""
    wl = inputs.make_workload("full_shot_set", seed=1)
    geom = d.Geometry.from_workload(wl)
    pb = _dufwi_problem(d, wl)
    cd = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda(), geom,
                    check=True).cpu().numpy()
    for k in (0, 11):
        ref = _oracle_traces(wl, wl.sos_true[0], tx=[k])[0]
        assert rel_l2(cd[0, k], ref) <= TRACE_TOL


def test_simulate_scale_config_sampled_transmit(d):
    """The 1024 x 1024, 12000-step, 64-transmit configuration in one call (as the precision
    benchmark runs it); the last transmit is recomputed by the oracle alone (~14 G cell updates
    in FP64). The trace tolerance holds at this length too."""
    wl = inputs.make_workload("scale", seed=0)
    geom = d.Geometry.from_workload(wl)
    pb = _dufwi_problem(d, wl)
    cd = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda(), geom,
                    check=True)
    k = wl.n_tx - 1
    got = cd[0, k].cpu().numpy()
    del cd
    ref = _oracle_traces(wl, wl.sos_true[0], tx=[k])[0]
    assert rel_l2(got, ref) <= TRACE_TOL


@pytest.mark.parametrize("ckpt", [0, 9])
def test_two_step_kernel_is_bit_identical_to_one_step(d, ckpt):
    """Fusing pairs of time steps into one launch changes no result bit: the grown-tile step
    repeats the one-step arithmetic, and injections are applied in list order either way."""
    wl = inputs.make_workload("linear_disk", seed=12, nx=90, nz=77, nt=257, n_elem=20, n_tx=3, n_maps=2)
    M_obs = _observed(wl)
    out = []
    for two in (0, 1):
        d.set_option(d.OPT_TWO_STEP, two)
        try:
            pb = _dufwi_problem(d, wl, ckpt_interval=ckpt)
            geom = d.Geometry.from_workload(wl)
            cd = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda(), geom,
                            check=True).cpu().numpy()
            J, g, cds = _gpu_grad(d, wl, M_obs, ckpt_interval=ckpt)
            out.append((cd, J, g, cds))
        finally:
            d.set_option(d.OPT_TWO_STEP, 0)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("ckpt,order,nx,nz,n_tx,n_maps", [(0, 8, 90, 77, 3, 2), (9, 8, 150, 61, 2, 1),
                                                          (25, 4, 33, 20, 1, 1), (7, 6, 300, 260, 4, 2)])
def test_multi_tile_kernel_is_bit_identical_to_one_step(d, ckpt, order, nx, nz, n_tx, n_maps):
    """The multi-tile form (co-resident CTAs walking the tiles with two-stage TMA loads) runs the
    per-tile arithmetic of the one-tile-per-CTA form with 32-row tiles: traces, misfit and
    gradient are identical bit for bit, for grids smaller and larger than one wave of CTAs, and
    for the Born step."""
    wl = inputs.make_workload("linear_disk", seed=13 + order, nx=nx, nz=nz, nt=180, n_elem=min(20, nx // 4),
                              n_tx=n_tx, n_maps=n_maps)
    wl.fd_order = order
    M_obs = _observed(wl)
    geom = d.Geometry.from_workload(wl)
    out = []
    for mt in (0, 1):
        d.set_option(d.OPT_MULTI_TILE, mt)
        try:
            pb = _dufwi_problem(d, wl, ckpt_interval=ckpt)
            sos = torch.from_numpy(wl.sos_true).cuda()
            w = torch.from_numpy(wl.wavelet).cuda()
            cd = d.simulate(pb, sos, w, geom, check=True).cpu().numpy()
            J, g, cds = _gpu_grad(d, wl, M_obs, ckpt_interval=ckpt)
            dsos = torch.from_numpy(np.random.default_rng(order).standard_normal(wl.sos_true.shape)
                                    .astype(np.float32)).cuda()
            jv = d.jvp(pb, sos, w, geom, dsos).cpu().numpy()
            out.append((cd, J, g, cds, jv))
        finally:
            d.set_option(d.OPT_MULTI_TILE, 0)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_multi_tile_kernel_sized_batch_is_bit_identical(d):
    """Uneven grids in one call: tiles outside a map's grid are skipped inside the tile walk."""
    wl, sizes = inputs.sized_batch(seed=4, sizes=[(96, 80), (64, 48), (130, 70)], nt=160, n_elem=16, n_tx=2)
    geom = d.Geometry.from_workload(wl)
    out = []
    for mt in (0, 1):
        d.set_option(d.OPT_MULTI_TILE, mt)
        try:
            pb = _dufwi_problem(d, wl, ckpt_interval=30)
            sos = torch.from_numpy(wl.sos_true).cuda()
            w = torch.from_numpy(wl.wavelet).cuda()
            cd = d.simulate(pb, sos, w, geom, check=True, sizes=sizes)
            J, g = d.misfit_gradient(pb, torch.from_numpy(wl.sos_start).cuda(), w, geom, cd * 1.01, check=True,
                                     sizes=sizes)
            out.append((cd.cpu().numpy(), J.cpu().numpy(), g.cpu().numpy()))
        finally:
            d.set_option(d.OPT_MULTI_TILE, 0)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("ckpt,order,nx,nz,n_tx,n_maps", [(0, 8, 90, 77, 3, 2), (40, 8, 150, 61, 2, 1),
                                                          (25, 4, 33, 20, 1, 1)])
def test_persistent_sweeps_are_bit_identical(d, ckpt, order, nx, nz, n_tx, n_maps):
    """One cooperative launch per sweep segment (tiles handed from step to step through per-tile
    counters) gives exactly the results of one launch per step: same tile arithmetic, same
    injection order. Cases: store-all, checkpointed with an odd segment count, and a grid of
    fewer tiles than resident CTAs."""
    wl = inputs.make_workload("linear_disk", seed=13, nx=nx, nz=nz, nt=257, n_elem=min(20, nx // 4), n_tx=n_tx,
                              n_maps=n_maps, fd_order=order)
    M_obs = _observed(wl)
    out = []
    for persistent in (0, 1):
        d.set_option(d.OPT_PERSISTENT, persistent)
        try:
            pb = _dufwi_problem(d, wl, ckpt_interval=ckpt)
            geom = d.Geometry.from_workload(wl)
            cd = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda(), geom,
                            check=True).cpu().numpy()
            J, g, cds = _gpu_grad(d, wl, M_obs, ckpt_interval=ckpt)
            out.append((cd, J, g, cds))
        finally:
            d.set_option(d.OPT_PERSISTENT, 0)
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_persistent_sweeps_sized_batch_bit_identical(d):
    sizes = [(96, 70), (64, 96), (80, 80)]
    wl, sizes = inputs.sized_batch(8, sizes, nt=200, n_elem=16, n_tx=2)
    M = []
    for persistent in (0, 1):
        d.set_option(d.OPT_PERSISTENT, persistent)
        try:
            pb = _dufwi_problem(d, wl, ckpt_interval=30)
            geom = d.Geometry.from_workload(wl)
            sos = torch.from_numpy(wl.sos_true).cuda()
            cd = d.simulate(pb, sos, torch.from_numpy(wl.wavelet).cuda(), geom, sizes=sizes, check=True)
            J, g = d.misfit_gradient(pb, torch.from_numpy(wl.sos_start).cuda(), torch.from_numpy(wl.wavelet).cuda(),
                                     geom, cd, sizes=sizes, check=True)
            M.append((cd.cpu().numpy(), J.cpu().numpy(), g.cpu().numpy()))
        finally:
            d.set_option(d.OPT_PERSISTENT, 0)
    for a, b in zip(M[0], M[1]):
        assert np.array_equal(a, b)


def test_persistent_wait_timeout_reports_status_and_device_stays_usable(d):
    """The bounded inter-CTA wait of the persistent sweep: the test hook makes one tile wait on a
    counter that nothing sets. The launch gives up after its 2 s limit with DUFWI_ERR_TIMEOUT in
    the status word, and the next call on the same device and workspace runs normally."""
    import time
    wl = inputs.make_workload("linear_disk", seed=3, nx=60, nz=50, nt=40, n_elem=8)
    geom = d.Geometry.from_workload(wl)
    pb = _dufwi_problem(d, wl)
    sos = torch.from_numpy(wl.sos_true).cuda()
    w = torch.from_numpy(wl.wavelet).cuda()
    ws = torch.empty(d.workspace_size(pb, geom, 1, gradient=False), dtype=torch.uint8, device="cuda")
    ref = d.simulate(pb, sos, w, geom, workspace=ws, check=True).clone()
    d.set_option(d.OPT_PERSISTENT, 1)
    try:
        d.set_option(d.OPT_TEST_STALL, 1)
        t0 = time.time()
        d.simulate(pb, sos, w, geom, workspace=ws)
        status = d.workspace_status(ws)
        waited = time.time() - t0
        assert status == d.ERR_TIMEOUT
        assert 1.5 < waited < 30.0
        assert d.get_option(d.OPT_TEST_STALL) == 0          # the hook clears itself
        again = d.simulate(pb, sos, w, geom, workspace=ws, check=True)
        torch.cuda.synchronize()
        assert torch.equal(again, ref)
    finally:
        d.set_option(d.OPT_TEST_STALL, 0)
        d.set_option(d.OPT_PERSISTENT, 0)


def test_autograd_matches_misfit_gradient_bit_for_bit(d):
    """loss = sum (M - M_obs)^2 through the autograd wrapper gives the misfit gradient exactly:
    the cotangent 2 (M - M_obs) enters the same adjoint kernels."""
    from paper_2603_04070_gb300 import autograd
    wl = inputs.make_workload("linear_disk", seed=14, nx=70, nz=62, nt=300, n_elem=18, n_tx=2, n_maps=2)
    M_obs = torch.from_numpy(_observed(wl)).cuda()
    pb = _dufwi_problem(d, wl, ckpt_interval=40)
    geom = d.Geometry.from_workload(wl)
    w = torch.from_numpy(wl.wavelet).cuda()
    sos = torch.from_numpy(wl.sos_start).cuda().requires_grad_(True)
    cd = autograd.simulate(pb, sos, w, geom)
    loss = ((cd - M_obs) ** 2).sum()
    loss.backward()
    J, g = d.misfit_gradient(pb, sos.detach(), w, geom, M_obs)
    assert torch.equal(sos.grad, g)
    assert abs(float(loss.detach()) - float(J.sum())) <= 1e-5 * float(J.sum())


def test_autograd_vjp_matches_oracle_for_random_cotangent(d):
    """A random linear functional of the traces: (dM/dC)^T q against the oracle, which computes
    the same product as the misfit gradient with M_obs = M_sim - q/2."""
    from paper_2603_04070_gb300 import autograd
    wl = inputs.make_workload("linear_disk", seed=15, nx=64, nz=60, nt=350, n_elem=16, n_tx=2)
    rng = np.random.default_rng(0)
    q = rng.standard_normal((1, wl.n_tx, wl.nt, wl.n_rx)).astype(np.float32) * 1e-9
    pb = _dufwi_problem(d, wl)
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_true).cuda().requires_grad_(True)
    cd = autograd.simulate(pb, sos, torch.from_numpy(wl.wavelet).cuda(), geom)
    (cd * torch.from_numpy(q).cuda()).sum().backward()
    sim = _oracle_traces(wl, wl.sos_true[0])
    J_ref, g_ref, _ = _oracle_grad(wl, wl.sos_true[0], sim - 0.5 * q[0].astype(np.float64))
    assert rel_l2(sos.grad.cpu().numpy()[0], g_ref) <= GRAD_TOL


def test_sized_batch_matches_oracle_per_map(d):
    """Maps of three different grids in one call (one launch per step for all shots): traces and
    gradient of each map against the oracle run on that map's own grid."""
    sizes = [(40, 36), (57, 49), (72, 64)]
    wl, sizes = inputs.sized_batch(seed=21, sizes=sizes, nt=350, n_elem=12, n_tx=2)
    geom = d.Geometry.from_workload(wl)
    pb = _dufwi_problem(d, wl, ckpt_interval=30)
    w = torch.from_numpy(wl.wavelet).cuda()
    tix, tiz = wl.tx_nodes()
    rix, riz = wl.rx_nodes()
    # observed data per map from the oracle on its own grid
    obs = np.zeros((len(sizes), wl.n_tx, wl.nt, wl.n_rx), np.float32)
    refs = []
    for b, (nx, nz) in enumerate(sizes):
        p = oracle.Problem(nx=nx, nz=nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml=wl.pml, pml_R=wl.pml_R,
                           pml_cref=wl.pml_cref, fd_order=wl.fd_order)
        for k in range(wl.n_tx):
            obs[b, k] = oracle.forward(p, wl.sos_true[b, :nz, :nx].astype(np.float64), (tix[k], tiz[k]),
                                       wl.wavelet.astype(np.float64), rix[k], riz[k])
        refs.append((p, oracle.misfit_gradient(p, wl.sos_start[b, :nz, :nx].astype(np.float64), tix, tiz,
                                               wl.wavelet.astype(np.float64), rix, riz, obs[b].astype(np.float64),
                                               return_traces=True)))
    cd = d.simulate(pb, torch.from_numpy(wl.sos_true).cuda(), w, geom, sizes=sizes, check=True).cpu().numpy()
    J, g, cds = d.misfit_gradient(pb, torch.from_numpy(wl.sos_start).cuda(), w, geom, torch.from_numpy(obs).cuda(),
                                  sizes=sizes, return_cd=True, check=True)
    J, g, cds = J.cpu().numpy(), g.cpu().numpy(), cds.cpu().numpy()
    for b, (nx, nz) in enumerate(sizes):
        _, (J_ref, g_ref, cd_ref) = refs[b]
        assert rel_l2(cd[b], obs[b]) <= TRACE_TOL
        assert rel_l2(cds[b], cd_ref) <= TRACE_TOL
        assert abs(J[b] - J_ref) <= 1e-4 * J_ref
        assert rel_l2(g[b, :nz, :nx], g_ref) <= GRAD_TOL
        assert np.all(g[b, nz:, :] == 0) and np.all(g[b, :, nx:] == 0)


def test_sized_call_with_full_sizes_equals_uniform_call(d):
    wl = inputs.make_workload("linear_disk", seed=22, nx=66, nz=58, nt=200, n_elem=16, n_tx=2, n_maps=2)
    pb = _dufwi_problem(d, wl, ckpt_interval=25)
    geom = d.Geometry.from_workload(wl)
    w = torch.from_numpy(wl.wavelet).cuda()
    sos = torch.from_numpy(wl.sos_true).cuda()
    a = d.simulate(pb, sos, w, geom)
    b = d.simulate(pb, sos, w, geom, sizes=[(wl.nx, wl.nz)] * 2)
    assert torch.equal(a, b)
    obs = a * 1.01
    Ja, ga = d.misfit_gradient(pb, torch.from_numpy(wl.sos_start).cuda(), w, geom, obs)
    Jb, gb = d.misfit_gradient(pb, torch.from_numpy(wl.sos_start).cuda(), w, geom, obs, sizes=[(wl.nx, wl.nz)] * 2)
    assert torch.equal(Ja, Jb) and torch.equal(ga, gb)


def test_gradient_call_captures_in_a_cuda_graph(d):
    """After one ordinary call on a workspace, a repeat call issues only device work and can be
    captured; replaying the graph reproduces the direct result bit for bit."""
    wl = inputs.make_workload("linear_disk", seed=23, nx=60, nz=52, nt=180, n_elem=14, n_tx=2)
    pb = _dufwi_problem(d, wl, ckpt_interval=20)
    geom = d.Geometry.from_workload(wl)
    w = torch.from_numpy(wl.wavelet).cuda()
    sos = torch.from_numpy(wl.sos_start).cuda()
    obs = torch.from_numpy(_observed(wl)).cuda()
    ws = torch.empty(d.workspace_size(pb, geom, 1), dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(sos)
    s = torch.cuda.Stream()
    try:
        with torch.cuda.stream(s):
            d.misfit_gradient(pb, sos, w, geom, obs, misfit=J, grad=g, workspace=ws)   # uploads the tables
            s.synchronize()
            J0, g0 = J.clone(), g.clone()
            d.set_option(d.OPT_REUSE_TABLES, 1)   # ws stays reserved: repeat calls may skip the copies
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=s):
                d.misfit_gradient(pb, sos, w, geom, obs, misfit=J, grad=g, workspace=ws)
        J.zero_(); g.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(J, J0) and torch.equal(g, g0)
    finally:
        d.set_option(d.OPT_REUSE_TABLES, 0)
        del ws


@pytest.mark.parametrize("kw", [dict(ckpt_interval=37), dict(ckpt_interval=37, kept_segments=3),
                                dict(ckpt_interval=37, snapshot_dtype="fp16"), dict(forward_precision="compensated"),
                                dict(boundary="cpml", pml_alpha=6e6, ckpt_interval=37), dict(density=True),
                                dict(tile_z=64)])
def test_shot_groups_are_bit_identical(d, kw):
    """Shot groups stepped on concurrent streams (DUFWI_OPT_SHOT_GROUPS 1..4, with 2 maps x 3
    transmits: groups of 3, 2 and 1-2 shots) give the traces, misfit and gradient of one group bit
    for bit, with checkpoints, the hybrid history, FP16 snapshots, the compensated steps, the
    CPML, a density map and 64-row tiles."""
    kw = dict(kw)
    density = kw.pop("density", False)
    tile_z = kw.pop("tile_z", 32)
    wl = inputs.make_workload("linear_disk", seed=12, nx=70, nz=66, nt=260, n_elem=16, n_tx=3, n_maps=2)
    M_obs = _observed(wl)
    pb = _dufwi_problem(d, wl, **kw)
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_start).cuda()
    sos[1] += 7.0
    wav = torch.from_numpy(wl.wavelet).cuda()
    obs = torch.from_numpy(M_obs).cuda()
    rho = None
    if density:
        rho = torch.from_numpy(np.stack([inputs.density_map(inputs.rng_for(40 + b), wl.nx, wl.nz, wl.dx)
                                         for b in range(2)]).astype(np.float32)).cuda()
    g_before, t_before = d.get_option(d.OPT_SHOT_GROUPS), d.get_option(d.OPT_TILE_Z)
    out = []
    try:
        d.set_option(d.OPT_TILE_Z, tile_z)
        for groups in (1, 2, 3, 4):
            d.set_option(d.OPT_SHOT_GROUPS, groups)
            cd = d.simulate(pb, sos, wav, geom, density=rho, check=True)
            J, g, cd2 = d.misfit_gradient(pb, sos, wav, geom, obs, density=rho, return_cd=True, check=True)
            torch.cuda.synchronize()
            out.append((cd, J, g, cd2))
    finally:
        d.set_option(d.OPT_SHOT_GROUPS, g_before)
        d.set_option(d.OPT_TILE_Z, t_before)
    for o in out[1:]:
        for a, b in zip(out[0], o):
            assert torch.equal(a, b)
    assert float(out[0][2].abs().max()) > 0.0


@pytest.mark.parametrize("nx,nz,order,kw", [(64, 56, 8, dict()), (64, 56, 8, dict(ckpt_interval=37)),
                                          (64, 56, 8, dict(ckpt_interval=37, kept_segments=3)),
                                          (97, 71, 8, dict(ckpt_interval=40)), (60, 52, 4, dict()),
                                          (128, 128, 8, dict(ckpt_interval=50)), (188, 188, 8, dict())])
def test_cluster_sweeps_are_bit_identical(d, nx, nz, order, kw):
    """DUFWI_OPT_CLUSTER: whole ranges of steps in one launch of a cluster of 8 CTAs per shot (the
    fields in shared memory, halos through distributed shared memory) give the traces, misfit and
    gradient of one launch per step bit for bit: store-all, checkpointed, the hybrid history, a
    ragged grid (97 x 71: padded width not a multiple of 4, a partial strip and an empty CTA),
    order 4, the 128 x 128 configuration and the paper's 188 x 188 grid."""
    wl = inputs.make_workload("linear_disk", seed=14, nx=nx, nz=nz, nt=230, n_elem=16, n_tx=3, n_maps=2,
                              fd_order=order)
    M_obs = _observed(wl)
    pb = _dufwi_problem(d, wl, **kw)
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_start).cuda()
    sos[1] += 9.0
    wav = torch.from_numpy(wl.wavelet).cuda()
    obs = torch.from_numpy(M_obs).cuda()
    before = d.get_option(d.OPT_CLUSTER)
    out = []
    try:
        for cl in (0, 1):
            d.set_option(d.OPT_CLUSTER, cl)
            cd = d.simulate(pb, sos, wav, geom, check=True)
            J, g, cd2 = d.misfit_gradient(pb, sos, wav, geom, obs, return_cd=True, check=True)
            torch.cuda.synchronize()
            out.append((cd, J, g, cd2))
    finally:
        d.set_option(d.OPT_CLUSTER, before)
    for a, b in zip(*out):
        assert torch.equal(a, b)
    assert float(out[0][2].abs().max()) > 0.0


def test_cluster_option_falls_back_on_large_grids(d):
    """A grid whose fields do not fit a cluster's shared memory runs one launch per step with the
    option set (same results)."""
    wl = inputs.make_workload("linear_disk", seed=15, nx=300, nz=280, nt=60, n_elem=16, n_tx=1)
    pb = _dufwi_problem(d, wl)
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_true).cuda()
    wav = torch.from_numpy(wl.wavelet).cuda()
    before = d.get_option(d.OPT_CLUSTER)
    try:
        d.set_option(d.OPT_CLUSTER, 0)
        a = d.simulate(pb, sos, wav, geom)
        d.set_option(d.OPT_CLUSTER, 1)
        b = d.simulate(pb, sos, wav, geom, check=True)
        torch.cuda.synchronize()
    finally:
        d.set_option(d.OPT_CLUSTER, before)
    assert torch.equal(a, b)


def test_capture_before_any_grouped_call_runs_one_group(d):
    """On a host thread that has made no uncaptured call yet, the group streams are not created
    during stream capture: the captured call runs its shots as one group and replays the result
    of an ordinary (grouped) call bit for bit."""
    import threading
    wl = inputs.make_workload("linear_disk", seed=24, nx=60, nz=52, nt=150, n_elem=14, n_tx=4)
    pb = _dufwi_problem(d, wl, ckpt_interval=30)
    geom = d.Geometry.from_workload(wl)
    w = torch.from_numpy(wl.wavelet).cuda()
    sos = torch.from_numpy(wl.sos_start).cuda()
    obs = torch.from_numpy(_observed(wl)).cuda()
    J0, g0 = d.misfit_gradient(pb, sos, w, geom, obs)
    torch.cuda.synchronize()
    ws = torch.empty(d.workspace_size(pb, geom, 1), dtype=torch.uint8, device="cuda")
    J = torch.empty(1, dtype=torch.float64, device="cuda")
    g = torch.empty_like(sos)
    box = {}

    def worker():
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=s):
                    d.misfit_gradient(pb, sos, w, geom, obs, misfit=J, grad=g, workspace=ws)
            box["graph"] = graph
        except Exception as e:          # reported on the main thread
            box["error"] = e

    try:
        d.set_option(d.OPT_REUSE_TABLES, 0)
        # the tables are copied from pageable host memory inside the capture: allowed for a graph
        # only when they are already in place, so upload them first with an ordinary call
        d.misfit_gradient(pb, sos, w, geom, obs, misfit=J, grad=g, workspace=ws)
        torch.cuda.synchronize()
        d.set_option(d.OPT_REUSE_TABLES, 1)
        t = threading.Thread(target=worker)
        t.start()
        t.join()
        assert "error" not in box, box.get("error")
        J.zero_(); g.zero_()
        box["graph"].replay()
        torch.cuda.synchronize()
        assert torch.equal(J, J0) and torch.equal(g, g0)
    finally:
        d.set_option(d.OPT_REUSE_TABLES, 0)
        del ws


def _born_case(seed, nt=320):
    wl = inputs.make_workload("linear_disk", seed=seed, nx=58, nz=52, nt=nt, n_elem=14, n_tx=2)
    rng = np.random.default_rng(seed)
    v = (rng.standard_normal(wl.sos_start.shape) * 5.0).astype(np.float32)
    return wl, v


def test_born_jvp_matches_oracle_finite_differences(d):
    """dM = (dM/dC) v against central differences of the FP64 oracle forward model."""
    wl, v = _born_case(31)
    C = wl.sos_true[0].astype(np.float64)
    h = 0.05
    ref = (_oracle_traces(wl, C + h * v[0]) - _oracle_traces(wl, C - h * v[0])) / (2 * h)
    pb = _dufwi_problem(d, wl)
    geom = d.Geometry.from_workload(wl)
    dcd, cd = d.jvp(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda(), geom,
                    torch.from_numpy(v).cuda(), return_cd=True, check=True)
    assert rel_l2(cd.cpu().numpy()[0], _oracle_traces(wl, C)) <= TRACE_TOL
    assert rel_l2(dcd.cpu().numpy()[0], ref) <= 1e-4


def test_born_jvp_and_adjoint_are_transposes(d):
    """<J w, q> = <w, J^T q> between the Born simulation and the adjoint (dot-product test)."""
    wl, w = _born_case(32)
    pb = _dufwi_problem(d, wl, ckpt_interval=40)
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_true).cuda()
    wav = torch.from_numpy(wl.wavelet).cuda()
    q = torch.randn((1, wl.n_tx, wl.nt, wl.n_rx), device="cuda") * 1e-9
    Jw = d.jvp(pb, sos, wav, geom, torch.from_numpy(w).cuda())
    _, ws = d.forward_save(pb, sos, wav, geom)
    JTq = d.backward(pb, sos, wav, geom, q, ws)
    lhs = float((Jw.double() * q.double()).sum())
    rhs = float((torch.from_numpy(w).cuda().double() * JTq.double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_gauss_newton_hvp_matches_oracle(d):
    """H v = 2 J^T J v: oracle J v by central differences, oracle J^T through its misfit gradient
    with M_obs = M - J v."""
    from paper_2603_04070_gb300 import autograd
    wl, v = _born_case(33)
    C = wl.sos_true[0].astype(np.float64)
    h = 0.05
    Jv = (_oracle_traces(wl, C + h * v[0]) - _oracle_traces(wl, C - h * v[0])) / (2 * h)
    M = _oracle_traces(wl, C)
    _, Hv_ref, _ = _oracle_grad(wl, C, M - Jv)
    pb = _dufwi_problem(d, wl, ckpt_interval=32)
    geom = d.Geometry.from_workload(wl)
    Hv = autograd.hvp_gauss_newton(pb, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda(),
                                   geom, torch.from_numpy(v).cuda())
    assert rel_l2(Hv.cpu().numpy()[0], Hv_ref) <= 1e-3


def test_autograd_forward_mode_uses_born(d):
    from paper_2603_04070_gb300 import autograd
    import torch.autograd.forward_ad as fwAD
    wl, v = _born_case(34, nt=200)
    pb = _dufwi_problem(d, wl)
    geom = d.Geometry.from_workload(wl)
    sos = torch.from_numpy(wl.sos_true).cuda()
    wav = torch.from_numpy(wl.wavelet).cuda()
    tv = torch.from_numpy(v).cuda()
    with fwAD.dual_level():
        out = autograd.simulate(pb, fwAD.make_dual(sos, tv), wav, geom)
        tangent = fwAD.unpack_dual(out).tangent
    assert torch.equal(tangent, d.jvp(pb, sos, wav, geom, tv))


@pytest.mark.parametrize("ckpt", [25, 50, 100])
def test_gradient_and_hvp_finite_differences_64x64(d, ckpt):
    """64 x 64 grid (random field plus rods, residual 4-8% of the traces), checkpoint interval
    swept: the GPU gradient against the FD-pinned oracle gradient, and the Gauss-Newton HVP at
    zero residual (where it equals the full Hessian) against central differences of the oracle
    gradient."""
    from paper_2603_04070_gb300 import autograd
    wl = inputs.make_workload("full_shot_set", seed=ckpt, nx=64, nz=64, nt=400, n_elem=16, n_tx=2)
    C = wl.sos_true[0].astype(np.float64)
    pb = _dufwi_problem(d, wl, ckpt_interval=ckpt)
    geom = d.Geometry.from_workload(wl)
    w = torch.from_numpy(wl.wavelet).cuda()
    # gradient at the homogeneous start against data of the true map
    M_obs = _observed(wl)
    J_ref, g_ref, _ = _oracle_grad(wl, wl.sos_start[0], M_obs[0], ckpt=ckpt)
    J, g = d.misfit_gradient(pb, torch.from_numpy(wl.sos_start).cuda(), w, geom, torch.from_numpy(M_obs).cuda())
    assert rel_l2(g.cpu().numpy()[0], g_ref) <= GRAD_TOL
    # Hessian-vector product at zero residual (M_obs = M(C))
    rng = np.random.default_rng(ckpt)
    v = rng.standard_normal(C.shape) * 5.0
    M0 = _oracle_traces(wl, C)
    h = 0.05
    _, gp, _ = _oracle_grad(wl, C + h * v, M0)
    _, gm, _ = _oracle_grad(wl, C - h * v, M0)
    Hv_fd = (gp - gm) / (2 * h)
    Hv = autograd.hvp_gauss_newton(pb, torch.from_numpy(wl.sos_true).cuda(), w, geom,
                                   torch.from_numpy(v[None].astype(np.float32)).cuda())
    assert rel_l2(Hv.cpu().numpy()[0], Hv_fd) <= 1e-3


def test_unfolded_loop_block_training_reduces_sos_error(d):
    """Two unfolded iterations with block-wise training on a handful of small synthetic maps: the
    trained updates lower the SoS-map MSE below that of the homogeneous start."""
    from paper_2603_04070_gb300 import unfolded
    torch.manual_seed(0)
    wl = inputs.make_workload("linear_disk", seed=50, nx=48, nz=48, nt=260, n_elem=14, n_tx=3, n_maps=6)
    pb = _dufwi_problem(d, wl, ckpt_interval=50)
    geom = d.Geometry.from_workload(wl)
    phys = unfolded.Physics(pb, torch.from_numpy(wl.wavelet).cuda(), geom)
    gt = torch.from_numpy(wl.sos_true).cuda()
    obs = d.simulate(pb, gt, phys.wavelet, geom)
    c0 = torch.from_numpy(wl.sos_start).cuda()
    model = unfolded.UnfoldedFWI(K=2).cuda()
    hist = model.train_blockwise(phys, c0, obs, gt, epochs=60, batch=6, lrs=(3e-3, 1e-3))
    outs = model.infer(phys, c0, obs)
    mse0 = float(((c0 - gt) ** 2).mean())
    mse2 = float(((outs[-1] - gt) ** 2).mean())
    assert hist[0][-1] < hist[0][0]
    assert mse2 < mse0


def test_gradient_weak_scatterer_meets_the_bound(d):
    """A weak scatterer leaves a residual below 1 % of the traces. The gradient is linear in the
    residual, so the FP32 forward's ~1e-6 trace error would reach it amplified by |M| / |r|; the
    compensated forward steps (hi + lo planes) keep it within the plain 1e-4 bound."""
    wl = inputs.make_workload("linear_disk", seed=65, nx=64, nz=64, nt=400, n_elem=16, n_tx=2)
    M_obs = _observed(wl)
    J_ref, g_ref, cd_ref = _oracle_grad(wl, wl.sos_start[0], M_obs[0])
    J, g, cd = _gpu_grad(d, wl, M_obs, ckpt_interval=50, forward_precision="compensated")
    ratio = np.linalg.norm(cd_ref - M_obs[0]) / np.linalg.norm(cd_ref)
    assert ratio < 1e-2
    assert rel_l2(cd[0], cd_ref) <= TRACE_TOL
    assert abs(J[0] - J_ref) <= 1e-6 * J_ref
    assert rel_l2(g[0], g_ref) <= GRAD_TOL
