"""Multi-rank logic on CPU: shard helpers, and the transmit-sharded gradient with its FP64 sum
over two gloo ranks (the oracle stands in for each rank's GPU computation)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2603_04070_gb300 import inputs, parallel


def test_block_ranges_partition_exactly():
    for n in (0, 1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            got = [list(parallel.block_range(n, world, r)) for r in range(world)]
            flat = [i for part in got for i in part]
            assert flat == list(range(n))
            sizes = [len(p) for p in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        parallel.block_range(4, 2, 2)


def test_allreduce_without_process_group_is_identity():
    J = torch.tensor([1.5, 2.0], dtype=torch.float64)
    g = torch.ones(2, 3, 4)
    J2, g2 = parallel.gradient_allreduce(J, g)
    assert torch.equal(J2, J) and torch.equal(g2, g)


def _oracle_compute(problem, sos, wavelet, geom, cd_obs):
    import oracle
    wl = problem
    p = oracle.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml=wl.pml_cells, pml_R=wl.pml_R,
                       pml_cref=wl.pml_cref, fd_order=wl.fd_order)
    ix = geom.elem_ix[geom.tx_elem]
    iz = geom.elem_iz[geom.tx_elem]
    Js, gs = [], []
    for b in range(sos.shape[0]):
        J, g = oracle.misfit_gradient(p, sos[b].double().numpy(), ix, iz, wavelet.double().numpy(),
                                      geom.elem_ix[geom.rx_elem], geom.elem_iz[geom.rx_elem],
                                      cd_obs[b].double().numpy())
        Js.append(J)
        gs.append(g)
    return torch.tensor(Js, dtype=torch.float64), torch.from_numpy(np.stack(gs)).float()


def _oracle_compute64(problem, sos, wavelet, geom, cd_obs):
    import oracle
    wl = problem
    p = oracle.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml=wl.pml_cells, pml_R=wl.pml_R,
                       pml_cref=wl.pml_cref, fd_order=wl.fd_order)
    return torch.from_numpy(np.stack([
        oracle.misfit_gradient(p, sos[b].double().numpy(), geom.elem_ix[geom.tx_elem], geom.elem_iz[geom.tx_elem],
                               wavelet.double().numpy(), geom.elem_ix[geom.rx_elem], geom.elem_iz[geom.rx_elem],
                               cd_obs[b].double().numpy())[1] for b in range(sos.shape[0])]))


def _oracle_compute_fp64(problem, sos, wavelet, geom, cd_obs):
    """(J, g) of this rank's transmits with g left in FP64, as the library's FP64 gradient output
    (dufwi_misfit_gradient_fp64) hands it to the sharded sum."""
    J, _ = _oracle_compute(problem, sos, wavelet, geom, cd_obs)
    return J, _oracle_compute64(problem, sos, wavelet, geom, cd_obs)


def _oracle_hvp(problem, sos, wavelet, geom, cd_obs, v):
    """(H v, J, g) of this rank's transmits: central differences (FP64) of the oracle gradient
    along v."""
    h = 0.05
    J, g = _oracle_compute(problem, sos, wavelet, geom, cd_obs)
    gp = _oracle_compute64(problem, sos.double() + h * v.double(), wavelet, geom, cd_obs)
    gm = _oracle_compute64(problem, sos.double() - h * v.double(), wavelet, geom, cd_obs)
    return (gp - gm) / (2 * h), J, g


def _case():
    from paper_2603_04070_gb300 import dufwi
    wl = inputs.make_workload("linear_disk", seed=31, nx=24, nz=20, nt=120, n_elem=6, n_tx=3, n_maps=2)
    wl.pml = 6
    pb = dufwi.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml_cells=6, pml_R=wl.pml_R,
                       pml_cref=wl.pml_cref, fd_order=wl.fd_order)
    geom = dufwi.Geometry.from_workload(wl)
    rng = np.random.default_rng(3)
    obs = torch.from_numpy(rng.standard_normal((2, wl.n_tx, wl.nt, wl.n_rx)).astype(np.float32) * 1e-9)
    return pb, geom, torch.from_numpy(wl.sos_true), torch.from_numpy(wl.wavelet), obs


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pb, geom, sos, w, obs = _case()
        J, g = parallel.sharded_misfit_gradient(pb, sos, w, geom, obs, compute=_oracle_compute)
        J64, g64 = parallel.sharded_misfit_gradient(pb, sos, w, geom, obs, compute=_oracle_compute_fp64)
        v = torch.from_numpy(np.random.default_rng(5).standard_normal(tuple(sos.shape))) * 5.0
        hv, J2, g2 = parallel.sharded_hvp(pb, sos, w, geom, obs, v, compute=_oracle_hvp)
        if rank == 0:
            torch.save({"J": J, "g": g, "g64": g64, "hv": hv, "J2": J2, "g2": g2, "v": v}, out_path)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_transmit_sharded_gradient_on_two_gloo_ranks(tmp_path):
    from paper_2603_04070_gb300 import build_lib
    build_lib.build()          # once, before the ranks import the binding
    out = str(tmp_path / "res.pt")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    res = torch.load(out)
    pb, geom, sos, w, obs = _case()
    J_ref, g_ref = _oracle_compute(pb, sos, w, geom, obs)
    assert torch.allclose(res["J"], J_ref, rtol=1e-12, atol=0)
    assert torch.allclose(res["g"], g_ref, rtol=1e-5, atol=1e-6 * float(g_ref.abs().max()))
    # FP64 partials: the sum is FP64 to the end and rounded once, so it is the whole-set FP64
    # gradient rounded to FP32, up to one unit in the last place from the FP64 summation order
    g64_ref = _oracle_compute64(pb, sos, w, geom, obs)
    assert res["g64"].dtype == torch.float32
    ulp = torch.abs(torch.nextafter(g64_ref.float(), torch.tensor(float("inf"))) - g64_ref.float())
    assert bool((res["g64"] - g64_ref.float()).abs().le(ulp).all())
    # the HVP split: the per-rank products (and misfits, gradients) sum to the whole-set ones
    hv_ref, _, _ = _oracle_hvp(pb, sos, w, geom, obs, res["v"])
    assert torch.allclose(res["J2"], J_ref, rtol=1e-12, atol=0)
    assert torch.allclose(res["g2"], g_ref, rtol=1e-5, atol=1e-6 * float(g_ref.abs().max()))
    assert float((res["hv"].double() - hv_ref).norm() / hv_ref.norm()) <= 1e-6


def _failing_worker(rank, world, port, out_dir):
    """Rank 1's computation fails before the collective (an exception on the host); rank 0 must
    see an error from the all-reduce within the process group's timeout instead of waiting."""
    import datetime
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    pb, geom, sos, w, obs = _case()

    def compute(problem, s, wav, g, o):
        if rank == 1:
            raise RuntimeError("injected failure on rank 1")
        return _oracle_compute(problem, s, wav, g, o)

    t0 = time.time()
    try:
        parallel.sharded_misfit_gradient(pb, sos, w, geom, obs, compute=compute)
        outcome = "completed"
    except Exception as e:   # rank 0: the collective fails; rank 1: the injected error
        outcome = "%s: %s" % (type(e).__name__, str(e).splitlines()[0] if str(e) else "")
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%s\n%.1f\n" % (outcome, time.time() - t0))
    if rank == 1:
        os._exit(3)                 # the failed rank leaves without tearing the group down
    try:
        dist.destroy_process_group()
    except Exception:
        pass


def test_a_failed_rank_is_reported_not_waited_for(tmp_path):
    """Failure detection on the host (no GPU involved): a rank that raises before the FP64
    all-reduce of the transmit-sharded gradient leaves; the other rank's collective ends with an
    error within the 10 s process-group timeout instead of waiting on it."""
    from paper_2603_04070_gb300 import build_lib
    build_lib.build()
    sp = mp.get_context("spawn")
    port = _free_port()
    procs = [sp.Process(target=_failing_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p_ in procs:
        p_.start()
    for p_ in procs:
        p_.join(timeout=120)
    alive = [p_ for p_ in procs if p_.is_alive()]
    for p_ in alive:                 # only if the bound above was exceeded: end this test's own processes
        p_.kill()
    assert not alive
    assert procs[1].exitcode == 3
    r0 = (tmp_path / "rank0.txt").read_text().split("\n")
    r1 = (tmp_path / "rank1.txt").read_text().split("\n")
    assert r1[0].startswith("RuntimeError: injected failure")
    assert not r0[0].startswith("completed")
    assert float(r0[1]) < 30.0
