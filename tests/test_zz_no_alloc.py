"""The allocation-free forward entry point against the regular one.

dufwi_simulate_noalloc serves callers that cannot allocate device memory while running, for
example a fixed-latency acquisition loop, or an application whose memory pool owns the whole GPU.
It draws its scratch from a static array in the library. Both entry points run the same kernels
on the same inputs, so their channel data must agree bit for bit. This file checks, through the
C ABI:
  - equality with dufwi_simulate (caller workspace) on two calls in a row, so leftovers in the
    shared array do not leak into results;
  - equality after the array was dirtied by a different problem with a larger workspace;
  - the same with DUFWI_OPT_REUSE_TABLES set, whose per-address table cache always sees the same
    scratch address on this path, alternating two problems;
  - the device status word of the array (an SoS value above c_max is reported, then cleared by
    the next good call);
  - problems larger than the array are rejected without device work.
The file name sorts last, so a first failure here comes after every other test has run.
"""
import pytest
import torch

from paper_2603_04070_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def d():
    from paper_2603_04070_gb300 import build_lib
    build_lib.build()
    from paper_2603_04070_gb300 import dufwi
    return dufwi


def _case(d, seed, nx, nz, nt, n_tx, n_maps):
    wl = inputs.make_workload("linear_disk", seed=seed, nx=nx, nz=nz, nt=nt, n_elem=20, n_tx=n_tx, n_maps=n_maps)
    pb = d.Problem(nx=wl.nx, nz=wl.nz, dx=wl.dx, dt=wl.dt, nt=wl.nt, pml_cells=wl.pml, pml_R=wl.pml_R,
                   pml_cref=wl.pml_cref, fd_order=wl.fd_order, c_max=wl.c_max)
    geom = d.Geometry.from_workload(wl)
    return pb, geom, torch.from_numpy(wl.sos_true).cuda(), torch.from_numpy(wl.wavelet).cuda()


def test_noalloc_matches_workspace_path_twice(d):
    pb, geom, sos, w = _case(d, 11, 97, 83, 700, 3, 2)
    ref = d.simulate(pb, sos, w, geom, check=True)
    assert d.workspace_size(pb, geom, 2, gradient=False) <= d.NOALLOC_SCRATCH_BYTES
    for _ in range(2):
        out = d.simulate_noalloc(pb, sos, w, geom, check=True)
        assert torch.equal(out, ref)
    # dirty the shared array with a problem whose workspace covers the first one's, then repeat
    pb2, geom2, sos2, w2 = _case(d, 12, 150, 140, 300, 4, 2)
    assert d.workspace_size(pb2, geom2, 2, gradient=False) >= d.workspace_size(pb, geom, 2, gradient=False)
    ref2 = d.simulate(pb2, sos2, w2, geom2)
    assert torch.equal(d.simulate_noalloc(pb2, sos2, w2, geom2, check=True), ref2)
    out = d.simulate_noalloc(pb, sos, w, geom, check=True)
    assert torch.equal(out, ref)


def test_noalloc_with_table_reuse_alternating_problems(d):
    """With DUFWI_OPT_REUSE_TABLES the library skips re-copying tables it already placed at a
    workspace address. On this path the address is always the static array's, so alternating
    two problems must still upload each problem's tables (their hashes differ)."""
    pb, geom, sos, w = _case(d, 14, 90, 70, 400, 2, 2)
    pb2, geom2, sos2, w2 = _case(d, 15, 120, 96, 250, 3, 1)
    ref = d.simulate(pb, sos, w, geom)
    ref2 = d.simulate(pb2, sos2, w2, geom2)
    d.set_option(d.OPT_REUSE_TABLES, 1)
    try:
        for _ in range(2):
            assert torch.equal(d.simulate_noalloc(pb, sos, w, geom, check=True), ref)
            assert torch.equal(d.simulate_noalloc(pb2, sos2, w2, geom2, check=True), ref2)
    finally:
        d.set_option(d.OPT_REUSE_TABLES, 0)


def test_noalloc_status_word(d):
    """An SoS value above c_max is recorded in the array's status word and reported by
    dufwi_noalloc_status; the next good call starts from a cleared word."""
    pb, geom, sos, w = _case(d, 16, 60, 50, 120, 2, 1)
    bad = sos.clone()
    bad[0, 7, 9] = 2.0 * pb.c_max
    d.simulate_noalloc(pb, bad, w, geom)
    assert d.noalloc_status() == d.ERR_CFL
    with pytest.raises(d.DufwiError) as e:
        d.simulate_noalloc(pb, bad, w, geom, check=True)
    assert e.value.status == d.ERR_CFL
    ref = d.simulate(pb, sos, w, geom)
    assert torch.equal(d.simulate_noalloc(pb, sos, w, geom, check=True), ref)
    assert d.noalloc_status() == d.OK


def test_noalloc_rejects_problems_beyond_the_array(d):
    pb, geom, sos, w = _case(d, 13, 512, 512, 100, 16, 2)
    assert d.workspace_size(pb, geom, 2, gradient=False) > d.NOALLOC_SCRATCH_BYTES
    with pytest.raises(d.DufwiError) as e:
        d.simulate_noalloc(pb, sos, w, geom)
    assert e.value.status == d.ERR_WORKSPACE
