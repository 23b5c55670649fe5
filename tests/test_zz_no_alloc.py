"""The allocation-free forward entry point against the regular one.

dufwi_simulate_noalloc serves callers that cannot allocate device memory while running, for
example a fixed-latency acquisition loop, or an application whose memory pool owns the whole GPU.
It draws its scratch from a static array in the library. This test checks four things through
the C ABI:
  - its channel data match dufwi_simulate with a caller workspace, within the traces tolerance;
  - this holds on two calls in a row, so leftovers in the shared array do not leak into results;
  - the second call still matches after the array was dirtied by a different, larger problem;
  - problems larger than the array are rejected without device work.
The file name sorts last, so a first failure here comes after every other test has run.
"""
import numpy as np
import pytest
import torch

from paper_2603_04070_gb300 import inputs

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-5


@pytest.fixture(scope="module")
def d():
    from paper_2603_04070_gb300 import build_lib
    build_lib.build()
    from paper_2603_04070_gb300 import dufwi
    return dufwi


def _rel_l2(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


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
        out = d.simulate_noalloc(pb, sos, w, geom)
        torch.cuda.synchronize()
        assert _rel_l2(out, ref) <= TRACE_TOL
    # dirty the shared array with a different problem, then repeat the first one
    pb2, geom2, sos2, w2 = _case(d, 12, 150, 140, 300, 4, 1)
    ref2 = d.simulate(pb2, sos2, w2, geom2)
    assert _rel_l2(d.simulate_noalloc(pb2, sos2, w2, geom2), ref2) <= TRACE_TOL
    out = d.simulate_noalloc(pb, sos, w, geom)
    torch.cuda.synchronize()
    assert _rel_l2(out, ref) <= TRACE_TOL


def test_noalloc_rejects_problems_beyond_the_array(d):
    pb, geom, sos, w = _case(d, 13, 512, 512, 100, 16, 2)
    assert d.workspace_size(pb, geom, 2, gradient=False) > d.NOALLOC_SCRATCH_BYTES
    with pytest.raises(d.DufwiError) as e:
        d.simulate_noalloc(pb, sos, w, geom)
    assert e.value.status == d.ERR_WORKSPACE
