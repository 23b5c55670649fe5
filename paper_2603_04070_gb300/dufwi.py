"""Python binding of the C ABI in ``include/dufwi.h`` (argument marshalling only).

Every step of the simulation and of the gradient runs in the sm_103a kernels of ``libdufwi.so``.
This module does four things: it checks tensor shapes, dtypes and devices; allocates outputs and
the workspace with torch; passes raw device pointers and the current CUDA stream; and turns
status codes into exceptions. There is no fallback: if the library is missing, importing this
module raises.

The names follow the paper (arXiv 2603.04070): ``sos`` is the SoS map C (Sec. II-A), channel
data ``cd`` are M = F(C) (Eqs. 3-4), ``misfit`` is the data term of Eq. 5 and ``grad`` is
g = dJ/dC (Eq. 6).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdufwi.so")

OK, ERR_INVALID_ARG, ERR_CFL, ERR_GEOMETRY, ERR_UNSUPPORTED = 0, 1, 2, 3, 4
ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE = 5, 6, 7, 8
SNAPSHOT_DTYPES = {"fp32": 0, "bf16": 1, "fp16": 2}
BOUNDARIES = {"damping": 0, "cpml": 1}
FORWARD_PRECISIONS = {"fp32": 0, "compensated": 1}
OPT_TILE_Z = 1
OPT_TWO_STEP = 2
OPT_REUSE_TABLES = 3
OPT_PERSISTENT = 4
OPT_TEST_STALL = 5
OPT_MULTI_TILE = 6
OPT_EARLY_LOADS = 7
OPT_SHOT_GROUPS = 8
OPT_MIN_CTAS = 9
OPT_CLUSTER = 10


class DufwiError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, status_string(status), status))


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("nt", ctypes.c_int32), ("pml_cells", ctypes.c_int32),
                ("pml_R", ctypes.c_double), ("pml_cref", ctypes.c_double),
                ("fd_order", ctypes.c_int32), ("snapshot_dtype", ctypes.c_int32),
                ("ckpt_interval", ctypes.c_int32), ("c_max", ctypes.c_double),
                ("boundary", ctypes.c_int32), ("pml_alpha", ctypes.c_double),
                ("forward_precision", ctypes.c_int32), ("kept_segments", ctypes.c_int32)]


class _Array(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int32),
                ("ix", ctypes.POINTER(ctypes.c_int32)),
                ("iz", ctypes.POINTER(ctypes.c_int32))]


class _MapSizes(ctypes.Structure):
    _fields_ = [("nx", ctypes.POINTER(ctypes.c_int32)), ("nz", ctypes.POINTER(ctypes.c_int32))]


class _Shots(ctypes.Structure):
    _fields_ = [("n_tx", ctypes.c_int32), ("n_rx", ctypes.c_int32),
                ("tx_elem", ctypes.POINTER(ctypes.c_int32)),
                ("rx_elem", ctypes.POINTER(ctypes.c_int32)),
                ("wavelet_per_tx", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdufwi.so is not built (run python -m paper_2603_04070_gb300.build_lib)")
    lib = ctypes.CDLL(LIB_PATH)
    P, A, S = ctypes.POINTER(_Problem), ctypes.POINTER(_Array), ctypes.POINTER(_Shots)
    vp, sz = ctypes.c_void_p, ctypes.c_size_t
    lib.dufwi_version.restype = ctypes.c_int32
    lib.dufwi_cfl_limit.argtypes = [ctypes.c_int32]
    lib.dufwi_cfl_limit.restype = ctypes.c_double
    lib.dufwi_status_string.argtypes = [ctypes.c_int]
    lib.dufwi_status_string.restype = ctypes.c_char_p
    lib.dufwi_simulate_workspace_size.argtypes = [P, S, ctypes.c_int32, ctypes.POINTER(sz)]
    lib.dufwi_workspace_size.argtypes = [P, S, ctypes.c_int32, ctypes.POINTER(sz)]
    lib.dufwi_workspace_status.argtypes = [vp, vp]
    lib.dufwi_simulate.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, sz, vp]
    lib.dufwi_misfit_gradient.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, vp, vp, vp, sz, vp]
    lib.dufwi_misfit.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, vp, vp, sz, vp]
    lib.dufwi_misfit_gradient_fp64.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, vp, vp, vp, sz, vp]
    lib.dufwi_profile_enable.argtypes = [ctypes.c_int]
    lib.dufwi_profile_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    lib.dufwi_launch_count.restype = ctypes.c_int64
    lib.dufwi_simulate_noalloc.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp]
    lib.dufwi_noalloc_status.argtypes = [vp]
    M = ctypes.POINTER(_MapSizes)
    lib.dufwi_simulate_sized.argtypes = [P, M, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, sz, vp]
    lib.dufwi_misfit_gradient_sized.argtypes = [P, M, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, vp, vp, vp, sz, vp]
    lib.dufwi_forward_save.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, sz, vp]
    lib.dufwi_jvp_workspace_size.argtypes = [P, S, ctypes.c_int32, ctypes.POINTER(sz)]
    lib.dufwi_jvp.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, vp, vp, sz, vp]
    lib.dufwi_backward.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, vp, sz, vp]
    lib.dufwi_second_order_workspace_size.argtypes = [P, S, ctypes.c_int32, ctypes.POINTER(sz)]
    lib.dufwi_second_order.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.dufwi_hvp.argtypes = [P, vp, vp, A, vp, S, ctypes.c_int32, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.dufwi_set_option.argtypes = [ctypes.c_int32, ctypes.c_int32]
    lib.dufwi_get_option.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    return lib


_lib = _load()


def status_string(status: int) -> str:
    return _lib.dufwi_status_string(int(status)).decode()


def cfl_limit(fd_order: int) -> float:
    return float(_lib.dufwi_cfl_limit(int(fd_order)))


def version() -> int:
    return int(_lib.dufwi_version())


@dataclass
class Problem:
    """Grid, time axis, absorbing layer, stencil and checkpointing (``dufwi_problem``)."""
    nx: int
    nz: int
    dx: float
    dt: float
    nt: int
    pml_cells: int = 20
    pml_R: float = 1e-3
    pml_cref: float = 1540.0
    fd_order: int = 8
    snapshot_dtype: str = "fp32"
    ckpt_interval: int = 0
    c_max: float = 1700.0
    boundary: str = "damping"          # "damping" (the term D of Eq. 1) or "cpml"
    pml_alpha: float = 0.0             # CPML frequency shift at the layer's inner edge (1/s)
    forward_precision: str = "fp32"    # "fp32" or "compensated" (hi + lo FP32 planes, error-free steps)
    kept_segments: int = 0             # last checkpoint segments whose history the forward sweep keeps

    def c_struct(self) -> _Problem:
        return _Problem(self.nx, self.nz, self.dx, self.dt, self.nt, self.pml_cells, self.pml_R,
                        self.pml_cref, self.fd_order, SNAPSHOT_DTYPES[self.snapshot_dtype],
                        self.ckpt_interval, self.c_max, BOUNDARIES[self.boundary], self.pml_alpha,
                        FORWARD_PRECISIONS[self.forward_precision], self.kept_segments)


class Geometry:
    """Element nodes and the transmit/receive pattern (``dufwi_array`` + ``dufwi_shots``)."""

    def __init__(self, elem_ix, elem_iz, tx_elem, rx_elem, wavelet_per_tx: bool = False):
        self.elem_ix = np.ascontiguousarray(elem_ix, dtype=np.int32)
        self.elem_iz = np.ascontiguousarray(elem_iz, dtype=np.int32)
        self.tx_elem = np.ascontiguousarray(tx_elem, dtype=np.int32).ravel()
        rx = np.ascontiguousarray(rx_elem, dtype=np.int32)
        self.rx_elem = rx.reshape(self.tx_elem.size, -1) if rx.size else rx.reshape(self.tx_elem.size, 0)
        self.wavelet_per_tx = bool(wavelet_per_tx)

    @property
    def n_tx(self) -> int:
        return self.tx_elem.size

    @property
    def n_rx(self) -> int:
        return self.rx_elem.shape[1]

    def c_structs(self):
        ip = ctypes.POINTER(ctypes.c_int32)
        arr = _Array(self.elem_ix.size, self.elem_ix.ctypes.data_as(ip), self.elem_iz.ctypes.data_as(ip))
        sh = _Shots(self.n_tx, self.n_rx, self.tx_elem.ctypes.data_as(ip),
                    self.rx_elem.ctypes.data_as(ip), int(self.wavelet_per_tx))
        return arr, sh

    @classmethod
    def from_workload(cls, wl) -> "Geometry":
        return cls(wl.elem_ix, wl.elem_iz, wl.tx_elem, wl.rx_elem)


def _check(rc: int, what: str):
    if rc != OK:
        raise DufwiError(rc, what)


def workspace_size(problem: Problem, geom: Geometry, n_maps: int, gradient: bool = True) -> int:
    pb = problem.c_struct()
    _, sh = geom.c_structs()
    out = ctypes.c_size_t(0)
    fn = _lib.dufwi_workspace_size if gradient else _lib.dufwi_simulate_workspace_size
    _check(fn(ctypes.byref(pb), ctypes.byref(sh), int(n_maps), ctypes.byref(out)), "workspace_size")
    return int(out.value)


def _dev_tensor(t: torch.Tensor, name: str, dtype, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _alloc_workspace(need: int, device) -> torch.Tensor:
    """The workspace buffer; an allocation failure becomes a DufwiError naming the size (the
    library itself never allocates device memory)."""
    try:
        return torch.empty(need, dtype=torch.uint8, device=device)
    except (torch.cuda.OutOfMemoryError, RuntimeError) as e:
        if "out of memory" not in str(e).lower():
            raise
        raise DufwiError(ERR_WORKSPACE, "could not allocate a workspace of %d bytes (%.2f GB) on %s: %s"
                         % (need, need / 1e9, device, str(e).splitlines()[0])) from e


def _workspace(problem, geom, n_maps, gradient, workspace, device):
    need = workspace_size(problem, geom, n_maps, gradient)
    if workspace is None:
        workspace = _alloc_workspace(need, device)
    elif workspace.numel() * workspace.element_size() < need:
        raise DufwiError(ERR_WORKSPACE, "workspace of %d bytes < %d" %
                         (workspace.numel() * workspace.element_size(), need))
    return workspace


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _sizes_struct(sizes, n_maps):
    """``sizes``: sequence of (nx, nz) per map -> (_MapSizes, keep-alive arrays)."""
    arr = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32).reshape(n_maps, 2))
    nx = np.ascontiguousarray(arr[:, 0])
    nz = np.ascontiguousarray(arr[:, 1])
    ip = ctypes.POINTER(ctypes.c_int32)
    return _MapSizes(nx.ctypes.data_as(ip), nz.ctypes.data_as(ip)), (nx, nz)


def simulate(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry, *,
             density: torch.Tensor | None = None, cd: torch.Tensor | None = None,
             workspace: torch.Tensor | None = None, stream=None, check: bool = False,
             sizes=None) -> torch.Tensor:
    """Channel data ``[n_maps][n_tx][nt][n_rx]`` for SoS maps ``sos [n_maps][nz][nx]`` (Eqs. 2-4).

    ``sizes``: optional per-map physical grids ``[(nx_b, nz_b)]`` inside the (nx, nz) envelope
    (``dufwi_simulate_sized``)."""
    n_maps = sos.shape[0]
    _dev_tensor(sos, "sos", torch.float32, (n_maps, problem.nz, problem.nx))
    wshape = (geom.n_tx, problem.nt) if geom.wavelet_per_tx else (problem.nt,)
    _dev_tensor(wavelet, "wavelet", torch.float32, wshape)
    if density is not None:
        _dev_tensor(density, "density", torch.float32, sos.shape)
    shape = (n_maps, geom.n_tx, problem.nt, geom.n_rx)
    if cd is None:
        cd = torch.empty(shape, dtype=torch.float32, device=sos.device)
    _dev_tensor(cd, "cd", torch.float32, shape)
    workspace = _workspace(problem, geom, n_maps, False, workspace, sos.device)
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    args = (sos.data_ptr(), density.data_ptr() if density is not None else None, ctypes.byref(arr),
            wavelet.data_ptr(), ctypes.byref(sh), n_maps, cd.data_ptr(), workspace.data_ptr(),
            workspace.numel() * workspace.element_size(), _stream(stream))
    if sizes is None:
        rc = _lib.dufwi_simulate(ctypes.byref(pb), *args)
    else:
        ms, _keep = _sizes_struct(sizes, n_maps)
        rc = _lib.dufwi_simulate_sized(ctypes.byref(pb), ctypes.byref(ms), *args)
    _check(rc, "dufwi_simulate")
    if check:
        _check(workspace_status(workspace, stream), "dufwi_simulate (device)")
    return cd


NOALLOC_SCRATCH_BYTES = 64 << 20


def simulate_noalloc(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry, *,
                     density: torch.Tensor | None = None, cd: torch.Tensor | None = None,
                     stream=None, check: bool = False) -> torch.Tensor:
    """Channel data as ``simulate``, through ``dufwi_simulate_noalloc``.

    That entry point is for callers that must not allocate device memory while running, e.g. a
    fixed-latency acquisition loop or an application that owns all device memory through its
    own pool. It takes its scratch space from a static 64 MiB array inside the library, instead
    of a workspace. All calls share that array, so calls that overlap on the GPU race. Only the
    output ``cd`` is allocated here, and only when the caller does not pass one. ``check``
    reads the device status word (``dufwi_noalloc_status``) and raises on a device-side error.
    """
    n_maps = sos.shape[0]
    _dev_tensor(sos, "sos", torch.float32, (n_maps, problem.nz, problem.nx))
    wshape = (geom.n_tx, problem.nt) if geom.wavelet_per_tx else (problem.nt,)
    _dev_tensor(wavelet, "wavelet", torch.float32, wshape)
    if density is not None:
        _dev_tensor(density, "density", torch.float32, sos.shape)
    shape = (n_maps, geom.n_tx, problem.nt, geom.n_rx)
    if cd is None:
        cd = torch.empty(shape, dtype=torch.float32, device=sos.device)
    _dev_tensor(cd, "cd", torch.float32, shape)
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    rc = _lib.dufwi_simulate_noalloc(ctypes.byref(pb), sos.data_ptr(),
                                     density.data_ptr() if density is not None else None, ctypes.byref(arr),
                                     wavelet.data_ptr(), ctypes.byref(sh), n_maps, cd.data_ptr(), _stream(stream))
    _check(rc, "dufwi_simulate_noalloc")
    if check:
        _check(noalloc_status(stream), "dufwi_simulate_noalloc (device)")
    return cd


def noalloc_status(stream=None) -> int:
    """Status word of the last ``simulate_noalloc`` on the current device (synchronises ``stream``)."""
    return int(_lib.dufwi_noalloc_status(_stream(stream)))


def misfit_gradient(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry,
                    cd_obs: torch.Tensor, *, density: torch.Tensor | None = None,
                    misfit: torch.Tensor | None = None, grad: torch.Tensor | None = None,
                    cd_sim: torch.Tensor | None = None, return_cd: bool = False,
                    workspace: torch.Tensor | None = None, stream=None, check: bool = False, sizes=None):
    """Misfit ``J [n_maps]`` (float64) and gradient ``dJ/dC [n_maps][nz][nx]`` (Eqs. 5-6).

    ``sizes``: optional per-map physical grids inside the envelope (``dufwi_misfit_gradient_sized``).
    A float64 ``grad`` selects ``dufwi_misfit_gradient_fp64`` (the FP64 cross-transmit sum and fold
    without the final rounding to FP32; uniform calls only)."""
    n_maps = sos.shape[0]
    _dev_tensor(sos, "sos", torch.float32, (n_maps, problem.nz, problem.nx))
    wshape = (geom.n_tx, problem.nt) if geom.wavelet_per_tx else (problem.nt,)
    _dev_tensor(wavelet, "wavelet", torch.float32, wshape)
    cshape = (n_maps, geom.n_tx, problem.nt, geom.n_rx)
    _dev_tensor(cd_obs, "cd_obs", torch.float32, cshape)
    if density is not None:
        _dev_tensor(density, "density", torch.float32, sos.shape)
    if misfit is None:
        misfit = torch.empty(n_maps, dtype=torch.float64, device=sos.device)
    if grad is None:
        grad = torch.empty_like(sos)
    _dev_tensor(misfit, "misfit", torch.float64, (n_maps,))
    grad64 = isinstance(grad, torch.Tensor) and grad.dtype == torch.float64
    if grad64 and sizes is not None:
        raise ValueError("a float64 gradient is available for uniform calls only")
    _dev_tensor(grad, "grad", torch.float64 if grad64 else torch.float32, sos.shape)
    if return_cd and cd_sim is None:
        cd_sim = torch.empty(cshape, dtype=torch.float32, device=sos.device)
    if cd_sim is not None:
        _dev_tensor(cd_sim, "cd_sim", torch.float32, cshape)
    workspace = _workspace(problem, geom, n_maps, True, workspace, sos.device)
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    args = (sos.data_ptr(), density.data_ptr() if density is not None else None,
            ctypes.byref(arr), wavelet.data_ptr(), ctypes.byref(sh), n_maps, cd_obs.data_ptr(),
            misfit.data_ptr(), grad.data_ptr(), cd_sim.data_ptr() if cd_sim is not None else None,
            workspace.data_ptr(), workspace.numel() * workspace.element_size(), _stream(stream))
    if grad64:
        rc = _lib.dufwi_misfit_gradient_fp64(ctypes.byref(pb), *args)
    elif sizes is None:
        rc = _lib.dufwi_misfit_gradient(ctypes.byref(pb), *args)
    else:
        ms, _keep = _sizes_struct(sizes, n_maps)
        rc = _lib.dufwi_misfit_gradient_sized(ctypes.byref(pb), ctypes.byref(ms), *args)
    _check(rc, "dufwi_misfit_gradient")
    if check:
        _check(workspace_status(workspace, stream), "dufwi_misfit_gradient (device)")
    if return_cd:
        return misfit, grad, cd_sim
    return misfit, grad


def misfit(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry, cd_obs: torch.Tensor, *,
           density: torch.Tensor | None = None, out: torch.Tensor | None = None,
           cd_sim: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None,
           check: bool = False) -> torch.Tensor:
    """Misfit ``J [n_maps]`` (float64) alone, from one forward sweep (``dufwi_misfit``). Takes the
    gradient's workspace; J equals the one ``misfit_gradient`` returns, bit for bit."""
    n_maps, cshape = _common_inputs(problem, sos, wavelet, geom, density)
    _dev_tensor(cd_obs, "cd_obs", torch.float32, cshape)
    if out is None:
        out = torch.empty(n_maps, dtype=torch.float64, device=sos.device)
    _dev_tensor(out, "misfit", torch.float64, (n_maps,))
    if cd_sim is not None:
        _dev_tensor(cd_sim, "cd_sim", torch.float32, cshape)
    workspace = _workspace(problem, geom, n_maps, True, workspace, sos.device)
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    rc = _lib.dufwi_misfit(ctypes.byref(pb), sos.data_ptr(), density.data_ptr() if density is not None else None,
                           ctypes.byref(arr), wavelet.data_ptr(), ctypes.byref(sh), n_maps, cd_obs.data_ptr(),
                           out.data_ptr(), cd_sim.data_ptr() if cd_sim is not None else None,
                           workspace.data_ptr(), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "dufwi_misfit")
    if check:
        _check(workspace_status(workspace, stream), "dufwi_misfit (device)")
    return out


def _common_inputs(problem, sos, wavelet, geom, density):
    n_maps = sos.shape[0]
    _dev_tensor(sos, "sos", torch.float32, (n_maps, problem.nz, problem.nx))
    wshape = (geom.n_tx, problem.nt) if geom.wavelet_per_tx else (problem.nt,)
    _dev_tensor(wavelet, "wavelet", torch.float32, wshape)
    if density is not None:
        _dev_tensor(density, "density", torch.float32, sos.shape)
    return n_maps, (n_maps, geom.n_tx, problem.nt, geom.n_rx)


def forward_save(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry, *,
                 workspace: torch.Tensor | None = None, density: torch.Tensor | None = None,
                 cd: torch.Tensor | None = None, stream=None):
    """Channel data plus the saved snapshots/history in ``workspace`` (``dufwi_forward_save``).

    Returns ``(cd, workspace)``; pass the same workspace to ``backward``."""
    n_maps, cshape = _common_inputs(problem, sos, wavelet, geom, density)
    if cd is None:
        cd = torch.empty(cshape, dtype=torch.float32, device=sos.device)
    _dev_tensor(cd, "cd", torch.float32, cshape)
    workspace = _workspace(problem, geom, n_maps, True, workspace, sos.device)
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    rc = _lib.dufwi_forward_save(ctypes.byref(pb), sos.data_ptr(), density.data_ptr() if density is not None else None,
                                 ctypes.byref(arr), wavelet.data_ptr(), ctypes.byref(sh), n_maps, cd.data_ptr(),
                                 workspace.data_ptr(), workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "dufwi_forward_save")
    return cd, workspace


def backward(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry, cd_grad: torch.Tensor,
             workspace: torch.Tensor, *, density: torch.Tensor | None = None, grad: torch.Tensor | None = None,
             stream=None, check: bool = False) -> torch.Tensor:
    """(dM/dC)^T cd_grad for every map (``dufwi_backward``), after ``forward_save`` on ``workspace``."""
    n_maps, cshape = _common_inputs(problem, sos, wavelet, geom, density)
    _dev_tensor(cd_grad, "cd_grad", torch.float32, cshape)
    if grad is None:
        grad = torch.empty_like(sos)
    _dev_tensor(grad, "grad", torch.float32, sos.shape)
    need = workspace_size(problem, geom, n_maps, True)
    if workspace.numel() * workspace.element_size() < need:
        raise DufwiError(ERR_WORKSPACE, "backward workspace")
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    rc = _lib.dufwi_backward(ctypes.byref(pb), sos.data_ptr(), density.data_ptr() if density is not None else None,
                             ctypes.byref(arr), wavelet.data_ptr(), ctypes.byref(sh), n_maps, cd_grad.data_ptr(),
                             grad.data_ptr(), workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                             _stream(stream))
    _check(rc, "dufwi_backward")
    if check:
        _check(workspace_status(workspace, stream), "dufwi_backward (device)")
    return grad


def jvp_workspace_size(problem: Problem, geom: Geometry, n_maps: int) -> int:
    pb = problem.c_struct()
    _, sh = geom.c_structs()
    out = ctypes.c_size_t(0)
    _check(_lib.dufwi_jvp_workspace_size(ctypes.byref(pb), ctypes.byref(sh), int(n_maps), ctypes.byref(out)),
           "jvp_workspace_size")
    return int(out.value)


def jvp(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry, dsos: torch.Tensor, *,
        density: torch.Tensor | None = None, dcd: torch.Tensor | None = None, cd: torch.Tensor | None = None,
        return_cd: bool = False, workspace: torch.Tensor | None = None, stream=None, check: bool = False):
    """Linearised (Born) channel data dM = (dM/dC) dsos (``dufwi_jvp``); optionally also M."""
    n_maps, cshape = _common_inputs(problem, sos, wavelet, geom, density)
    _dev_tensor(dsos, "dsos", torch.float32, sos.shape)
    if dcd is None:
        dcd = torch.empty(cshape, dtype=torch.float32, device=sos.device)
    _dev_tensor(dcd, "dcd", torch.float32, cshape)
    if return_cd and cd is None:
        cd = torch.empty(cshape, dtype=torch.float32, device=sos.device)
    if cd is not None:
        _dev_tensor(cd, "cd", torch.float32, cshape)
    need = jvp_workspace_size(problem, geom, n_maps)
    if workspace is None:
        workspace = _alloc_workspace(need, sos.device)
    elif workspace.numel() * workspace.element_size() < need:
        raise DufwiError(ERR_WORKSPACE, "jvp workspace")
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    rc = _lib.dufwi_jvp(ctypes.byref(pb), sos.data_ptr(), density.data_ptr() if density is not None else None,
                        ctypes.byref(arr), wavelet.data_ptr(), ctypes.byref(sh), n_maps, dsos.data_ptr(),
                        dcd.data_ptr(), cd.data_ptr() if cd is not None else None, workspace.data_ptr(),
                        workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "dufwi_jvp")
    if check:
        _check(workspace_status(workspace, stream), "dufwi_jvp (device)")
    return (dcd, cd) if return_cd else dcd


def second_order_workspace_size(problem: Problem, geom: Geometry, n_maps: int) -> int:
    pb = problem.c_struct()
    _, sh = geom.c_structs()
    out = ctypes.c_size_t(0)
    _check(_lib.dufwi_second_order_workspace_size(ctypes.byref(pb), ctypes.byref(sh), int(n_maps),
                                                  ctypes.byref(out)), "second_order_workspace_size")
    return int(out.value)


def second_order(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry, cd_grad: torch.Tensor,
                 dsos: torch.Tensor, *, so: torch.Tensor | None = None, dcd: torch.Tensor | None = None,
                 grad: torch.Tensor | None = None, return_grad: bool = False, workspace: torch.Tensor | None = None,
                 stream=None, check: bool = False, density: torch.Tensor | None = None):
    """Second-order product ``so = d/dC[(dM/dC)^T cd_grad] . dsos`` and the Born data
    ``dcd = (dM/dC) dsos`` (``dufwi_second_order``); with ``return_grad`` also
    ``grad = (dM/dC)^T cd_grad``. Returns ``(so, dcd)`` or ``(so, dcd, grad)``.

    With ``cd_grad = 2 (M - M_obs)`` the exact Hessian-vector product of the misfit is
    ``so + 2 (dM/dC)^T dcd``. ``density``: optional map (variable-density operator of Eq. 1)."""
    n_maps, cshape = _common_inputs(problem, sos, wavelet, geom, density)
    _dev_tensor(cd_grad, "cd_grad", torch.float32, cshape)
    _dev_tensor(dsos, "dsos", torch.float32, sos.shape)
    if so is None:
        so = torch.empty_like(sos)
    _dev_tensor(so, "so", torch.float32, sos.shape)
    if dcd is None:
        dcd = torch.empty(cshape, dtype=torch.float32, device=sos.device)
    _dev_tensor(dcd, "dcd", torch.float32, cshape)
    if return_grad and grad is None:
        grad = torch.empty_like(sos)
    if grad is not None:
        _dev_tensor(grad, "grad", torch.float32, sos.shape)
    need = second_order_workspace_size(problem, geom, n_maps)
    if workspace is None:
        workspace = _alloc_workspace(need, sos.device)
    elif workspace.numel() * workspace.element_size() < need:
        raise DufwiError(ERR_WORKSPACE, "second_order workspace")
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    rc = _lib.dufwi_second_order(ctypes.byref(pb), sos.data_ptr(), density.data_ptr() if density is not None else None,
                                 ctypes.byref(arr), wavelet.data_ptr(),
                                 ctypes.byref(sh), n_maps, cd_grad.data_ptr(), dsos.data_ptr(), dcd.data_ptr(),
                                 so.data_ptr(), grad.data_ptr() if grad is not None else None, workspace.data_ptr(),
                                 workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "dufwi_second_order")
    if check:
        _check(workspace_status(workspace, stream), "dufwi_second_order (device)")
    return (so, dcd, grad) if return_grad else (so, dcd)


def hvp(problem: Problem, sos: torch.Tensor, wavelet: torch.Tensor, geom: Geometry, cd_obs: torch.Tensor,
        dsos: torch.Tensor, *, hv: torch.Tensor | None = None, misfit: torch.Tensor | None = None,
        grad: torch.Tensor | None = None, return_all: bool = False, workspace: torch.Tensor | None = None,
        stream=None, check: bool = False, density: torch.Tensor | None = None):
    """Exact Hessian-vector product ``H dsos`` of the misfit J = sum (M - M_obs)^2 per map
    (``dufwi_hvp``), one call. With ``return_all`` returns ``(hv, misfit [n_maps] float64,
    grad)``: the misfit and its gradient come from the same sweeps. ``density``: optional map
    (variable-density operator of Eq. 1)."""
    n_maps, cshape = _common_inputs(problem, sos, wavelet, geom, density)
    _dev_tensor(cd_obs, "cd_obs", torch.float32, cshape)
    _dev_tensor(dsos, "dsos", torch.float32, sos.shape)
    if hv is None:
        hv = torch.empty_like(sos)
    _dev_tensor(hv, "hv", torch.float32, sos.shape)
    if return_all:
        if misfit is None:
            misfit = torch.empty(n_maps, dtype=torch.float64, device=sos.device)
        if grad is None:
            grad = torch.empty_like(sos)
    if misfit is not None:
        _dev_tensor(misfit, "misfit", torch.float64, (n_maps,))
    if grad is not None:
        _dev_tensor(grad, "grad", torch.float32, sos.shape)
    need = second_order_workspace_size(problem, geom, n_maps)
    if workspace is None:
        workspace = _alloc_workspace(need, sos.device)
    elif workspace.numel() * workspace.element_size() < need:
        raise DufwiError(ERR_WORKSPACE, "hvp workspace")
    pb = problem.c_struct()
    arr, sh = geom.c_structs()
    rc = _lib.dufwi_hvp(ctypes.byref(pb), sos.data_ptr(), density.data_ptr() if density is not None else None,
                        ctypes.byref(arr), wavelet.data_ptr(),
                        ctypes.byref(sh), n_maps, cd_obs.data_ptr(), dsos.data_ptr(), hv.data_ptr(),
                        misfit.data_ptr() if misfit is not None else None,
                        grad.data_ptr() if grad is not None else None, workspace.data_ptr(),
                        workspace.numel() * workspace.element_size(), _stream(stream))
    _check(rc, "dufwi_hvp")
    if check:
        _check(workspace_status(workspace, stream), "dufwi_hvp (device)")
    return (hv, misfit, grad) if return_all else hv


def workspace_status(workspace: torch.Tensor, stream=None) -> int:
    """Synchronises the stream and returns the device status word of the last call."""
    return int(_lib.dufwi_workspace_status(ctypes.c_void_p(workspace.data_ptr()), _stream(stream)))


PROFILE_KINDS = ("forward", "recompute", "adjoint", "other")


def profile_enable(enable: bool = True):
    """Start/stop event timing of the sweeps (``dufwi_profile_enable``)."""
    _check(_lib.dufwi_profile_enable(int(bool(enable))), "dufwi_profile_enable")


def profile_read(reset: bool = True) -> dict:
    """Accumulated sweep times (ms) and kernel launches per kind since the last reset."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int64 * 4)()
    rc = _lib.dufwi_profile_read(ms, n, int(bool(reset)))
    if rc not in (OK, ERR_WORKSPACE):
        raise DufwiError(rc, "dufwi_profile_read")
    return {k: {"ms": ms[i], "launches": int(n[i])} for i, k in enumerate(PROFILE_KINDS)} | {
        "complete": rc == OK}


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(_lib.dufwi_launch_count())


def set_option(option: int, value: int):
    """Process-wide tuning option (``dufwi_set_option``), e.g. ``OPT_TILE_Z`` = 32 or 64."""
    _check(_lib.dufwi_set_option(int(option), int(value)), "dufwi_set_option")


def get_option(option: int) -> int:
    v = ctypes.c_int32(0)
    _check(_lib.dufwi_get_option(int(option), ctypes.byref(v)), "dufwi_get_option")
    return int(v.value)
