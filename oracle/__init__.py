"""FP64 CPU oracle for the damped 2-D acoustic simulator and its misfit gradient.

Test infrastructure only: the tests, the smoke check and the CPU-baseline leg
of the benchmark load it; the library path never does. The arithmetic lives
in ``dufwi_oracle.c`` (plain C, FP64, one routine per passage of the paper);
this module compiles it with gcc and marshals numpy arrays through ctypes.

Physical conventions (paper Sec. II-A, Eqs. 2-6; readings in the C header):
``C`` is the SoS map ``[nz][nx]`` in m/s on the physical grid, element
positions are physical-grid node indices ``(ix, iz)``, traces are
``M[t][r] = U[t]`` at the receivers, ``J = sum (M_sim - M_obs)^2`` and
``g = dJ/dC``. An optional density map ``rho [nz][nx]`` (kg/m^3) selects the
variable-density operator of Eq. 1 (staggered differences with half-point
buoyancies); without it the density is constant and the compact Laplacian of
Eq. 2 is used.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dufwi_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("nt", ctypes.c_int), ("pml", ctypes.c_int),
                ("pml_R", ctypes.c_double), ("pml_cref", ctypes.c_double),
                ("fd_order", ctypes.c_int), ("boundary", ctypes.c_int),
                ("pml_alpha", ctypes.c_double)]


@dataclass(frozen=True)
class Problem:
    """Grid and time axis of one simulation (physical grid, unpadded)."""
    nx: int
    nz: int
    dx: float
    dt: float
    nt: int
    pml: int = 20
    pml_R: float = 1e-3
    pml_cref: float = 1540.0
    fd_order: int = 8
    boundary: int = 0          # 0: damping term D of Eq. 1; 1: convolutional PML
    pml_alpha: float = 0.0     # CPML frequency shift at the inner edge of the layer (1/s)

    @property
    def nxp(self) -> int:
        return self.nx + 2 * self.pml

    @property
    def nzp(self) -> int:
        return self.nz + 2 * self.pml

    def c_struct(self) -> _Problem:
        return _Problem(self.nx, self.nz, self.dx, self.dt, self.nt, self.pml,
                        self.pml_R, self.pml_cref, self.fd_order, self.boundary, self.pml_alpha)


def _get():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(_Problem)
        _lib.orc_fd_coeffs.argtypes = [ctypes.c_int, dp]
        _lib.orc_d0.argtypes = [pp]
        _lib.orc_d0.restype = ctypes.c_double
        _lib.orc_damping.argtypes = [pp, dp]
        _lib.orc_pad.argtypes = [pp, dp, dp]
        _lib.orc_laplacian.argtypes = [pp, dp, dp]
        _lib.orc_forward.argtypes = [pp, dp, ctypes.c_int, ctypes.c_int, dp,
                                     ctypes.c_int, ip, ip, dp]
        _lib.orc_adjoint_probe.argtypes = [pp, dp, ctypes.c_int, ip, ip, dp,
                                           ctypes.c_int, ctypes.c_int, dp]
        _lib.orc_misfit_gradient.argtypes = [pp, dp, ctypes.c_int, ip, ip, dp, ctypes.c_int,
                                             ctypes.c_int, ip, ip, dp, ctypes.c_int,
                                             dp, dp, dp]
        _lib.orc_stagger_coeffs.argtypes = [ctypes.c_int, dp]
        _lib.orc_cpml_coeffs.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp]
        _lib.orc_buoyancy.argtypes = [pp, dp, dp, dp]
        _lib.orc_div_b_grad.argtypes = [pp, dp, dp, dp, dp]
        _lib.orc_forward_rho.argtypes = [pp, dp, dp, ctypes.c_int, ctypes.c_int, dp,
                                         ctypes.c_int, ip, ip, dp]
        _lib.orc_adjoint_probe_rho.argtypes = [pp, dp, dp, ctypes.c_int, ip, ip, dp,
                                               ctypes.c_int, ctypes.c_int, dp]
        _lib.orc_misfit_gradient_rho.argtypes = [pp, dp, dp, ctypes.c_int, ip, ip, dp, ctypes.c_int,
                                                 ctypes.c_int, ip, ip, dp, ctypes.c_int,
                                                 dp, dp, dp]
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _rho(p, rho):
    """Density argument: None (constant density) or a [nz][nx] FP64 array (kept alive by the caller)."""
    if rho is None:
        return None, None
    r = _f64(rho)
    assert r.shape == (p.nz, p.nx)
    return r, _d(r)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError("oracle %s failed with status %d" % (what, rc))


def fd_coeffs(order: int) -> np.ndarray:
    c = np.zeros(5)
    _check(_get().orc_fd_coeffs(order, _d(c)), "fd_coeffs")
    return c[: order // 2 + 1].copy()


def d0(p: Problem) -> float:
    s = p.c_struct()
    return _get().orc_d0(ctypes.byref(s))


def damping(p: Problem) -> np.ndarray:
    s = p.c_struct()
    D = np.zeros((p.nzp, p.nxp))
    _check(_get().orc_damping(ctypes.byref(s), _d(D)), "damping")
    return D


def pad(p: Problem, C) -> np.ndarray:
    s = p.c_struct()
    C = _f64(C)
    out = np.zeros((p.nzp, p.nxp))
    _check(_get().orc_pad(ctypes.byref(s), _d(C), _d(out)), "pad")
    return out


def laplacian(p: Problem, u) -> np.ndarray:
    s = p.c_struct()
    u = _f64(u)
    assert u.shape == (p.nzp, p.nxp)
    out = np.zeros_like(u)
    _check(_get().orc_laplacian(ctypes.byref(s), _d(u), _d(out)), "laplacian")
    return out


def stagger_coeffs(order: int) -> np.ndarray:
    """Staggered first-difference weights s_1..s_{order/2}."""
    s = np.zeros(4)
    _check(_get().orc_stagger_coeffs(order, _d(s)), "stagger_coeffs")
    return s[: order // 2].copy()


def cpml_coeffs(p: Problem) -> dict:
    """CPML recursion coefficients (a, b) at the nodes and half points of each axis."""
    s = p.c_struct()
    ax = [np.zeros(p.nxp) for _ in range(4)]
    az = [np.zeros(p.nzp) for _ in range(4)]
    _check(_get().orc_cpml_coeffs(ctypes.byref(s), *[_d(v) for v in ax + az]), "cpml_coeffs")
    return {"a_node_x": ax[0], "b_node_x": ax[1], "a_half_x": ax[2], "b_half_x": ax[3],
            "a_node_z": az[0], "b_node_z": az[1], "a_half_z": az[2], "b_half_z": az[3]}


def buoyancy(p: Problem, rho_pad) -> tuple[np.ndarray, np.ndarray]:
    """Half-point buoyancies (bx at (x+1/2, z), bz at (x, z+1/2)) of a padded density map."""
    s = p.c_struct()
    r = _f64(rho_pad)
    assert r.shape == (p.nzp, p.nxp)
    bx, bz = np.zeros_like(r), np.zeros_like(r)
    _check(_get().orc_buoyancy(ctypes.byref(s), _d(r), _d(bx), _d(bz)), "buoyancy")
    return bx, bz


def div_b_grad(p: Problem, bx, bz, u) -> np.ndarray:
    """Staggered (1/dx^2)[D-_x(bx D+_x u) + D-_z(bz D+_z u)] on the padded grid."""
    s = p.c_struct()
    bx, bz, u = _f64(bx), _f64(bz), _f64(u)
    assert u.shape == bx.shape == bz.shape == (p.nzp, p.nxp)
    out = np.zeros_like(u)
    _check(_get().orc_div_b_grad(ctypes.byref(s), _d(bx), _d(bz), _d(u), _d(out)), "div_b_grad")
    return out


def forward(p: Problem, C, src, wavelet, rx_ix, rx_iz, rho=None) -> np.ndarray:
    """Traces ``[nt][n_rx]`` of one transmit from node ``src = (ix, iz)``."""
    s = p.c_struct()
    C = _f64(C)
    w = _f64(wavelet)
    rx_ix, rx_iz = _i32(rx_ix), _i32(rx_iz)
    assert C.shape == (p.nz, p.nx) and w.shape == (p.nt,) and rx_ix.shape == rx_iz.shape
    out = np.zeros((p.nt, rx_ix.size))
    r, rp = _rho(p, rho)
    _check(_get().orc_forward_rho(ctypes.byref(s), _d(C), rp, int(src[0]), int(src[1]), _d(w),
                                  rx_ix.size, _i(rx_ix), _i(rx_iz), _d(out)), "forward")
    return out


def adjoint_probe(p: Problem, C, rx_ix, rx_iz, q, probe, rho=None) -> np.ndarray:
    """Adjoint field ``lam[t]`` at node ``probe`` for receiver series ``q[nt][n_rx]``."""
    s = p.c_struct()
    C, q = _f64(C), _f64(q)
    rx_ix, rx_iz = _i32(rx_ix), _i32(rx_iz)
    assert q.shape == (p.nt, rx_ix.size)
    out = np.zeros(p.nt)
    r, rp = _rho(p, rho)
    _check(_get().orc_adjoint_probe_rho(ctypes.byref(s), _d(C), rp, rx_ix.size, _i(rx_ix), _i(rx_iz),
                                        _d(q), int(probe[0]), int(probe[1]), _d(out)), "adjoint_probe")
    return out


def misfit_gradient(p: Problem, C, tx_ix, tx_iz, wavelet, rx_ix, rx_iz, M_obs, ckpt: int = 0,
                    return_traces: bool = False, rho=None):
    """Misfit ``J`` and gradient ``g = dJ/dC`` (``[nz][nx]``) of one map.

    ``tx_ix, tx_iz``: ``[n_tx]``; ``wavelet``: ``[nt]`` or ``[n_tx][nt]``;
    ``rx_ix, rx_iz``: ``[n_tx][n_rx]``; ``M_obs``: ``[n_tx][nt][n_rx]``;
    ``ckpt``: snapshot interval of the forward fields (0 = keep all);
    ``rho``: optional density map ``[nz][nx]`` (variable-density operator).
    """
    s = p.c_struct()
    C = _f64(C)
    tx_ix, tx_iz = _i32(tx_ix).ravel(), _i32(tx_iz).ravel()
    n_tx = tx_ix.size
    w = _f64(wavelet)
    n_wav = 1 if w.ndim == 1 else w.shape[0]
    rx_ix, rx_iz = _i32(rx_ix).reshape(n_tx, -1), _i32(rx_iz).reshape(n_tx, -1)
    n_rx = rx_ix.shape[1]
    M_obs = _f64(M_obs).reshape(n_tx, p.nt, n_rx)
    J = np.zeros(1)
    g = np.zeros((p.nz, p.nx))
    M_sim = np.zeros((n_tx, p.nt, n_rx))
    r, rp = _rho(p, rho)
    _check(_get().orc_misfit_gradient_rho(ctypes.byref(s), _d(C), rp, n_tx, _i(tx_ix), _i(tx_iz),
                                          _d(w), n_wav, n_rx, _i(rx_ix), _i(rx_iz), _d(M_obs),
                                          int(ckpt), _d(J), _d(g), _d(M_sim)), "misfit_gradient")
    if return_traces:
        return float(J[0]), g, M_sim
    return float(J[0]), g
