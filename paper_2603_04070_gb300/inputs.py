"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and the benchmark.

This module draws speed-of-sound maps, the source pulse and the array geometry. It holds no
part of the simulator's or the gradient's arithmetic. Every draw comes from
``numpy.random.Generator(PCG64(seed))``.

These inputs stand in for the paper's datasets (MNIST-derived maps, the simulated arm and the
phantom rods, Sec. V). Those datasets are not available here. The maps reuse the paper's
structure: a water-like background with compact inclusions (Sec. V, Sec. VII). The workloads:

* ``disk``: one hard disk, radius U[1.5, 3] mm, SoS U[1450, 1520] m/s, in 1540 m/s.
* ``grf_rods``: 1540 m/s plus a smooth Gaussian random field (+-20 m/s, correlation 3 mm),
  plus 1-4 non-overlapping rods, radius U[1, 5] mm, SoS U[1450, 1600] m/s.
* a linear array on the top physical row, point elements every 3 cells (0.3 mm at
  dx = 0.1 mm), centred; transmits evenly spaced as floor((j + 0.5) n_elem / n_tx).
* a 2 MHz Ricker pulse of peak 1, delayed by 1.5 / f0.
* ``ring_phantom`` (the paper's own hardware geometry, Sec. IV and Sec. VII): a 188 x 188 grid
  over 10 cm, a 16-element ring of 10 cm diameter, every element transmits and the opposite
  element and its two neighbours receive (3 channels per transmit), a 350 kHz
  derivative-of-Gaussian pulse, 1034 steps of 90.243 ns. Maps hold 1-3 rods of 1 cm diameter,
  each bone (2700 m/s) or edema (1588 m/s), in 1500 m/s water. Observed data may carry additive
  white Gaussian noise at a given SNR (30 dB in the paper's tests, Sec. V).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BACKGROUND_SOS = 1540.0
WATER_SOS = 1500.0


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ricker(nt: int, dt: float, f0: float, delay: float | None = None) -> np.ndarray:
    """Ricker pulse w(n dt) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = n dt - delay."""
    if delay is None:
        delay = 1.5 / f0
    tau = np.arange(nt, dtype=np.float64) * dt - delay
    arg = (math.pi * f0 * tau) ** 2
    return ((1.0 - 2.0 * arg) * np.exp(-arg)).astype(np.float32)


def gaussian_derivative_pulse(nt: int, dt: float, f0: float) -> np.ndarray:
    """Time derivative of a Gaussian (the paper's simulated pulse shape, Sec. IV), peak |w| = 1."""
    sigma = 1.0 / (2.0 * math.pi * f0)
    tau = np.arange(nt, dtype=np.float64) * dt - 4.0 * sigma
    w = -tau * np.exp(-0.5 * (tau / sigma) ** 2)
    return (w / np.max(np.abs(w))).astype(np.float32)


def linear_array(nx: int, n_elem: int, pitch_cells: int = 3, row: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Point elements on physical row ``row``, ``pitch_cells`` apart, centred in x."""
    span = pitch_cells * (n_elem - 1)
    if span >= nx:
        raise ValueError("array of %d elements does not fit %d cells" % (n_elem, nx))
    x0 = (nx - 1 - span) // 2
    ix = x0 + pitch_cells * np.arange(n_elem, dtype=np.int32)
    iz = np.full(n_elem, row, dtype=np.int32)
    return ix.astype(np.int32), iz


def ring_array(n: int, n_elem: int, radius_cells: float) -> tuple[np.ndarray, np.ndarray]:
    """Point elements evenly spaced on a circle centred in an n x n grid (the paper's ring, Sec. IV)."""
    c = (n - 1) / 2.0
    ang = 2.0 * math.pi * np.arange(n_elem) / n_elem
    ix = np.rint(c + radius_cells * np.cos(ang)).astype(np.int32)
    iz = np.rint(c + radius_cells * np.sin(ang)).astype(np.int32)
    return ix, iz


def evenly_spaced_transmits(n_elem: int, n_tx: int) -> np.ndarray:
    """Transmit element j = floor((j + 0.5) n_elem / n_tx)."""
    return np.floor((np.arange(n_tx) + 0.5) * n_elem / n_tx).astype(np.int32)


def disk_map(rng, nx: int, nz: int, dx: float, margin_m: float = 3e-3) -> np.ndarray:
    """One hard disk (node-centre test) in the 1540 m/s background."""
    r = rng.uniform(1.5e-3, 3e-3)
    c = rng.uniform(1450.0, 1520.0)
    lx, lz = (nx - 1) * dx, (nz - 1) * dx
    cx = rng.uniform(min(margin_m, lx / 2), max(lx - margin_m, lx / 2))
    cz = rng.uniform(min(margin_m, lz / 2), max(lz - margin_m, lz / 2))
    X = np.arange(nx) * dx
    Z = np.arange(nz) * dx
    inside = (X[None, :] - cx) ** 2 + (Z[:, None] - cz) ** 2 <= r * r
    sos = np.full((nz, nx), BACKGROUND_SOS, dtype=np.float64)
    sos[inside] = c
    return sos.astype(np.float32)


def _gaussian_field(rng, nx: int, nz: int, sigma_cells: float) -> np.ndarray:
    white = rng.standard_normal((nz, nx))
    kx = np.fft.fftfreq(nx)[None, :]
    kz = np.fft.fftfreq(nz)[:, None]
    filt = np.exp(-2.0 * (math.pi * sigma_cells) ** 2 * (kx * kx + kz * kz))
    return np.real(np.fft.ifft2(np.fft.fft2(white) * filt))


def grf_rods_map(rng, nx: int, nz: int, dx: float, max_rods: int = 4,
                 amp: float = 20.0, corr_m: float = 3e-3) -> np.ndarray:
    """1540 m/s + smooth Gaussian random field (max |.| = amp) + 1..max_rods hard rods."""
    f = _gaussian_field(rng, nx, nz, corr_m / math.sqrt(2.0) / dx)
    f *= amp / max(np.max(np.abs(f)), 1e-30)
    sos = BACKGROUND_SOS + f
    X = np.arange(nx) * dx
    Z = np.arange(nz) * dx
    n_rods = int(rng.integers(1, max_rods + 1))
    rods: list[tuple[float, float, float]] = []
    tries = 0
    while len(rods) < n_rods and tries < 1000:
        tries += 1
        r = rng.uniform(1e-3, max(1e-3, min(5e-3, 0.3 * (min(nx, nz) - 1) * dx)))   # fits small test grids
        cx = rng.uniform(r, (nx - 1) * dx - r)
        cz = rng.uniform(r, (nz - 1) * dx - r)
        if any((cx - x) ** 2 + (cz - z) ** 2 < (r + q) ** 2 for x, z, q in rods):
            continue
        rods.append((cx, cz, r))
        inside = (X[None, :] - cx) ** 2 + (Z[:, None] - cz) ** 2 <= r * r
        sos[inside] = rng.uniform(1450.0, 1600.0)
    return sos.astype(np.float32)


@dataclass
class Workload:
    """One batch of maps on one grid: everything both implementations need as input."""
    name: str
    nx: int
    nz: int
    dx: float
    dt: float
    nt: int
    sos_true: np.ndarray           # [B][nz][nx] float32, the map that produces the observed data
    sos_start: np.ndarray          # [B][nz][nx] float32, the map the gradient is taken at
    wavelet: np.ndarray            # [nt] float32 (shared by all transmits)
    elem_ix: np.ndarray            # [n_elem] int32, physical-grid node indices
    elem_iz: np.ndarray            # [n_elem] int32
    tx_elem: np.ndarray            # [n_tx] int32, element index of each transmit
    rx_elem: np.ndarray            # [n_tx][n_rx] int32, element indices receiving each transmit
    pml: int = 20
    pml_R: float = 1e-3
    pml_cref: float = BACKGROUND_SOS
    fd_order: int = 8
    c_max: float = 1700.0
    meta: dict = field(default_factory=dict)

    @property
    def n_maps(self) -> int:
        return self.sos_true.shape[0]

    @property
    def n_tx(self) -> int:
        return self.tx_elem.size

    @property
    def n_rx(self) -> int:
        return self.rx_elem.shape[1]

    def tx_nodes(self):
        return self.elem_ix[self.tx_elem], self.elem_iz[self.tx_elem]

    def rx_nodes(self):
        return self.elem_ix[self.rx_elem], self.elem_iz[self.rx_elem]

    @property
    def padded_cells(self) -> int:
        return (self.nx + 2 * self.pml) * (self.nz + 2 * self.pml)


def make_workload(name: str, seed: int = 0, *, n_maps: int | None = None, nt: int | None = None,
                  n_tx: int | None = None, nx: int | None = None, nz: int | None = None,
                  n_elem: int | None = None, fd_order: int = 8) -> Workload:
    """Named workloads (sizes overridable for small test cases).

    ``linear_disk``: 128 x 128, 2000 steps, 32 elements, 1 transmit (the centre element), all
    receive; one disk map; the gradient is taken at the homogeneous 1540 m/s map.
    ``full_shot_set``: 512 x 512, 6000 steps, 128 elements, 16 evenly spaced transmits, all
    receive; ``grf_rods`` maps.
    ``scale``: 1024 x 1024, 12000 steps, 128 elements, 64 transmits, up to 8 rods.
    """
    rng = rng_for(seed)
    dx, dt, f0 = 1e-4, 1e-8, 2e6
    if name == "linear_disk":
        nx_, nz_, nt_, ne, ntx, B, kind = 128, 128, 2000, 32, 1, 1, "disk"
    elif name == "full_shot_set":
        nx_, nz_, nt_, ne, ntx, B, kind = 512, 512, 6000, 128, 16, 1, "grf_rods"
    elif name == "scale":
        nx_, nz_, nt_, ne, ntx, B, kind = 1024, 1024, 12000, 128, 64, 1, "grf_rods8"
    else:
        raise ValueError("unknown workload %r" % name)
    nx_ = nx if nx is not None else nx_
    nz_ = nz if nz is not None else nz_
    nt_ = nt if nt is not None else nt_
    ne = n_elem if n_elem is not None else ne
    ntx = n_tx if n_tx is not None else ntx
    B = n_maps if n_maps is not None else B
    maps = []
    for _ in range(B):
        if kind == "disk":
            maps.append(disk_map(rng, nx_, nz_, dx))
        elif kind == "grf_rods":
            maps.append(grf_rods_map(rng, nx_, nz_, dx, max_rods=4))
        else:
            maps.append(grf_rods_map(rng, nx_, nz_, dx, max_rods=8))
    sos_true = np.stack(maps)
    sos_start = np.full_like(sos_true, BACKGROUND_SOS)
    elem_ix, elem_iz = linear_array(nx_, ne)
    if ntx == 1:
        tx = np.array([ne // 2], dtype=np.int32)
    else:
        tx = evenly_spaced_transmits(ne, ntx)
    rx = np.tile(np.arange(ne, dtype=np.int32), (ntx, 1))
    return Workload(name=name, nx=nx_, nz=nz_, dx=dx, dt=dt, nt=nt_, sos_true=sos_true,
                    sos_start=sos_start, wavelet=ricker(nt_, dt, f0), elem_ix=elem_ix,
                    elem_iz=elem_iz, tx_elem=tx, rx_elem=rx, fd_order=fd_order,
                    meta={"seed": seed, "f0": f0, "kind": kind})


def phantom_rods_map(rng, n: int, dx: float, ring_radius_cells: float, max_rods: int = 3,
                     diameter_m: float = 1e-2, sos_choices=(2700.0, 1588.0),
                     background: float = WATER_SOS) -> np.ndarray:
    """1..max_rods non-overlapping hard rods (each bone or edema SoS) in water, all inside the
    ring with a one-diameter margin (the rod phantom of Sec. VII)."""
    r = 0.5 * diameter_m
    c = (n - 1) / 2.0 * dx
    reach = ring_radius_cells * dx - 2.0 * r           # rod centres stay this far from the centre
    X = np.arange(n) * dx
    sos = np.full((n, n), background, dtype=np.float64)
    n_rods = int(rng.integers(1, max_rods + 1))
    rods: list[tuple[float, float]] = []
    tries = 0
    while len(rods) < n_rods and tries < 1000:
        tries += 1
        rho = reach * math.sqrt(rng.uniform(0.0, 1.0))
        phi = rng.uniform(0.0, 2.0 * math.pi)
        cx, cz = c + rho * math.cos(phi), c + rho * math.sin(phi)
        if any((cx - x) ** 2 + (cz - z) ** 2 < (2.0 * r) ** 2 for x, z in rods):
            continue
        rods.append((cx, cz))
        inside = (X[None, :] - cx) ** 2 + (X[:, None] - cz) ** 2 <= r * r
        sos[inside] = sos_choices[int(rng.integers(0, len(sos_choices)))]
    return sos.astype(np.float32)


def density_map(rng, nx: int, nz: int, dx: float, max_rods: int = 3, background: float = 1000.0,
                amp: float = 50.0, corr_m: float = 2e-3) -> np.ndarray:
    """Density (kg/m^3) for the variable-density operator: water-like background plus a smooth
    Gaussian random field (max |.| = amp), plus 1..max_rods hard rods of density U[1050, 1900]
    (soft tissue to bone), radius U[1, 3] mm clamped to small grids."""
    f = _gaussian_field(rng, nx, nz, corr_m / math.sqrt(2.0) / dx)
    f *= amp / max(np.max(np.abs(f)), 1e-30)
    rho = background + f
    X = np.arange(nx) * dx
    Z = np.arange(nz) * dx
    for _ in range(int(rng.integers(1, max_rods + 1))):
        r = rng.uniform(1e-3, max(1e-3, min(3e-3, 0.3 * (min(nx, nz) - 1) * dx)))
        cx = rng.uniform(r, (nx - 1) * dx - r)
        cz = rng.uniform(r, (nz - 1) * dx - r)
        rho[(X[None, :] - cx) ** 2 + (Z[:, None] - cz) ** 2 <= r * r] = rng.uniform(1050.0, 1900.0)
    return rho.astype(np.float32)


def add_awgn(rng, cd: np.ndarray, snr_db: float) -> np.ndarray:
    """Channel data plus white Gaussian noise at the given SNR, with the signal power taken over
    all channels and samples of each map (axis 0 indexes maps)."""
    cd = np.asarray(cd, dtype=np.float64)
    p = np.mean(cd.reshape(cd.shape[0], -1) ** 2, axis=1)
    sigma = np.sqrt(p / 10.0 ** (snr_db / 10.0))
    noise = rng.standard_normal(cd.shape) * sigma.reshape((-1,) + (1,) * (cd.ndim - 1))
    return (cd + noise).astype(np.float32)


def ring_phantom(seed: int = 0, n_maps: int = 1, *, n: int = 188, nt: int = 1034, n_elem: int = 16,
                 f0: float = 350e3, dt: float = 90.243e-9, width_m: float = 0.1, fd_order: int = 8,
                 rod_diameter_m: float = 1e-2) -> Workload:
    """The paper's hardware geometry with rod-phantom maps (Sec. IV, Sec. VII). Element j
    transmits; elements j + n_elem/2 - 1, j + n_elem/2, j + n_elem/2 + 1 (mod n_elem) receive.
    The gradient is taken at homogeneous water. The absorbing-layer reference speed is 1500 m/s,
    which reproduces the printed d0 = 1.46e6 /s at this grid."""
    rng = rng_for(seed)
    dx = width_m / n
    radius = (n - 1) / 2.0
    sos_true = np.stack([phantom_rods_map(rng, n, dx, radius, diameter_m=rod_diameter_m) for _ in range(n_maps)])
    elem_ix, elem_iz = ring_array(n, n_elem, radius)
    tx = np.arange(n_elem, dtype=np.int32)
    h = n_elem // 2
    rx = np.stack([(j + h + np.array([-1, 0, 1])) % n_elem for j in range(n_elem)]).astype(np.int32)
    return Workload(name="ring_phantom", nx=n, nz=n, dx=dx, dt=dt, nt=nt, sos_true=sos_true,
                    sos_start=np.full_like(sos_true, WATER_SOS), wavelet=gaussian_derivative_pulse(nt, dt, f0),
                    elem_ix=elem_ix, elem_iz=elem_iz, tx_elem=tx, rx_elem=rx, pml_cref=WATER_SOS,
                    fd_order=fd_order, c_max=2700.0, meta={"seed": seed, "f0": f0, "kind": "phantom_rods"})


def sized_batch(seed: int, sizes, nt: int, n_elem: int, n_tx: int, dx: float = 1e-4, dt: float = 1e-8,
                f0: float = 2e6, kind: str = "disk"):
    """Maps of different physical grids (nx_b, nz_b) embedded in the envelope (max nx, max nz).

    One shared linear array, centred on the smallest map so that every element lies inside every
    map. Returns (Workload with envelope sizes and embedded maps, list of sizes)."""
    rng = rng_for(seed)
    NX = max(s[0] for s in sizes)
    NZ = max(s[1] for s in sizes)
    B = len(sizes)
    true = np.full((B, NZ, NX), BACKGROUND_SOS, dtype=np.float32)
    for b, (nx, nz) in enumerate(sizes):
        m = disk_map(rng, nx, nz, dx) if kind == "disk" else grf_rods_map(rng, nx, nz, dx, max_rods=4)
        true[b, :nz, :nx] = m
    start = np.full_like(true, BACKGROUND_SOS)
    nx_min = min(s[0] for s in sizes)
    elem_ix, elem_iz = linear_array(nx_min, n_elem)
    tx = np.array([n_elem // 2], dtype=np.int32) if n_tx == 1 else evenly_spaced_transmits(n_elem, n_tx)
    rx = np.tile(np.arange(n_elem, dtype=np.int32), (tx.size, 1))
    wl = Workload(name="sized", nx=NX, nz=NZ, dx=dx, dt=dt, nt=nt, sos_true=true, sos_start=start,
                  wavelet=ricker(nt, dt, f0), elem_ix=elem_ix, elem_iz=elem_iz, tx_elem=tx, rx_elem=rx,
                  meta={"seed": seed, "sizes": [tuple(s) for s in sizes]})
    return wl, [tuple(s) for s in sizes]


UNEVEN_GRIDS = ((384, 384), (512, 512), (640, 512))


def uneven_batch(seed: int = 0, n_maps: int = 32, n_tx: int = 16, nt: int = 6000, n_elem: int = 128):
    """Batching workload: n_maps disk maps (the linear-disk distribution), each on a grid drawn
    from 384 x 384, 512 x 512 and 640 x 512 (nx x nz), with a 128-element array and n_tx evenly
    spaced transmits shared by all maps."""
    rng = rng_for(seed + 1000)
    sizes = [UNEVEN_GRIDS[int(rng.integers(0, len(UNEVEN_GRIDS)))] for _ in range(n_maps)]
    wl, sizes = sized_batch(seed, sizes, nt, n_elem, n_tx)
    wl.name = "uneven_batch"
    return wl, sizes
