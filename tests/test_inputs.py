"""The seeded input generators (no GPU): each workload follows the recipe stated for it (grid,
time axis, array, transmits, map statistics), and equal seeds give equal inputs. The generators
hold none of the method's arithmetic; both the oracle and the CUDA path read their output."""
import math

import numpy as np
import pytest

from paper_2603_04070_gb300 import inputs


def test_linear_disk_recipe():
    """128 x 128 at 0.1 mm and 10 ns, 2000 steps; 32 elements 3 cells apart on row 0, centred
    (first element at x = 17); the centre element transmits and all receive; one hard disk of
    radius 1.5-3 mm and 1450-1520 m/s in 1540 m/s; the gradient is taken at 1540 m/s."""
    for seed in range(10):
        wl = inputs.make_workload("linear_disk", seed=seed)
        assert (wl.nx, wl.nz, wl.nt, wl.dx, wl.dt) == (128, 128, 2000, 1e-4, 1e-8)
        assert wl.elem_ix[0] == 17 and np.all(np.diff(wl.elem_ix) == 3) and np.all(wl.elem_iz == 0)
        assert wl.tx_elem.tolist() == [16] and wl.rx_elem.tolist() == [list(range(32))]
        m = wl.sos_true[0]
        vals = np.unique(m)
        assert vals.size == 2 and vals.max() == 1540.0 and 1450.0 <= vals.min() <= 1520.0
        n_in = int((m != 1540.0).sum())
        r_eq = math.sqrt(n_in / math.pi) * wl.dx                   # radius of the equal-area disk
        assert 1.5e-3 - wl.dx <= r_eq <= 3e-3 + wl.dx
        assert np.all(wl.sos_start == 1540.0)


def test_full_shot_set_recipe():
    """512 x 512, 6000 steps; 128 elements; transmits floor((j + 0.5) 128 / 16) = 4, 12, ...,
    124; all 128 receive; 1540 m/s plus a smooth field of max |.| = 20 m/s plus 1-4 rods of
    1450-1600 m/s."""
    wl = inputs.make_workload("full_shot_set", seed=0)
    assert (wl.nx, wl.nz, wl.nt) == (512, 512, 6000)
    assert wl.tx_elem.tolist() == list(range(4, 128, 8))
    assert wl.rx_elem.shape == (16, 128)
    m = wl.sos_true[0].astype(np.float64)
    smooth = np.abs(m - 1540.0) <= 20.0 + 1e-3
    assert smooth.mean() > 0.8                                     # most cells: background + field
    assert abs(m[smooth] - 1540.0).max() > 15.0                    # the field reaches near its bound
    rods = m[~smooth]
    assert rods.size == 0 or (rods.min() >= 1450.0 and rods.max() <= 1600.0)


def test_gaussian_field_correlation_length():
    """The smooth field is white noise filtered by a Gaussian of sigma = 3 mm / sqrt(2), so its
    autocorrelation is Gaussian with a 3 mm length: rho(3 mm) = exp(-1/2) = 0.61 and
    rho(6 mm) = exp(-2) = 0.14 (the field is periodic, so the circular estimate is exact in
    expectation)."""
    dx = 1e-4
    acc = {30: [], 60: []}
    for seed in range(4):
        f = inputs._gaussian_field(inputs.rng_for(seed), 512, 512, 3e-3 / math.sqrt(2.0) / dx)
        f = f - f.mean()
        v = np.mean(f * f)
        for lag in acc:
            acc[lag].append(0.5 * (np.mean(f * np.roll(f, lag, axis=1)) + np.mean(f * np.roll(f, lag, axis=0))) / v)
    assert np.mean(acc[30]) == pytest.approx(math.exp(-0.5), abs=0.05)
    assert np.mean(acc[60]) == pytest.approx(math.exp(-2.0), abs=0.05)


def test_density_map_recipe():
    """1000 kg/m^3 plus a smooth field of max |.| = 50, plus 1-3 rods of 1050-1900 kg/m^3."""
    rng = inputs.rng_for(7)
    for _ in range(5):
        rho = inputs.density_map(rng, 200, 160, 1e-4).astype(np.float64)
        assert rho.shape == (160, 200)
        smooth = np.abs(rho - 1000.0) <= 50.0 + 1e-3
        assert smooth.mean() > 0.7
        rods = rho[~smooth]
        assert rods.size > 0 and rods.min() >= 1050.0 - 1e-3 and rods.max() <= 1900.0 + 1e-3


def test_ricker_pulse():
    """w(t) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2), tau = t - 1.5/f0: peak 1 at the delay,
    zeros at tau = +-1/(sqrt(2) pi f0)."""
    f0, dt = 2e6, 1e-9
    w = inputs.ricker(2000, dt, f0).astype(np.float64)
    assert int(np.argmax(w)) == round(1.5 / f0 / dt) and w.max() == pytest.approx(1.0, abs=1e-6)
    z = 1.5 / f0 + 1.0 / (math.sqrt(2.0) * math.pi * f0)
    i = int(z / dt)
    assert w[i] * w[i + 1] <= 0.0


def test_uneven_batch_recipe():
    """32 maps, each on a grid drawn from 384 x 384, 512 x 512 and 640 x 512, embedded in the
    640 x 512 envelope; the shared array is centred on the smallest grid; 16 transmits x 128."""
    wl, sizes = inputs.uneven_batch(seed=0, nt=10)
    assert len(sizes) == 32 and set(sizes) <= set(inputs.UNEVEN_GRIDS) and len(set(sizes)) == 3
    assert (wl.nx, wl.nz) == (640, 512) and wl.n_tx == 16 and wl.n_rx == 128
    assert wl.elem_ix.max() < 384
    for b, (nx, nz) in enumerate(sizes):
        assert np.all(wl.sos_true[b, nz:, :] == 1540.0) and np.all(wl.sos_true[b, :, nx:] == 1540.0)


def test_equal_seeds_give_equal_inputs():
    a = inputs.make_workload("full_shot_set", seed=3, nx=96, nz=80, nt=50, n_elem=16, n_tx=2)
    b = inputs.make_workload("full_shot_set", seed=3, nx=96, nz=80, nt=50, n_elem=16, n_tx=2)
    c = inputs.make_workload("full_shot_set", seed=4, nx=96, nz=80, nt=50, n_elem=16, n_tx=2)
    assert np.array_equal(a.sos_true, b.sos_true) and np.array_equal(a.wavelet, b.wavelet)
    assert not np.array_equal(a.sos_true, c.sos_true)
    r1 = inputs.ring_phantom(seed=2, n_maps=2)
    r2 = inputs.ring_phantom(seed=2, n_maps=2)
    assert np.array_equal(r1.sos_true, r2.sos_true)
