"""The seeded synthetic inputs shared by the oracle's tests and the CUDA path: each generator
follows its stated recipe (workload shapes, value distributions, spectra) and is reproducible
from its seed alone.
"""
import numpy as np
import pytest
import scipy.fft

import inputs


def test_generators_are_reproducible_and_seeded():
    a, b = inputs.gray_scott_2d(n=64, seed=3), inputs.gray_scott_2d(n=64, seed=3)
    np.testing.assert_array_equal(a.u0, b.u0)
    assert not np.array_equal(a.u0, inputs.gray_scott_2d(n=64, seed=4).u0)
    np.testing.assert_array_equal(inputs.adv_diff_1d(seed=2).u0, inputs.adv_diff_1d(seed=2).u0)
    # an ensemble instance depends on its index only, not on the size of the batch
    np.testing.assert_array_equal(inputs.ensemble(7)[5].u0, inputs.ensemble_instance(5).u0)


def test_adv_diff_1d_has_exactly_modes_1_to_8():
    w = inputs.adv_diff_1d()
    assert (w.n, w.dt, w.nsteps, w.order, w.nu, w.a) == (256, 1 / 512, 512, 4, (0.01,), 1.0)
    spec = np.abs(np.fft.rfft(w.u0)) / (w.n / 2)
    amp = np.abs(np.asarray(w.meta["amp"]))
    np.testing.assert_allclose(spec[1:9], amp, atol=1e-12)
    assert spec[0] < 1e-12 and spec[9:].max() < 1e-12


def test_paper_workloads_match_section_iv():
    up = inputs.adv_diff_upwind_1d()
    assert (up.n, up.nsteps, up.restart_every, up.a, up.nu) == (1000, 4000, 400, -0.1, (1e-3,))
    assert up.dt * up.nsteps == pytest.approx(40.0)
    np.testing.assert_allclose(up.u0, 2.0 + np.sin(2 * np.pi * np.arange(1000) / 1000))
    bu = inputs.burgers_1d()
    assert (bu.n, bu.nsteps, bu.nu) == (999, 2000, (1e-3,)) and bu.dt * bu.nsteps == pytest.approx(1)
    x = np.arange(1, 1000) / 1000
    np.testing.assert_allclose(bu.u0, np.sin(2 * np.pi * x) + 0.5 * np.sin(np.pi * x))


@pytest.mark.parametrize("seed", [0, 1, 7])
def test_gray_scott_square_and_noise(seed):
    n, width = 256, 0.1
    w = inputs.gray_scott_2d(n=n, seed=seed, width=width)
    assert w.species == 2 and (w.F, w.k, w.nu, w.dt) == (0.04, 0.06, (2e-5, 1e-5), 0.5)
    u, v = w.u0
    inside = v > 0.1
    # the square: (u, v) = (0.5, 0.25) on the cells whose centres lie in it, (1, 0) elsewhere,
    # each value times 1 + 0.01 U[-1, 1]
    assert np.all(np.abs(u[inside] / 0.5 - 1) <= 0.01 + 1e-15)
    assert np.all(np.abs(v[inside] / 0.25 - 1) <= 0.01 + 1e-15)
    assert np.all(np.abs(u[~inside] - 1) <= 0.01 + 1e-15) and not np.any(v[~inside])
    rows, cols = np.nonzero(inside)
    side = round(width * n)
    assert abs(np.ptp(rows) + 1 - side) <= 1 and abs(np.ptp(cols) + 1 - side) <= 1
    assert inside.sum() == (np.ptp(rows) + 1) * (np.ptp(cols) + 1)       # one full rectangle
    assert 0 < rows.min() and rows.max() < n - 1 and 0 < cols.min() and cols.max() < n - 1
    noise = np.concatenate([u[~inside] - 1, u[inside] / 0.5 - 1])
    assert noise.min() < -0.009 and noise.max() > 0.009                  # spans U[-1, 1]


def test_dirichlet_field_is_low_mode():
    """kx, ky <= kmax with coefficients N(0,1) / (kx^2 + ky^2): the DST-II of the field on the
    cell centres has no energy above kmax."""
    n, kmax = 64, 16
    w = inputs.adv_diff_2d(n=n, kmax=kmax)
    assert (w.a, w.b, w.nu, w.dt) == (1.0, 1.0, (1e-3,), 1 / n)
    c = scipy.fft.dstn(w.u0[0], type=2, norm="ortho")
    energy = (c ** 2).sum()
    assert (c[kmax:, :] ** 2).sum() < 1e-24 * energy and (c[:, kmax:] ** 2).sum() < 1e-24 * energy


def test_ensemble_parameters_follow_the_recipe():
    ws = inputs.ensemble(512)
    sides = {w.n for w in ws}
    assert sides == set(inputs.ENSEMBLE_SIDES)
    assert {w.order for w in ws} == {2, 3, 4}
    for w in ws:
        assert w.dt == 1.0 / (4 * w.n) and w.nsteps == 256
        assert 1e-4 <= w.nu[0] <= 1e-2 and -1 <= w.a <= 1 and -1 <= w.b <= 1
        assert w.u0.shape == (1, w.n, w.n)
    # logU[1e-4, 1e-2]: the log10 of nu is uniform, so about half the draws lie below 1e-3
    below = np.mean([w.nu[0] < 1e-3 for w in ws])
    assert 0.4 < below < 0.6
