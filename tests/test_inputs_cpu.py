"""Properties of the seeded synthetic stack inputs (CPU only).

The Navier-Stokes-like field must be divergence-free with its energy inside
|k| <= 16 and the target one step ahead; the CO2-like input must carry the
static fields repeated along t, one well column, and a target in (0, 1).
"""
import numpy as np

from paper_2211_12709_gb300 import inputs


def test_ns_velocity_is_divergence_free_and_band_limited():
    x0, target = inputs.ns_stack_inputs(1, (32, 32, 32, 4), 7, kmax=8.0)
    ks = [np.fft.fftfreq(32, 1.0 / 32)] * 3
    K = np.stack(np.meshgrid(*ks, indexing="ij"))
    for t in range(4):
        u = x0[0, 0:3, ..., t].astype(np.float64)
        uh = np.fft.fftn(u, axes=(1, 2, 3))
        div = np.fft.ifftn((1j * K * uh).sum(0)).real
        grad = np.fft.ifftn(1j * K[0] * uh[0]).real
        assert np.abs(div).max() <= 1e-5 * np.abs(grad).max()
        kmag = np.sqrt((K ** 2).sum(0))
        e = (np.abs(uh) ** 2).sum(0)
        assert e[kmag > 8.5].sum() <= 1e-10 * e.sum()
    # |omega| is non-negative before standardisation: its minimum sits below the mean
    assert x0[0, 3].min() < 0 < x0[0, 3].max()
    assert np.array_equal(target[..., :-1], x0[..., 1:])
    assert np.array_equal(target[..., -1], x0[..., 0])
    np.testing.assert_allclose(np.sqrt((x0[:, 0:3].astype(np.float64) ** 2).mean()), 1.0, rtol=1e-5)


def test_co2_inputs_are_static_in_time_with_one_well_column():
    x0, target = inputs.co2_stack_inputs(2, (16, 12, 8, 5), 3)
    assert x0.shape == (2, 3, 16, 12, 8, 5) and target.shape == (2, 1, 16, 12, 8, 5)
    assert np.array_equal(x0[..., 1:], np.repeat(x0[..., :1], 4, axis=-1))
    for b in range(2):
        well = x0[b, 2, ..., 0]
        cols = np.argwhere(well.sum(axis=2) > 0)
        assert len(cols) == 1 and well[tuple(cols[0])].min() == 1.0
        assert set(np.unique(well)) <= {0.0, 1.0}
    assert 0.0 < target.min() and target.max() < 1.0
    phi = x0[:, 1]
    assert phi.min() >= 0.05 and phi.max() <= 0.40
