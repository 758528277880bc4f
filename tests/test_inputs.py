"""The seeded input generator: deterministic, standard-normal, independent streams."""
import numpy as np

from paper_2211_09815_gb300 import inputs


def test_white_noise_is_deterministic_and_standard_normal():
    a = inputs.white_noise(32, 7)
    b = inputs.white_noise(32, 7)
    assert a.dtype == np.float32 and a.shape == (32, 32, 32)
    assert np.array_equal(a, b)
    assert abs(a.mean()) < 5 / np.sqrt(a.size)
    assert abs(a.std() - 1) < 5 / np.sqrt(a.size)
    c = inputs.white_noise(32, 8)
    assert abs(np.corrcoef(a.ravel(), c.ravel())[0, 1]) < 5 / np.sqrt(a.size)


def test_white_noise_chunking_does_not_change_values():
    a = inputs.white_noise(16, 3)
    b = inputs.white_noise(16, 3, chunk=100)
    assert np.array_equal(a, b)


def test_ensemble_theta_ranges():
    th = inputs.ensemble_theta(16)
    assert th.shape == (16, 5)
    assert np.all((th[:, 2] >= 0.25) & (th[:, 2] <= 0.35))
    assert np.all((th[:, 0] >= 1.8e-9) & (th[:, 0] <= 2.4e-9))
    assert np.all((th[:, 1] >= 0.94) & (th[:, 1] <= 0.99))
