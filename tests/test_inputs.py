"""The seeded input generators: layout, reproducibility and the C_l variance."""
import numpy as np

from paper_1106_0159_gb300 import inputs


def test_gaussian_alm_layout_and_variance():
    L = 300
    a = inputs.gaussian_alm(L, L, seed=1, nmaps=2)
    assert a.shape == (2, inputs.nalm(L, L))
    l, m = inputs.lm_arrays(L, L)
    assert np.all(a[:, m == 0].imag == 0)
    assert np.array_equal(a, inputs.gaussian_alm(L, L, seed=1, nmaps=2))
    cl = 1.0 / (l * (l + 1.0) + 1.0)
    z = np.abs(a) ** 2 / cl            # E|a|^2 = C_l for every (l, m)
    assert abs(z.mean() - 1.0) < 0.02


def test_uniform_alm_and_white_map():
    a = inputs.uniform_alm(20, 10, seed=2)
    assert a.shape == (1, inputs.nalm(20, 10))
    assert np.all(np.abs(a.real) < 1) and np.all(np.abs(a.imag) < 1)
    s = inputs.white_map(10000, seed=3)
    assert abs(s.std() - 1) < 0.03
