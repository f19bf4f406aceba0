"""pc_cv_labels (the control variate's training labels, in the library):
value and central-difference hedge ratios from prices at spots bumped by
+-h per underlying.  A central difference is exact for prices that are
quadratic in the bumped spot, so the labels of such price functions equal
their derivatives; bad arguments are refused."""
import numpy as np
import pytest

import paper_2108_03076_gb300 as pc


def bumped_prices(f, S, h):
    """[2d + 1, n]: f at S, then at S_i (1 + h) and S_i (1 - h) for each i."""
    n, d = S.shape
    rows = [f(S)]
    for i in range(d):
        for s in (1.0, -1.0):
            Sb = S.copy()
            Sb[:, i] *= 1.0 + s * h
            rows.append(f(Sb))
    return np.stack(rows)


@pytest.mark.parametrize("d", [1, 3, 4])
def test_labels_of_quadratic_prices_are_their_gradients(d):
    rng = np.random.default_rng(d)
    n, h = 257, 0.02
    S = rng.uniform(0.5, 1.5, (n, d))
    a = rng.normal(size=d)
    b = rng.normal(size=d)

    def f(X):
        return 0.3 + X @ a + (X ** 2) @ b + X[:, 0] * X[:, -1] * 0.25 * (d > 1)

    grad = a[None, :] + 2.0 * b[None, :] * S
    if d > 1:
        grad[:, 0] += 0.25 * S[:, -1]
        grad[:, -1] += 0.25 * S[:, 0]
    y = pc.pc_cv_labels(bumped_prices(f, S, h), S, h, 6)
    assert y.shape == (n, 6) and y.dtype == np.float32
    np.testing.assert_allclose(y[:, 0], f(S), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(y[:, 1:1 + d], grad, rtol=2e-5, atol=2e-5)
    assert np.all(y[:, 1 + d:] == 0.0)


def test_labels_refuse_bad_arguments():
    S = np.ones((4, 2))
    p = np.zeros((5, 4))
    with pytest.raises(pc.PcError):
        pc.pc_cv_labels(p, S, 0.0, 5)          # bump must be positive
    with pytest.raises(pc.PcError):
        pc.pc_cv_labels(p, S, 0.01, 2)         # width below 1 + d
    with pytest.raises(pc.PcError):
        pc.pc_cv_labels(np.zeros((11, 4)), np.ones((4, 5)), 0.01, 8)   # d above 4
    with pytest.raises(ValueError):
        pc.pc_cv_labels(np.zeros((3, 4)), S, 0.01, 5)   # prices for d = 1, spots for d = 2
