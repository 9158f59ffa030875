"""Pins for the CPU oracle of the learned price predictor (no GPU).

The backward pass is checked against central finite differences of the
loss, which depend only on the forward pass; the loss's blindness to a
shift of all outputs (prices are defined up to a constant) is checked
through the bias of the last layer; features are checked on a matrix
worked by hand.
"""

import numpy as np
import pytest

from oracle import set_encoder as se


def _problem(seed, sizes=(4, 7, 5)):
    rng = np.random.default_rng(seed)
    P = se.init_params(seed)
    # perturb biases so that no ReLU sits exactly at zero
    P[se.OFF_B1:se.OFF_W2] += rng.normal(0, 0.1, se.H)
    P[se.OFF_B2:se.OFF_W3] += rng.normal(0, 0.1, se.H)
    seg = np.concatenate([[0], np.cumsum(sizes)])
    N = seg[-1]
    X = np.zeros((N, se.F))
    X[:, :se.NF] = rng.normal(0, 1, (N, se.NF))
    t = rng.normal(0, 1, N)
    return P, X, t, seg


def test_features_hand_worked():
    C = np.array([[5, 1, 4], [3, 6, 0], [2, 7, 8]])
    X, T = se.features(C)
    # column minima a = (2,1,0), second minima b = (3,6,4), gaps (1,5,4)
    assert T == pytest.approx(1 + 10 / 3)
    np.testing.assert_allclose(X[:, 0], (np.array([2, 1, 0]) - 1) / T)
    np.testing.assert_allclose(X[:, 1], np.array([1, 5, 4]) / T)
    # row minima (1,0,2); C - u = [[4,0,3],[3,6,0],[0,5,6]]: q = (0,0,0), q2 = (3,5,3)
    np.testing.assert_allclose(X[:, 2], 0.0)
    np.testing.assert_allclose(X[:, 3], np.array([3, 5, 3]) / T)
    # each column is the minimum of exactly one row
    np.testing.assert_allclose(X[:, 4], np.log(2.0))
    m = np.array([10, 14, 12]) / 3
    sd = np.sqrt(np.mean((m - m.mean()) ** 2)) + 1
    np.testing.assert_allclose(X[:, 5], (m - m.mean()) / sd)
    np.testing.assert_allclose(X[:, 6], np.log(T) / 10)
    np.testing.assert_allclose(X[:, 7], np.log(3) / 10)
    assert np.all(X[:, 8:] == 0)


def test_features_single_column():
    X, T = se.features(np.array([[7]]))
    assert T == 1.0 and np.all(X[:, :4] == 0) and X[0, 4] == pytest.approx(np.log(2))


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(seed):
    P, X, t, seg = _problem(seed)
    L, g = se.loss_grad(P, X, t, seg)
    assert L == pytest.approx(se.loss(P, X, t, seg))
    rng = np.random.default_rng(100 + seed)
    blocks = [(se.OFF_W1, se.OFF_W1 + se.NF * se.H), (se.OFF_B1, se.OFF_W2), (se.OFF_W2, se.OFF_B2),
              (se.OFF_B2, se.OFF_W3)]
    idx = np.concatenate([rng.integers(a, b, 40) for a, b in blocks] +
                         [np.arange(se.OFF_W3, se.OFF_B3, 8)[:40], [se.OFF_B3]])
    h = 1e-6
    for k in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[k] += h
        Pm[k] -= h
        fd = (se.loss(Pp, X, t, seg) - se.loss(Pm, X, t, seg)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-5 * max(abs(fd), abs(g[k])), (k, fd, g[k])


def test_loss_blind_to_output_shift():
    P, X, t, seg = _problem(3)
    L, g = se.loss_grad(P, X, t, seg)
    Q = P.copy()
    Q[se.OFF_B3] += 5.0                     # shifts every y by 5
    assert se.loss(Q, X, t, seg) == pytest.approx(L)
    assert abs(g[se.OFF_B3]) < 1e-12        # so its gradient vanishes
    assert se.loss(P, X, t + 3.0, seg) == pytest.approx(L)


def test_bf16_rounding():
    assert se.bf16(1.0) == 1.0
    assert se.bf16(1 + 2 ** -8) == 1.0                   # tie goes to even
    assert se.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6        # tie goes to even (up)
    assert se.bf16(1 + 2 ** -8 + 2 ** -12) == 1 + 2 ** -7
    assert se.bf16(-2.5) == -2.5
    x = np.random.default_rng(0).normal(size=1000)
    assert np.max(np.abs(se.bf16(x) - x) / np.abs(x)) <= 2 ** -8
