"""The float64 ranker reference against central finite differences (CPU)."""
import numpy as np

from tests import ranker_ref


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(61)
    P = ranker_ref.n_params()
    assert P == 51136
    w = rng.normal(0, 0.15, P)
    x = rng.random((9, 76))
    y = rng.integers(0, 64, 9)
    _, g = ranker_ref.loss_and_grad(w, x, y)
    eps = 1e-6
    # coordinates in every weight block and every bias block
    starts = [0, 9728, 9856, 26240, 26368, 42752, 42880, 51072]
    for s in starts:
        for k in rng.integers(0, 60, 3):
            i = s + int(k)
            e = np.zeros(P)
            e[i] = eps
            fd = (ranker_ref.loss_only(w + e, x, y) - ranker_ref.loss_only(w - e, x, y)) / (2 * eps)
            assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_reference_loss_of_uniform_logits():
    """Zero output layer: every logit equal, loss = log 64 exactly."""
    P = ranker_ref.n_params()
    w = np.zeros(P)
    rng = np.random.default_rng(62)
    loss, g = ranker_ref.loss_and_grad(w, rng.random((5, 76)), rng.integers(0, 64, 5))
    assert abs(loss - np.log(64)) < 1e-12
