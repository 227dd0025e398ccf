"""Pins of the oracle's factor-free sampler (step (1) drawn from the last update's elites):
its samples have the mean and the covariance sigma^2 C of the paper's update (steps (5)-(6),
itself pinned against numpy's weighted covariance) within the statistical error, a
projection is standard normal, and with one elite (the mean itself) only the eps term is
left, in closed form."""
import math

import numpy as np
import pytest
from scipy import stats

from helpers import ROOT  # noqa: F401  (puts the oracle on sys.path)


@pytest.fixture(scope="module")
def oracle():
    import oracle as o
    return o


def _elites(D, nu, seed):
    g = np.random.default_rng(seed)
    X = g.normal(size=(2 * nu, D)) * np.linspace(0.5, 2.0, D) + 0.3
    J = g.random(2 * nu)
    return X, J


def test_mean_and_covariance_are_the_update(oracle):
    K, nu, N = 2, 16, 200_000
    D = 4 * K
    X, J = _elites(D, nu, 1)
    mu, C = oracle.update(X, J, nu, 1e-3)
    order = oracle.rank(J)
    w = oracle.log_rank_weights(nu)
    xi = oracle.sample_elites(mu, X[order[:nu]], w, 0.7, 1e-3, seed=3, t=5, query=1, N=N, K=K).reshape(N, D)
    want = 0.49 * C
    got = np.cov(xi.T, bias=True)
    sd = np.sqrt(np.outer(np.diag(want), np.diag(want)))
    # standard error of a covariance entry over N samples is about sd sqrt(2 / N) = 3e-3 sd
    np.testing.assert_array_less(np.abs(got - want) / sd, 0.015)
    np.testing.assert_array_less(np.abs(xi.mean(axis=0) - mu) / np.sqrt(np.diag(want)), 0.012)


def test_projection_is_standard_normal(oracle):
    K, nu, N = 3, 24, 20_000
    D = 4 * K
    X, J = _elites(D, nu, 2)
    mu, C = oracle.update(X, J, nu, 1e-4)
    order = oracle.rank(J)
    xi = oracle.sample_elites(mu, X[order[:nu]], oracle.log_rank_weights(nu), 1.3, 1e-4, seed=9, t=0,
                              query=0, N=N, K=K).reshape(N, D)
    u = np.random.default_rng(4).normal(size=D)
    s = (xi - mu) @ u / math.sqrt(1.69 * u @ C @ u)
    assert stats.kstest(s, "norm").pvalue > 1e-3


def test_single_elite_leaves_the_eps_term(oracle):
    K, N = 2, 50
    D = 4 * K
    x = np.random.default_rng(5).normal(size=(1, D))
    mu = x[0]
    xi = oracle.sample_elites(mu, x, np.ones(1), 0.5, 1e-6, seed=11, t=2, query=0, N=N, K=K).reshape(N, D)
    z = oracle.normals(11, 2, 0, N, (1 + D + 3) // 4)
    np.testing.assert_allclose(xi, mu[None, :] + 0.5 * 1e-3 * z[:, 1:1 + D], rtol=0, atol=1e-15)
