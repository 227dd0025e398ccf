"""Pins of the oracle's CMA-ES update variant (the evolution strategy Algorithm 1 is modelled
on): the behaviour the method's definition fixes, not its formulas retyped.

- Under neutral selection (costs independent of the samples) the update is unbiased: the
  expected new covariance is the old one, the step-size path keeps the length of a
  standard normal vector, and the step size does not drift. Each fails for a covariance
  taken about the new mean, a wrong path normalisation or a path not whitened by C.
- On a linear function the step size grows geometrically; on the sphere the mean
  converges linearly to the optimum; on a rotated ill-conditioned ellipsoid the
  covariance learns the inverse Hessian up to scale.
- The mean is the paper's weighted mean of the same elites.
"""
import math

import numpy as np
import pytest

from helpers import ROOT  # noqa: F401  (puts the oracle on sys.path)


@pytest.fixture(scope="module")
def oracle():
    import oracle as o
    return o


def _sample(st, n, g):
    L = np.linalg.cholesky(st.C)
    return st.mu[None, :] + st.sigma * g.standard_normal((n, st.mu.shape[0])) @ L.T


def _run(oracle, f, D, N, T, sigma0, seed, mu0=None):
    g = np.random.default_rng(seed)
    st = oracle.cma_init(np.zeros(D) if mu0 is None else mu0, np.eye(D), sigma0)
    for _ in range(T):
        X = _sample(st, N, g)
        st = oracle.update_cmaes(st, X, f(X), N // 2)
    return st


def test_neutral_selection_is_unbiased(oracle):
    D, N, M = 6, 24, 8000
    g = np.random.default_rng(0)
    A = g.standard_normal((D, D))
    C = A @ A.T / D + 0.5 * np.eye(D)
    nu = N // 2
    k = oracle.cma_constants(D, oracle.log_rank_weights(nu))
    Lc = np.linalg.cholesky(C)
    sigma = 0.7
    acc_C = np.zeros((D, D))
    acc_ps2, acc_logs = 0.0, 0.0
    for _ in range(M):
        # paths drawn from their stationary laws under neutral selection
        st = oracle.CMAState(np.zeros(D), C.copy(), sigma, g.standard_normal(D),
                             Lc @ g.standard_normal(D), 100)
        X = _sample(st, N, g)
        new = oracle.update_cmaes(st, X, g.random(N), nu)
        acc_C += new.C
        acc_ps2 += float(new.p_sigma @ new.p_sigma)
        acc_logs += math.log(new.sigma / sigma)
    scale = np.sqrt(np.outer(np.diag(C), np.diag(C)))
    # statistical error of the mean over M trials is ~1.5e-3 of the scale; a covariance
    # about the new mean is biased low by c_mu / mu_eff (2% here)
    assert k.c_mu / k.mu_eff > 0.015
    np.testing.assert_array_less(np.abs(acc_C / M - C) / scale, 6e-3)
    assert acc_ps2 / M == pytest.approx(D, rel=0.03)
    assert abs(acc_logs / M) < 3e-3


def test_linear_function_grows_the_step_size(oracle):
    st = _run(oracle, lambda X: X[:, 0], D=6, N=24, T=40, sigma0=1.0, seed=1)
    assert st.sigma > 10.0
    assert st.mu[0] < -10.0


def test_sphere_converges(oracle):
    target = np.ones(6)
    st = _run(oracle, lambda X: np.sum((X - target) ** 2, axis=1), D=6, N=24, T=250, sigma0=0.5, seed=2)
    assert np.sum((st.mu - target) ** 2) < 1e-12
    assert st.sigma < 1e-4


def test_covariance_learns_a_rotated_ellipsoid(oracle):
    D = 5
    g = np.random.default_rng(3)
    R, _ = np.linalg.qr(g.standard_normal((D, D)))
    a = 10.0 ** (4.0 * np.arange(D) / (D - 1))
    H = R.T @ np.diag(a) @ R

    def f(X):
        return np.einsum("ni,ij,nj->n", X, H, X)

    st = _run(oracle, f, D=D, N=20, T=700, sigma0=0.3, seed=4, mu0=np.ones(D))
    # C^1/2 H C^1/2 is a multiple of the identity when C = c H^-1
    Lc = np.linalg.cholesky(st.C)
    ev = np.linalg.eigvalsh(Lc.T @ H @ Lc)
    assert ev.max() / ev.min() < 5.0, ev.max() / ev.min()
    assert np.linalg.cond(H) == pytest.approx(1e4, rel=1e-6)


def test_mean_is_the_paper_weighted_mean(oracle):
    g = np.random.default_rng(5)
    D, N = 8, 40
    X = g.standard_normal((N, D))
    J = g.random(N)
    st = oracle.cma_init(np.zeros(D), np.eye(D), 1.0)
    mu_paper, _ = oracle.update(X, J, N // 2, 0.0)
    np.testing.assert_allclose(oracle.update_cmaes(st, X, J, N // 2).mu, mu_paper, rtol=0, atol=1e-15)


def test_rank_mu_term_is_the_weighted_scatter_about_the_old_mean(oracle):
    """The rank-mu matrix sum_j w_j y_j y_j^T about the old mean m equals the weighted
    covariance about the new mean (numpy's weighted covariance) plus (m' - m)(m' - m)^T,
    since the weights sum to one; the rest of C' is rebuilt from the returned paths."""
    g = np.random.default_rng(6)
    D, N = 7, 30
    A = g.standard_normal((D, D))
    C = A @ A.T / D + 0.3 * np.eye(D)
    st = oracle.CMAState(g.standard_normal(D), C, 0.8, g.standard_normal(D), g.standard_normal(D), 3)
    X = _sample(st, N, g)
    J = np.sum(X ** 2, axis=1)
    nu = N // 2
    new = oracle.update_cmaes(st, X, J, nu)
    w = oracle.log_rank_weights(nu)
    elites = X[np.argsort(J, kind="stable")[:nu]]
    d = new.mu - st.mu
    scatter = (np.cov(elites.T, aweights=w, bias=True) + np.outer(d, d)) / st.sigma ** 2
    k = oracle.cma_constants(D, w)
    h = 1.0 if np.linalg.norm(new.p_sigma) / math.sqrt(1 - (1 - k.c_sigma) ** (2 * (st.t + 1))) \
        < (1.4 + 2 / (D + 1)) * k.chi_n else 0.0
    a = 1 + k.c_1 * (1 - h) * k.c_c * (2 - k.c_c) - k.c_1 - k.c_mu
    want = a * C + k.c_1 * np.outer(new.p_c, new.p_c) + k.c_mu * scatter
    np.testing.assert_allclose(new.C, want, rtol=1e-12, atol=1e-14)
