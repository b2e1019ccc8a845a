"""Pins of the oracle's block Metropolis-Hastings driver (App. D) on log-densities with known
answers: acceptance of everything when log u = -inf (the chain is the running sum of the
proposals), greedy behaviour when u = 1, the prior's support, fixed components, and the moments
of a long chain on a Gaussian target (stationary distribution)."""
import math

import numpy as np


def test_mcmc_accepts_all_with_zero_uniforms(orc):
    rng = np.random.default_rng(1)
    P, T = 4, 30
    normals = rng.normal(size=(T, P))
    block = np.array([0, 0, 1, -1])
    step = np.array([0.1, 0.2, 0.3, 0.4])
    chain, acc = orc.mcmc(lambda th: -float(th @ th), np.zeros(P), block, step, -np.inf, np.inf, normals,
                          np.zeros((T, 2)))
    assert acc.all()
    expect = np.cumsum(normals * step * (block >= 0), axis=0)
    np.testing.assert_allclose(chain[:, :P], expect, rtol=0, atol=1e-15)
    assert np.all(chain[:, 3] == 0.0)
    np.testing.assert_allclose(chain[:, P], -np.sum(expect ** 2, axis=1), rtol=1e-14)


def test_mcmc_greedy_with_unit_uniforms_and_bounds(orc):
    rng = np.random.default_rng(2)
    T = 200
    f = lambda th: -float(np.sum((th - 0.3) ** 2))  # noqa: E731
    chain, acc = orc.mcmc(f, np.zeros(2), np.array([0, 1]), np.array([0.05, 0.05]), np.array([-1.0, 0.0]),
                          np.array([1.0, 0.25]), rng.normal(size=(T, 2)), np.ones((T, 2)))
    assert np.all(np.diff(chain[:, 2]) >= 0.0)                  # only improvements pass log u = 0
    assert np.all(chain[:, 1] <= 0.25) and np.all(chain[:, 0] >= -1.0)
    assert abs(chain[-1, 0] - 0.3) < 0.05 and chain[-1, 1] > 0.2


def test_mcmc_stationary_moments_of_a_gaussian_target(orc):
    rng = np.random.default_rng(3)
    T = 40000
    mu, sd = 1.5, 0.7
    f = lambda th: -0.5 * ((th[0] - mu) / sd) ** 2  # noqa: E731
    chain, acc = orc.mcmc(f, np.array([mu]), np.array([0]), np.array([1.2]), -np.inf, np.inf,
                          rng.normal(size=(T, 1)), rng.random((T, 1)))
    x = chain[2000:, 0]
    # a random-walk chain's samples are correlated: allow ~10 effective-sample standard errors
    assert abs(x.mean() - mu) < 0.05 and abs(x.std() - sd) < 0.05
    assert 0.3 < acc.mean() < 0.8
