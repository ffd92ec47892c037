"""Pins of the standard error that the oracle reports with its gradient.

The gradient estimate is the sample mean of the per-sample scores
Y_h = 1_F(x_h) 1{x_{h,i} = k} / q_{i,k}, so its standard error is the
population standard deviation of the Y_h divided by sqrt(H).  Three pins that
do not restate the oracle's closed form:

* the standard deviation of the explicit score vector, formed sample by
  sample with numpy, on the 3x4 grid and on a series system with a large
  failure probability (where a dropped (1 - p) factor would show);
* a 50-digit decimal evaluation of the variance of a scaled Bernoulli mean for
  hand-picked counts, including p > 1/2 and p = 1;
* the spread of the estimate over independent sample streams: the standard
  deviation of g over 400 seeds agrees with the reported standard error.
"""
from decimal import Decimal, getcontext

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


def _scores(X, labels, pmf, i, k):
    """Y_h for every sample h, as the definition writes it."""
    fail = (labels == 0).astype(np.float64)
    hit = (X[:, i] == k).astype(np.float64)
    return fail * hit / pmf[i, k]


@pytest.mark.parametrize("system", ["grid", "series"])
def test_se_is_population_std_of_scores(system):
    if system == "grid":
        p = W.c1_grid()
        N, seed = 50_000, 11
    else:
        # P(F) = 1 - prod(1 - p_fail) ~ 0.76: the (1 - p) factor of the variance is far from 1
        p = W.series_system(np.array([0.3, 0.45, 0.2, 0.25]))
        N, seed = 20_000, 12
    X = O.sample(p.pmf, seed=seed, offset=0, N=N)
    labels, _ = O.classify(X, p.ref_L, p.ref_U)
    g, se = O.grad(O.grad_counts(X, labels, p.K), N, p.pmf)
    for i in range(p.n):
        for k in range(p.K):
            Y = _scores(X, labels, p.pmf, i, k)
            assert g[i, k] == pytest.approx(Y.mean(), rel=1e-12, abs=1e-300)
            want = Y.std(ddof=0) / np.sqrt(N)
            assert se[i, k] == pytest.approx(want, rel=1e-10, abs=1e-300), (i, k)


def _decimal_se(C, N, q):
    getcontext().prec = 50
    C, N, q = Decimal(C), Decimal(N), Decimal(repr(q))
    mean = C / N / q                    # E[Y] over the H samples
    second = C / N / (q * q)            # E[Y^2]: Y^2 = Y / q on the samples with Y != 0
    var = second - mean * mean          # population variance of Y
    return (var / N).sqrt()


@pytest.mark.parametrize("C,N,q", [(3, 10, 0.25), (7, 10, 0.8), (999_999, 1_000_000, 0.999_999),
                                   (1, 3, 1.0), (12_345, 67_890, 0.3), (5, 5, 0.5), (0, 8, 0.5)])
def test_se_against_50_digit_decimal(C, N, q):
    Cm = np.array([[C, 0]], dtype=np.int64)
    pmf = np.array([[q, 1.0 - q]])
    g, se = O.grad(Cm, N, pmf)
    want = _decimal_se(C, N, q)
    # fp64 forms 1 - p from a rounded p = C/H: relative error up to about
    # eps * p / (1 - p) in the variance, half of it in the square root
    pf = C / N
    rel = 1e-14 + (2.0 ** -52) * (pf / (1.0 - pf) if pf < 1.0 else 0.0)
    assert se[0, 0] == pytest.approx(float(want), rel=rel, abs=1e-300)
    assert g[0, 0] == pytest.approx(float(Decimal(C) / Decimal(N) / Decimal(repr(q))), rel=1e-15)


def test_se_predicts_spread_over_independent_streams():
    # a series system with P(F) ~ 0.6: every entry has p = C/H well inside (0, 1)
    p = W.series_system(np.array([0.2, 0.3, 0.25]))
    N, reps = 2_000, 400
    gs, ses = [], []
    for r in range(reps):
        X = O.sample(p.pmf, seed=5000 + r, offset=0, N=N)
        labels, _ = O.classify(X, p.ref_L, p.ref_U)
        g, se = O.grad(O.grad_counts(X, labels, p.K), N, p.pmf)
        gs.append(g)
        ses.append(se)
    spread = np.std(np.array(gs), axis=0, ddof=1)
    mean_se = np.mean(np.array(ses), axis=0)
    # the standard deviation of 400 draws is known to about 1/sqrt(800) = 3.5%;
    # 0.85..1.15 is four of those either way, for each of the six entries
    ratio = spread / mean_se
    assert np.all((ratio > 0.85) & (ratio < 1.15)), ratio
