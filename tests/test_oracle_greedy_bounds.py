"""Pins for Procedure Max-Coverage (Algorithm 4) and the LSBM/GSBM host math.

* Max-Coverage on random set systems: every pick has the largest marginal
  coverage (ties to the smaller id), Cov(B_i) and the top-k marginal sums match
  direct recounts, greedy >= (1 - 1/e) OPT and Cov^u >= OPT (brute-force OPT).
* sigma^L / sigma^U solve the tail equations of Lemma 5.1 that Lemma 5.3's
  proof inverts: x - y = sqrt(2 a y + a^2/9) + a/3 and y - x = sqrt(2 a y).
* theta_max (Lemma 5.2) equals theta_1 = theta_2 of the lemma's proof at the
  balancing epsilon_1; the GSBM analogue likewise (Sec. 5.2).
* Table 3: 2 * floor(theta_0) = 2818 for DBLP with k=100, |S|=10, delta=1/n.
"""
import itertools
import math
import os

import numpy as np
import pytest

from conftest import GOLDEN
import oracle

E = math.e


def _random_sets(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 11))
    ns = int(rng.integers(3, 25))
    sets = []
    for _ in range(ns):
        sz = int(rng.integers(1, 5))
        sets.append(sorted(set(int(x) for x in rng.integers(0, n, sz))))
    return n, sets


def _cov(sets, B):
    Bs = set(B)
    return sum(1 for s in sets if Bs.intersection(s))


@pytest.mark.parametrize("seed", range(25))
def test_max_coverage_against_brute_force(seed):
    n, sets = _random_sets(seed)
    k = 1 + seed % 4
    B, cov, topk = oracle.max_coverage_sets(sets, n, k)
    assert len(B) <= k and len(cov) == len(B) + 1 and len(topk) == len(B) + 1
    for i in range(len(B) + 1):
        Bi = list(B[:i])
        assert int(cov[i]) == _cov(sets, Bi)
        marg = sorted((_cov(sets, Bi + [v]) - _cov(sets, Bi) for v in range(n)), reverse=True)
        assert int(topk[i]) == sum(marg[:k])
        if i < len(B):
            gains = [_cov(sets, Bi + [v]) - _cov(sets, Bi) for v in range(n)]
            best = max(gains)
            assert best > 0 and int(B[i]) == gains.index(best)
    if len(B) < k:                      # stopped early: nothing left to cover
        assert all(_cov(sets, list(B) + [v]) == int(cov[-1]) for v in range(n))
    opt = max(_cov(sets, c) for c in itertools.combinations(range(n), min(k, n)))
    assert int(cov[-1]) >= (1 - 1 / E) * opt - 1e-9
    cov_u = min(int(c) + int(t) for c, t in zip(cov, topk))
    assert cov_u >= opt


@pytest.mark.parametrize("a", [0.5, 3.0, 17.2, 40.0])
@pytest.mark.parametrize("xf", [5 / 18, 0.5, 1.0, 7.0, 300.0])
def test_sigma_low_solves_upper_tail_equation(a, xf):
    x = xf * a
    y = oracle.sigma_low(x, a, 1.0)
    assert x - y == pytest.approx(math.sqrt(2 * a * y + a * a / 9) + a / 3, rel=1e-10, abs=1e-10)
    # theta scaling
    assert oracle.sigma_low(x, a, 8.0) == pytest.approx(y / 8.0, rel=1e-14)
    # below 5a/18 the value is not on the monotone branch: at x = 0 it is 0
    assert oracle.sigma_low(0.0, a, 1.0) == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("a", [0.5, 3.0, 17.2])
@pytest.mark.parametrize("x", [0.0, 1.0, 12.5, 1e4])
def test_sigma_up_solves_lower_tail_equation(a, x):
    y = oracle.sigma_up(x, a, 1.0)
    assert y - x == pytest.approx(math.sqrt(2 * a * y), rel=1e-10)
    assert oracle.sigma_up(x, a, 4.0) == pytest.approx(y / 4.0, rel=1e-14)


def _balanced_theta(E_I, OPT, eps, L1, L2):
    """Lemma 5.2's proof: theta_1 = 2 E L1 / (eps1^2 OPT) and
    theta_2 = (2 - 2/e) E L2 / (OPT (eps - (1-1/e) eps1)^2); bisect for equality."""
    a = 1 - 1 / E
    t1 = lambda e1: 2 * E_I * L1 / (e1 * e1 * OPT)
    t2 = lambda e1: (2 - 2 / E) * E_I * L2 / (OPT * (eps - a * e1) ** 2)
    lo, hi = 1e-12, eps / a - 1e-15
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if t1(mid) > t2(mid):
            lo = mid
        else:
            hi = mid
    return t1(0.5 * (lo + hi))


@pytest.mark.parametrize("n,nS,k,eps,delta,beta,I,OPT", [
    (317080, 10, 100, 0.1, 1 / 317080, 0.1, 2500.0, 30.0),
    (1000, 10, 5, 0.2, 1e-3, 0.1, 120.5, 3.2),
    (10**6, 50, 100, 0.1, 1e-6, 0.1, 20000.0, 70.0),
])
def test_lsbm_theta_max_from_lemma_5_2(n, nS, k, eps, delta, beta, I, OPT):
    got = oracle.lsbm_theta_max(I, n, nS, k, eps, delta, beta, OPT)
    lnC = math.lgamma(n - nS + 1) - math.lgamma(k + 1) - math.lgamma(n - nS - k + 1)
    L1 = math.log(12 / delta)
    want = _balanced_theta(I / (1 - beta), OPT, eps, L1, lnC + L1)
    assert got == pytest.approx(want, rel=1e-9)


def test_gsbm_theta_max_from_proof():
    nVs, nS, k, eps, delta, OPT = 5000, 10, 20, 0.2, 1e-4, 12.0
    got = oracle.gsbm_theta_max(nVs, nS, k, eps, delta, OPT)
    lnC = math.lgamma(nVs - nS + 1) - math.lgamma(k + 1) - math.lgamma(nVs - nS - k + 1)
    L1 = math.log(6 / delta)
    assert got == pytest.approx(_balanced_theta(nVs, OPT, eps, L1, lnC + L1), rel=1e-9)


def test_table3_theta0():
    vals = {}
    for line in open(os.path.join(GOLDEN, "table3.txt")):
        w = line.split()
        if not w or w[0].startswith("#"):
            continue
        if w[0] == "lsbm":
            vals[float(w[1])] = int(w[2])
        else:
            vals[w[0]] = float(w[1])
    n, nS, k, beta = int(vals["n"]), int(vals["S"]), int(vals["k"]), vals["beta"]
    delta = 1 / n
    for eps in (0.4, 0.5):
        for I, OPT in ((3000.0, 40.0), (17.0, 2.5)):      # theta_0 is free of I and OPT
            tmax = oracle.lsbm_theta_max(I, n, nS, k, eps, delta, beta, OPT)
            th0 = math.floor(tmax * (1 - beta) * eps * eps * OPT / I)
            assert 2 * th0 == vals[eps]
    # the other columns are 2 * theta_0 doubled once per extra iteration
    th0 = vals[0.5] // 2
    assert vals[0.3] == 2 * th0 * 2 and vals[0.2] == 2 * th0 * 4 and vals[0.1] == 2 * th0 * 8
