"""The cost model of Section 4 (Eq. 1) in the autotuner, pinned to the paper's Tables 1-2.

`tune.fit_eq1` fits t(n) = n*s + 2*tau/n to measured times and returns s, tau and the
optimum n* = sqrt(2 tau / s); the latency bench reports that fit.  The fixture
`tests/golden/eq1_tables.txt` holds the values the paper prints (Table 1: interconnect
latencies; Table 2: node speed, FLOP per step-point and the resulting s) and, as ranges,
Section 4's remarks on the tables' extremes (the optimum node size is of order 10^4 points
at cloud latency for the cheapest step, between 1 and 2 for an expensive step on a slow
node, and the best time per step is of order a nanosecond).  The tests check Table 2's arithmetic, that the fit recovers s and
tau from exact Eq. 1 samples for every table combination, and the paper's statements
through the fitted n* and the minimum of the fitted curve.
"""
from __future__ import annotations

import math
import os

import pytest

from paper_1504_01380_gb300 import tune

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq1_tables.txt")


def load():
    taus, nodes, claims = [], [], []
    with open(GOLDEN) as f:
        for line in f:
            w = line.split()
            if not w or w[0].startswith("#"):
                continue
            if w[0] == "table1":
                taus.append(float(w[2]))
            elif w[0] == "table2":
                nodes.append((float(w[2]), float(w[3]), float(w[4])))
            elif w[0] == "claim":
                claims.append((float(w[1]), float(w[2]), w[3], float(w[4]), float(w[5])))
    return taus, nodes, claims


def eq1(n, s, tau):
    return n * s + 2.0 * tau / n


def test_table2_is_f_over_F():
    _, nodes, _ = load()
    assert len(nodes) == 6
    for F, f, s_printed in nodes:
        assert f / F == pytest.approx(s_printed, rel=1e-12)


@pytest.mark.parametrize("i_tau", range(4))
def test_fit_recovers_s_tau_and_optimum(i_tau):
    taus, nodes, _ = load()
    tau = taus[i_tau]
    for _, _, s in nodes:
        nstar = math.sqrt(2 * tau / s)
        ns = [max(1.0, nstar * x) for x in (0.125, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0)]
        fit = tune.fit_eq1([(n, eq1(n, s, tau)) for n in ns])
        assert fit["s"] == pytest.approx(s, rel=1e-9)
        assert fit["tau"] == pytest.approx(tau, rel=1e-9)
        assert fit["n_star"] == pytest.approx(nstar, rel=1e-9)
        # the curve's minimum is t* = sqrt(8 tau s), at n*
        assert eq1(fit["n_star"], fit["s"], fit["tau"]) == pytest.approx(math.sqrt(8 * tau * s), rel=1e-9)


def test_paper_statements_on_the_extremes():
    _, _, claims = load()
    assert len(claims) == 3
    for tau, s, what, lo, hi in claims:
        ns = [1.0, 2.0, 4.0, 16.0, 256.0, 4096.0, 65536.0]
        fit = tune.fit_eq1([(n, eq1(n, s, tau)) for n in ns])
        value = fit["n_star"] if what == "n_star" else eq1(fit["n_star"], fit["s"], fit["tau"])
        assert lo <= value <= hi, (what, tau, s, value)


def test_degenerate_inputs():
    assert tune.fit_eq1([(8.0, 1.0)]) is None                        # one point: singular
    fit = tune.fit_eq1([(1.0, 2.0), (2.0, 4.0), (4.0, 8.0)])         # t = 2n: no latency term
    assert fit["n_star"] is None
