"""Growth statistics (mean, mode, variance, skewness, kurtosis of the distance distribution) on
host-side layer vectors, pinned to closed forms: Coxeter growth is the Mahonian distribution
(mean n(n-1)/4, symmetric: skewness 0; Section 3.3 table, Coxeter row); all transpositions give
distance n - (number of cycles), so the mean is n - H_n (H_n the harmonic number) and the
variance is H_n - H_n^(2)."""

from fractions import Fraction

import pytest

import oracle
import workloads as w
from paper_2509_19162_gb300.api import GrowthResult


@pytest.mark.parametrize("n", range(2, 9))
def test_coxeter_moments(n):
    st = GrowthResult(oracle.growth(n, w.coxeter(n))[0], 0).statistics()
    assert st["mean"] == pytest.approx(n * (n - 1) / 4)
    assert st["skewness"] == pytest.approx(0.0, abs=1e-12)
    # variance of the inversion count: sum_{j<=n} (j^2 - 1) / 12
    assert st["variance"] == pytest.approx(sum((j * j - 1) / 12 for j in range(1, n + 1)))
    assert st["diameter"] == n * (n - 1) // 2


@pytest.mark.parametrize("n", range(2, 9))
def test_all_transpositions_moments(n):
    st = GrowthResult(oracle.growth(n, w.all_transpositions(n))[0], 0).statistics()
    H1 = sum(Fraction(1, j) for j in range(1, n + 1))
    H2 = sum(Fraction(1, j * j) for j in range(1, n + 1))
    assert st["mean"] == pytest.approx(float(n - H1))
    assert st["variance"] == pytest.approx(float(H1 - H2))


def test_mode_and_degenerate_cases():
    assert GrowthResult([1], 0).statistics()["variance"] == 0.0
    assert GrowthResult([1, 3, 3, 1], 0).statistics()["mode"] == 1      # first of equal maxima
    st = GrowthResult([1, 2, 4, 8], 0).statistics()
    assert st["mode"] == 3 and st["skewness"] < 0
