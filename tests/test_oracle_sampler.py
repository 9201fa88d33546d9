"""Pins of the oracle's Philox generator and importance sampler (Eq. F_long_RBE).

The mode density P(k) ~ exp(-k^2/4 alpha) on K \\ {0} (Sec. 2.1) factorises over axes;
these tests check the oracle's sampler against facts that do not come from its code:
published Philox known-answer vectors, the Poisson-summation closed form of the axis
normaliser, a chi-square test of the draws, and the unbiasedness of S f(k).
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat_rows())
def test_philox_known_answers(orc, ctr, key, want):
    assert list(orc.philox4x32_10(ctr, key)) == want


def _axis_weight(m, L, alpha):
    k = 2.0 * math.pi * m / L
    return math.exp(-k * k / (4.0 * alpha))


@pytest.mark.parametrize("L,alpha", [(32.0, 0.09), (8.0, 0.5), (218.877, 0.09), (11.3, 0.3)])
def test_axis_normaliser_poisson_summation(orc, L, alpha):
    """Z = sum_m exp(-pi^2 m^2/(alpha L^2)) = L sqrt(alpha/pi) sum_n exp(-alpha L^2 n^2)."""
    T, Z = orc.kdim_table(L, alpha)
    dual = L * math.sqrt(alpha / math.pi) * sum(
        math.exp(-alpha * L * L * n * n) for n in range(-20, 21))
    assert Z == pytest.approx(dual, rel=1e-13)
    assert T[-1] == 1 << 32
    assert np.all(np.diff(T.astype(np.int64)) >= 0)
    M = (len(T) - 1) // 2
    # weight beyond the table is below 2^-53 of the peak; inside, the next one is not
    assert _axis_weight(M, L, alpha) < 2.0 ** -53
    assert _axis_weight(M - 1, L, alpha) >= 2.0 ** -53 * 0.999


@pytest.mark.parametrize("L,alpha", [(8.0, 0.5), (32.0, 0.09)])
def test_axis_thresholds_match_probabilities(orc, L, alpha):
    """Each threshold step is the axis probability times 2^32 (to one unit)."""
    T, Z = orc.kdim_table(L, alpha)
    M = (len(T) - 1) // 2
    prev = 0
    for i, t in enumerate(T.astype(np.int64)):
        p = _axis_weight(i - M, L, alpha) / Z
        assert abs((int(t) - prev) - p * 2 ** 32) <= 1.0 + 1e-6
        prev = int(t)


def test_sampler_chi_square_and_rejection(orc):
    """Draw frequencies follow exp(-k^2/4 alpha) conditioned on m != 0."""
    box = np.array([8.0, 9.0, 10.0])
    alpha = 0.5
    P = 60000
    m, S = orc.sample_k(seed=12345, step=7, replica=0, box=box, alpha=alpha, P=P)
    assert not np.any(np.all(m == 0, axis=1))
    Zs = [orc.kdim_table(L, alpha)[1] for L in box]
    w0 = [1.0 / Z for Z in Zs]           # axis probability of m_d = 0
    p000 = w0[0] * w0[1] * w0[2]
    for d in range(3):
        L = box[d]
        lo, hi = int(m[:, d].min()), int(m[:, d].max())
        vals = np.arange(lo - 2, hi + 3)
        others = np.prod([w0[e] for e in range(3) if e != d])
        p = np.array([_axis_weight(a, L, alpha) / Zs[d] * (1.0 - (others if a == 0 else 0.0))
                      for a in vals]) / (1.0 - p000)
        counts = np.array([(m[:, d] == a).sum() for a in vals])
        keep = p * P >= 5
        exp_ = np.append(p[keep] * P, p[~keep].sum() * P)
        obs = np.append(counts[keep], counts[~keep].sum())
        chi2 = ((obs - exp_) ** 2 / exp_).sum()
        pval = stats.chi2.sf(chi2, len(obs) - 1)
        assert pval > 1e-4, (d, chi2, pval)
    assert S == pytest.approx(Zs[0] * Zs[1] * Zs[2] - 1.0, rel=1e-15)


def test_sampler_determinism_and_streams(orc):
    box = np.array([32.0, 32.0, 32.0])
    a, Sa = orc.sample_k(1, 0, 0, box, 0.09, 100)
    b, Sb = orc.sample_k(1, 0, 0, box, 0.09, 100)
    c, _ = orc.sample_k(1, 1, 0, box, 0.09, 100)
    d, _ = orc.sample_k(1, 0, 1, box, 0.09, 100)
    e, _ = orc.sample_k(2, 0, 0, box, 0.09, 100)
    assert np.array_equal(a, b) and Sa == Sb
    for other in (c, d, e):
        assert not np.array_equal(a, other)
    # a prefix of a larger sample is the smaller sample (mode l depends on l only)
    f, _ = orc.sample_k(1, 0, 0, box, 0.09, 250)
    assert np.array_equal(f[:100], a)


def test_importance_sampling_is_unbiased(orc):
    """E[S f(k)] = sum_{k != 0} exp(-k^2/4 alpha) f(k) for f(k) = 1/k^2 (the RBE weight)."""
    box = np.array([6.0, 7.0, 8.0])
    alpha = 0.4
    m, S = orc.sample_k(99, 3, 0, box, alpha, 200000)
    k = 2 * np.pi * m / box
    k2 = (k * k).sum(axis=1)
    est = S / k2
    Ms = [orc.kdim_M(L, alpha) for L in box]
    g = np.meshgrid(*[np.arange(-M, M + 1) for M in Ms], indexing="ij")
    kk = sum((2 * np.pi * g[d] / box[d]) ** 2 for d in range(3))
    kk[Ms[0], Ms[1], Ms[2]] = np.inf
    exact = np.sum(np.exp(-kk / (4 * alpha)) / kk)
    sem = est.std() / math.sqrt(len(est))
    assert abs(est.mean() - exact) < 4 * sem, (est.mean(), exact, sem)
