"""Pins of the two oracle parts that set GPU test tolerances and the
benchmark's poles, against facts fixed outside the oracle.

* The stored pole tables of the drift test (K=16, R1=24) and of the benchmark
  (K=32, R1=68): Theorem 1 puts the CF error at sigma_{K+1}; after the Faber
  transform the largest error of r on i[-R1, R1] lies between sigma_{K+1} and
  about twice it (the map of Eq. (9) covers the segment twice).  Evaluated in
  40-digit arithmetic from the tables' 30-digit entries, so the stored values
  themselves are checked, not their FP64 rounding.
* ``oracle.plan.amplification`` (A = max_w sum_j |beta_j| / |w - sigma_j| on
  i[-R1, R1], the factor by which per-pole solve errors can grow in the pole
  sum of Eq. (5)):
  - one pole: A = |beta| / Re(sigma), attained at w = i Im(sigma) (closed form);
  - two poles mirrored about the real axis with equal weights: by symmetry and
    concavity of the sum near the axis, the maximum over the segment is at one
    of the two closest points i Im(sigma_j) or at w = 0 -- computed here from
    the three candidates;
  - the real tables: the 4001-point sampled maximum is within its sampling
    error (bounded by a local refinement with a continuous optimiser at 40
    digits) of the true maximum and never above it.
"""

import os

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from oracle import plan as oplan  # noqa: E402
from oracle import tables  # noqa: E402


def mp_table(K, R1):
    """(sigma, beta, sigma_K+1) of a stored table, parsed at 40 digits."""
    sig, bet, meta = [], [], {}
    with mp.workdps(40):
        for line in open(tables.table_path(K, R1)):
            p = line.split()
            if not p or p[0].startswith("#"):
                continue
            if p[0] in ("K", "L", "R1", "sigma_K+1"):
                meta[p[0]] = mp.mpf(p[1])
                continue
            v = [mp.mpf(x) for x in p]
            sig.append(mp.mpc(v[0], v[1]))
            bet.append(mp.mpc(v[2], v[3]))
    return sig, bet, meta["sigma_K+1"]


def max_err_mp(sig, bet, R1, npts):
    """max over an even grid of w in [-R1, R1] of |r(i w) - e^{i w}| at 40 digits."""
    with mp.workdps(40):
        best = mp.mpf(0)
        for w in np.linspace(-R1, R1, npts):
            z = mp.mpc(0, w)
            r = mp.fsum(b / (z - s) for s, b in zip(sig, bet))
            best = max(best, abs(r - mp.expj(w)))
        return best


@pytest.mark.parametrize("K,R1", [(16, 24.0), (32, 68.0)])
def test_theorem1_error_level_of_stored_tables(K, R1):
    sig, bet, sK1 = mp_table(K, R1)
    assert len(sig) == K
    # ~25 samples per lobe of the error curve (at most ~K + R1/pi lobes)
    e = max_err_mp(sig, bet, R1, 25 * int(2 * (K + R1 / np.pi)))
    assert 0.9 * sK1 <= e <= 2.2 * sK1, (float(e), float(sK1))
    # and the level itself is the one the default-radius rule aims at (2 sigma <= 1e-9)
    assert 2 * sK1 <= 1e-9


def test_amplification_one_pole_closed_form():
    # A = |beta| / Re(sigma) at w = i Im(sigma); R1 = 5 with Im(sigma) on the
    # sampling grid (so the sampled maximum is the exact one), and off the
    # grid (within the quadratic sampling error of the peak).
    R1 = 5.0
    beta = np.array([3.0 - 4.0j])                         # |beta| = 5
    for a in (0.7, 2.0):
        on = np.array([a + 1j * 2.5])                     # 2.5 = -5 + 3000 * (10 / 4000): a grid point
        A = oplan.amplification(on, beta, R1)
        assert abs(A - 5.0 / a) <= 1e-12 * (5.0 / a)
        off = np.array([a + 1j * (2.5 + 0.5 * 10.0 / 4000)])   # half-way between two samples
        Aoff = oplan.amplification(off, beta, R1)
        d = 0.5 * 10.0 / 4000
        assert 5.0 / np.hypot(a, d) * (1 - 1e-12) <= Aoff <= 5.0 / a
    # the pole outside the interval's reach: the maximum sits at the end of the
    # segment nearest to it
    far = np.array([1.0 + 9.0j])
    assert abs(oplan.amplification(far, beta, R1) - 5.0 / abs(5.0j - far[0])) < 1e-12


def test_amplification_two_mirrored_poles():
    # sigma = a +- i b with equal |beta|: f(y) = |beta| (1/|i y - s1| + 1/|i y - s2|)
    # is even in y; its maximum over [-R1, R1] is at y = 0 or y = +-b
    # (the candidates of the two-bump / one-bump shapes); compare with both.
    R1 = 8.0
    for a, b in ((1.0, 3.0), (2.0, 0.5)):
        sig = np.array([a + 1j * b, a - 1j * b])
        beta = np.array([2.0 + 0.0j, 0.0 - 2.0j])
        f = lambda y: 2.0 * (1 / np.hypot(a, y - b) + 1 / np.hypot(a, y + b))
        ys = np.linspace(-R1, R1, 400001)
        true = float(np.max(f(ys)))                                   # fine brute force
        assert true >= max(f(0.0), f(b)) - 1e-12
        A = oplan.amplification(sig, beta, R1)
        assert A <= true * (1 + 1e-12)
        assert A >= true * (1 - 1e-5)


@pytest.mark.parametrize("K,R1", [(16, 24.0), (32, 68.0)])
def test_amplification_sampling_error_on_stored_tables(K, R1):
    sigma, beta, _ = tables.poles(K, R1)
    A = oplan.amplification(sigma, beta, R1)
    sig, bet, _ = mp_table(K, R1)
    absb = [abs(b) for b in bet]

    def f(y):
        with mp.workdps(40):
            z = mp.mpc(0, y)
            return mp.fsum(ab / abs(z - s) for ab, s in zip(absb, sig))

    # refine around every sampled local maximum with a golden-section search
    w = np.linspace(-R1, R1, 4001)
    vals = np.sum(np.abs(beta)[None, :] / np.abs(1j * w[:, None] - sigma[None, :]), axis=1)
    peaks = [i for i in range(1, len(w) - 1) if vals[i] >= vals[i - 1] and vals[i] >= vals[i + 1]]
    peaks += [0, len(w) - 1]
    best = mp.mpf(0)
    for i in peaks:
        lo, hi = w[max(i - 1, 0)], w[min(i + 1, len(w) - 1)]
        with mp.workdps(40):
            g = (mp.sqrt(5) - 1) / 2
            a_, b_ = mp.mpf(lo), mp.mpf(hi)
            for _ in range(60):
                c_, d_ = b_ - g * (b_ - a_), a_ + g * (b_ - a_)
                if f(c_) >= f(d_):
                    b_ = d_
                else:
                    a_ = c_
            best = max(best, f((a_ + b_) / 2), f(lo), f(hi))
    best = float(best)
    assert A <= best * (1 + 1e-12)            # a sampled maximum never exceeds the true one
    assert A >= best * (1 - 1e-4)             # and the 4001-point grid resolves the peak
    # the value the library reports for its own construction agrees
    assert os.path.exists(tables.table_path(K, R1))
