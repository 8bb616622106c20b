"""Pins of the oracle's FCF construction (Algorithm 1, Algorithm 2) against
facts the paper and the mathematics fix, not against the oracle itself.

* a_n of Eq. (8) for exp and the map of Eq. (9) equal the Bessel values J_n(R1)
  (generating function of the Bessel functions; checked with scipy).
* Theorem 1: the CF error is sigma_{n+1}; after the Faber transform the
  maximum error on i[-R1, R1] lies between sigma_{K+1} and 2 sigma_{K+1}
  (eta maps the circle twice onto the segment).
* Table 1: K=16, R1=10, ||e||_inf = 2.38e-9 (golden fixture).
* Sec. 3.4: |r(i w)| - 1 <= ||e||_inf on the interval, |r(z)| -> 0 for |z| -> inf.
* Algorithm 2's linear system agrees with the residue formula
  beta_k = Res_{z_k} r^cf * eta'(z_k), derived independently from the Faber
  generating function eta'(t)/(eta(t) - w) = sum_j p_j(w) t^{-j-1}.
* The Faber coefficients of 1/(w - sigma_k) equal -2 z_k^{-j} / (R1 (z_k + 1/z_k)).
"""

import os

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from oracle import fcf, tables  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_fcf.txt")


def read_golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


@pytest.fixture(scope="module")
def small():
    return fcf.faber_cf(8, 8)


@pytest.fixture(scope="module")
def table1():
    g = read_golden()
    return fcf.faber_cf(g["R1"], int(g["K"]))


def max_err(sigma, beta, R1, npts=1501):
    with mp.workdps(40):
        return max(abs(fcf.rational_eval(sigma, beta, mp.mpc(0, w)) - mp.expj(w))
                   for w in np.linspace(-R1, R1, npts))


def test_faber_coefficients_are_bessel_values():
    scipy_special = pytest.importorskip("scipy.special")
    for R1 in (3.0, 10.0, 24.0):
        with mp.workdps(40):
            a = fcf.faber_sequence_exp(R1, 40)
        ref = scipy_special.jv(np.arange(41), R1)
        got = np.array([float(x) for x in a])
        assert np.max(np.abs(got - ref)) < 1e-14, R1


def test_faber_coefficients_sign_and_decay():
    # exp(eta(z)) = sum_n J_n(R) z^n: a_0 = J_0(R), and superexponential decay.
    with mp.workdps(40):
        a = fcf.faber_sequence_exp(5, 30)
        assert abs(a[0] - mp.besselj(0, 5)) < mp.mpf(10) ** -35
        assert abs(a[30]) < mp.mpf(10) ** -15


def test_theorem1_error_level(small):
    sigma, beta, info = small
    e = max_err(sigma, beta, 8.0)
    s = info["sigma"]
    assert s < 1e-5
    assert 0.9 * s <= e <= 2.2 * s


def test_laurent_tail_vanishes(small):
    # q_out * r~* has no terms of degree >= n (r~* lies in R~_{n-1,n}).
    _, _, info = small
    assert max(abs(x) for x in info["numerator_tail"]) < mp.mpf(10) ** -40


def test_outer_root_count_and_mapping(small):
    sigma, _, info = small
    assert len(info["z"]) == 8
    with mp.workdps(60):
        for z, s in zip(info["z"], sigma):
            assert abs(z) > 1
            # eta maps |z| > 1 off the segment: poles are not on i[-R1, R1].
            assert abs(mp.re(s)) > 0.5
            assert abs(s - fcf.eta(z, 8)) < mp.mpf(10) ** -40
    # real-coefficient q: roots in conjugate pairs -> poles symmetric about the real axis
    ims = sorted(float(mp.im(s)) for s in sigma)
    assert np.allclose(ims, [-x for x in reversed(ims)], atol=1e-20)


def test_table1_error(table1):
    g = read_golden()
    sigma, beta, info = table1
    e_exact = max_err(sigma, beta, g["R1"])
    assert e_exact <= g["err_inf"]
    # FP64-stored weights: the error is at the FP64 evaluation floor, within an
    # order of magnitude of the printed 2.38e-9.
    s64 = np.array([complex(s) for s in sigma])
    b64 = np.array([complex(b) for b in beta])
    w = 1j * np.linspace(-g["R1"], g["R1"], 20001)
    r = (b64[None, :] / (w[:, None] - s64[None, :])).sum(1)
    e64 = np.max(np.abs(r - np.exp(w)))
    assert g["err_inf"] / 10 <= e64 <= g["err_inf"] * 10


def test_stability_statements(table1):
    g = read_golden()
    sigma, beta, _ = table1
    s64 = np.array([complex(s) for s in sigma])
    b64 = np.array([complex(b) for b in beta])
    w = 1j * np.linspace(-g["R1"], g["R1"], 20001)
    r = (b64[None, :] / (w[:, None] - s64[None, :])).sum(1)
    e64 = np.max(np.abs(r - np.exp(w)))
    # |r(i w)| - 1 is at most ||e||_inf on the interval (Sec. 3.4)
    assert np.max(np.abs(r)) - 1.0 <= e64 * 1.0001
    # |r(z)| -> 0 as |z| -> infinity (strictly proper)
    big = np.array([1e3, 1e4, 1e5]) * (1 + 1j)
    rb = np.abs((b64[None, :] / (big[:, None] - s64[None, :])).sum(1))
    assert rb[2] < rb[1] < rb[0] and rb[2] < 1e-3
    # Dahlquist's test equation: u_{n+1} = r(w) u_n decays for w in the left
    # half-plane away from the interval.
    wl = -2.0 + 3.0j
    rl = abs(np.sum(b64 / (wl - s64)))
    assert rl < 1.0
    # the paper's arithmetic: (1 + 1e-9)^n = 2 at n = ln 2 / ln(1 + 1e-9) ~ 7e8
    n2 = np.log(2.0) / np.log1p(g["abs_r_minus_1"])
    assert abs(n2 - g["steps_to_double"]) / g["steps_to_double"] < 0.05


def test_vandermonde_route_equals_residue_route(small):
    sigma, beta, info = small
    R1 = info["R1"]
    zs = info["z"]
    num = info["numerator"]
    with mp.workdps(60):
        for k, zk in enumerate(zs):
            # residue of N(z)/prod(z - z_j) at z_k
            Nk = sum(c * zk ** j for j, c in enumerate(num))
            den = mp.mpc(1)
            for j, zj in enumerate(zs):
                if j != k:
                    den *= (zk - zj)
            res = Nk / den
            eta_prime = R1 / 2 * (1 + 1 / zk ** 2)
            assert abs(res * eta_prime - beta[k]) <= mp.mpf(10) ** -30 * (1 + abs(beta[k]))


def test_resolvent_faber_coefficients_closed_form(small):
    sigma, _, info = small
    R1 = info["R1"]
    with mp.workdps(60):
        for zk, sk in list(zip(info["z"], sigma))[:3]:
            b = fcf.faber_sequence_resolvent(sk, zk, R1, 6)
            for j in range(6):
                ref = -2 * zk ** (-j) / (R1 * (zk + 1 / zk))
                assert abs(b[j] - ref) < mp.mpf(10) ** -40


def test_stored_tables_agree_with_fresh_construction(small):
    sigma, beta, info = small
    s_t, b_t, meta = tables.poles(8, 8)
    assert meta["K"] == 8
    s = np.array([complex(x) for x in sigma])
    b = np.array([complex(x) for x in beta])
    assert np.max(np.abs(s_t - s) / np.abs(s)) < 1e-15
    assert np.max(np.abs(b_t - b) / np.abs(b)) < 1e-15


def test_exp_at_zero(small):
    sigma, beta, _ = small
    with mp.workdps(40):
        assert abs(fcf.rational_eval(sigma, beta, mp.mpc(0)) - 1) < 1e-5
