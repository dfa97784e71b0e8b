"""Pins of the property the near-threshold channel tables rest on, checked
with the oracle's own binary128 functions (no library code):

At fixed r = a, with A(eps, l) = prod_{p=1..l} (1 + p^2 eps / z^2),
  * the open-side s / sqrt(A) continues analytically into the closed side's
    energy-analytic regular solution f;
  * the open-side c sqrt(A) continues into g~, the quantum-defect g at
    half-integer nu (where theta ~ g~ and f'g~ - f g~' = 1 give
    g~ = -1/(f L - f'), L = theta'/theta);
  * the decaying solution is theta ~ A f cos(pi nu) - g~ sin(pi nu) at every
    closed energy, so its log-derivative follows from f and g~ alone.
Each is checked by polynomial interpolation in energy through nodes on the
other side (or at other energies) against the direct continued fractions.
"""
import numpy as np
import pytest

from oracle import _clib

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _A(eps, l, z):
    return np.prod([1.0 + p * p * eps / z ** 2 for p in range(1, l + 1)], axis=0) if l else np.ones_like(eps)


def _open(l, eps, z, a):
    k = np.sqrt(eps)
    out, st = _clib.coulomb_open(np.full(eps.size, l, np.int32), -z / k, k * a)
    assert not st.any()
    sk = np.sqrt(k)
    return out[:, 0] / sk, out[:, 1] * sk, out[:, 2] / sk, out[:, 3] * sk


def _closed(l, eps, z, a):
    kap = np.sqrt(-eps)
    y, st = _clib.whittaker_logderiv(np.full(eps.size, l, np.int32), z / kap, 2 * kap * a)
    assert not st.any()
    fo, st2 = _clib.regular_analytic(np.full(eps.size, l, np.int32), z, eps, a)
    assert not st2.any()
    return 2 * kap * y, fo[:, 0], fo[:, 1]


def _interp(xs, ys, x):
    return np.polyval(np.polyfit(xs, ys, xs.size - 1), x)


CASES = [(2.0, 15.0, 0), (2.0, 15.0, 6), (1.0, 10.0, 3), (5.0, 8.0, 9)]


@pytest.mark.parametrize("z,a,l", CASES)
def test_open_pair_continues_into_closed_pair(z, a, l):
    h = min(0.0164 * np.sqrt(z) / a ** 1.5, 0.05 * z * z / (l + 1.0) ** 2)
    xo = h * np.arange(1, 9)
    s, sp, c, cp = _open(l, xo, z, a)
    sA = np.sqrt(_A(xo, l, z))
    nu = np.floor(z / np.sqrt(h * np.array([1.0, 2.0]))) + 0.5        # half-integer nu below threshold
    xc = -(z / nu) ** 2
    L, f, fp = _closed(l, xc, z, a)
    gt = -1.0 / (f * L - fp)
    for ys, exp in ((s / sA, f), (sp / sA, fp), (c * sA, gt), (cp * sA, L * gt)):
        got = _interp(xo / h, ys, xc / h)
        assert np.all(np.abs(got - exp) <= 1e-9 * np.abs(ys).max()), (z, a, l, got, exp)


@pytest.mark.parametrize("z,a,l", CASES)
def test_theta_from_f_and_g_at_half_integer_nu(z, a, l):
    h = min(0.0164 * np.sqrt(z) / a ** 1.5, 0.05 * z * z / (l + 1.0) ** 2)
    nus = []
    for j in range(1, 9):
        v = np.floor(z / np.sqrt(h * j)) + 0.5
        nus.append(v if not nus else min(nus[-1] - 1.0, v))
    xc = -(z / np.array(nus)) ** 2
    L, f, fp = _closed(l, xc, z, a)
    gt = -1.0 / (f * L - fp)
    gtp = L * gt
    # targets between the nodes, at general (not half-integer) nu
    xt = -h * np.array([1.37, 2.61, 4.22, 6.9])
    Lt, ft, fpt = _closed(l, xt, z, a)
    g_i = _interp(xc / h, gt, xt / h)
    gp_i = _interp(xc / h, gtp, xt / h)
    nu_t = z / np.sqrt(-xt)
    fr = nu_t - np.floor(nu_t)
    sb, cb = np.sin(np.pi * fr), np.cos(np.pi * fr)
    A = _A(xt, l, z)
    th = A * ft * cb - g_i * sb
    thp = A * fpt * cb - gp_i * sb
    # the same direction as the continued fraction's log-derivative
    d1 = th / np.hypot(th, a * thp)
    d2 = 1.0 / np.hypot(1.0, a * Lt)
    assert np.all(np.abs(np.abs(d1) - d2) <= 1e-9), (z, a, l)
    assert np.all(np.abs(thp / th - Lt) <= 1e-9 * np.maximum(1.0, np.abs(Lt))), (z, a, l)
    # without A the relation fails visibly whenever l > 0
    if l > 0:
        th0 = ft * cb - g_i * sb
        thp0 = fpt * cb - gp_i * sb
        assert np.max(np.abs(thp0 / th0 - Lt)) > 1e-6


@pytest.mark.parametrize("z,a,l", [(1.0, 5.0, 15), (1.0, 10.0, 15), (2.0, 15.0, 8), (2.0, 15.0, 0),
                                   (1.0, 20.0, 3), (5.0, 8.0, 9)])
def test_open_regular_solution_matches_its_power_series(z, a, l):
    """The open-channel s, s' (continued fractions at l = 0, G carried up,
    F_l by the Wronskian) against the energy-analytic regular solution f
    from its power series: s = sqrt(B) f with B = A / (1 - exp(-2 pi z/k)),
    the ratio of the two normalisations at r -> 0 (C_l(eta)^2 k^(2l+1) over
    f's). Includes r = a deep inside an l = 15 barrier (F/G ~ 1e-35)."""
    eps = np.array([3e-7, 4e-5, 1e-3, 0.05, 0.5])
    s, sp, c, cp = _open(l, eps, z, a)
    fo, st = _clib.regular_analytic(np.full(eps.size, l, np.int32), z, eps, a)
    assert not st.any()
    k = np.sqrt(eps)
    sB = np.sqrt(_A(eps, l, z) / (1.0 - np.exp(-2.0 * np.pi * z / k)))
    np.testing.assert_allclose(s, sB * fo[:, 0], rtol=1e-13)
    np.testing.assert_allclose(sp, sB * fo[:, 1], rtol=1e-13)
    np.testing.assert_allclose(sp * c - s * cp, 1.0, rtol=0, atol=1e-14)
