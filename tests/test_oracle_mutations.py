"""Plant plausible mistakes in the oracle (CPU only) and check that the pins
in test_oracle_pins.py catch each of them: a pin set that passed a dropped
factor, a flipped sign or a swapped operand would not pin anything."""
import numpy as np
import pytest

import oracle
import oracle.rmatrix as orm

pytest.importorskip("mpmath")
import test_oracle_pins as pins  # noqa: E402


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def _r_no_half_a(E, E_k, W, a):
    d = 1.0 / (np.asarray(E_k) - E)
    return (W * d[None, :]) @ W.T / a


def _r_sign(E, E_k, W, a):
    d = 1.0 / (E - np.asarray(E_k))
    return (W * d[None, :]) @ W.T / (2 * a)


def _t_no_inverse(K):
    n = K.shape[0]
    return 2j * K @ (np.eye(n) - 1j * K)


def _omega_double_count(row, T, open_idx, level, n_levels, g):
    level = np.asarray(level)
    T2 = np.abs(T) ** 2
    lv = level[open_idx]
    for p in range(lv.size):
        for q in range(lv.size):
            I, J = sorted((int(lv[p]), int(lv[q])))
            row[orm.tri_index(I, J, n_levels)] += g * T2[p, q]
    return row


def _omega_level_by_position(row, T, open_idx, level, n_levels, g):
    # level of the open-channel position instead of the channel's own level
    T2 = np.abs(T) ** 2
    lv = np.asarray(level)[: len(open_idx)]
    lv = np.sort(lv)
    for p in range(lv.size):
        for q in range(lv.size):
            I, J = int(lv[p]), int(lv[q])
            if I <= J:
                row[orm.tri_index(I, J, n_levels)] += g * T2[p, q]
    return row


_orig_cf = orm.channel_functions


def _cf_bad_norm(*a, **k):
    cf = _orig_cf(*a, **k)
    op = cf["open"]
    eps = cf["eps"]
    kk = np.sqrt(np.where(op, eps, 1.0))
    cf["s"] = np.where(op, cf["s"] * kk, 0.0)   # F sqrt(k) instead of F / sqrt(k)
    cf["c"] = np.where(op, cf["c"] * kk, 0.0)
    return cf


def _cf_flip_L(*a, **k):
    cf = _orig_cf(*a, **k)
    cf["thp"] = -cf["thp"]
    cf["L"] = -cf["L"]
    return cf


_orig_mqdt = orm.match_mqdt


def _mqdt_flip_tan(R, cf, l, z, a, b=0.0, Q=None, fnumin=0.0, margin=0.1):
    cf2 = dict(cf)
    cf2["nu"] = cf["nu"].copy()
    # pi nu -> -pi nu flips tan and sin; only the eliminating tan is flipped by
    # shifting nu by 1/2 period inside the elimination step
    K, Ku, oi, qi = _orig_mqdt(R, cf, l, z, a, b, Q, fnumin, margin)
    if K is None or len(qi) == 0:
        return K, Ku, oi, qi
    po = cf["open"][np.nonzero(cf["open"] | np.isin(np.arange(len(cf["open"])), qi))[0]]
    Koo, Koc = Ku[np.ix_(po, po)], Ku[np.ix_(po, ~po)]
    Kco, Kcc = Ku[np.ix_(~po, po)], Ku[np.ix_(~po, ~po)]
    tanb = np.tan(np.pi * cf["nu"][qi])
    return Koo - Koc @ np.linalg.solve(Kcc - np.diag(tanb), Kco), Ku, oi, qi


MUTATIONS = [
    ("r_matrix", _r_no_half_a, [(pins.test_r_matrix_bruteforce_and_symmetry,)]),
    ("r_matrix", _r_sign, [(pins.test_r_matrix_bruteforce_and_symmetry,)]),
    ("t_matrix", _t_no_inverse, [(pins.test_k_symmetric_and_s_unitary,)]),
    ("omega_add", _omega_double_count, [(pins.test_omega_real_form_and_symmetry,),
                                        (pins.test_omega_aggregation_from_unitarity, 3)]),
    ("omega_add", _omega_level_by_position, [(pins.test_omega_aggregation_from_unitarity, 17),
                                             (pins.test_omega_two_levels_by_hand,)]),
    ("channel_functions", _cf_bad_norm, [(pins.test_square_well_tan_delta, 6.0)]),
    ("channel_functions", _cf_flip_L, [(pins.test_mqdt_two_channel_vs_mpmath,)]),
    ("match_mqdt", _mqdt_flip_tan, [(pins.test_mqdt_equals_direct,)]),
]


@pytest.mark.parametrize("name,fn,checks", MUTATIONS,
                         ids=[m[1].__name__ for m in MUTATIONS])
def test_mutation_is_caught(monkeypatch, name, fn, checks):
    monkeypatch.setattr(orm, name, fn)
    monkeypatch.setattr(oracle, name, fn)
    for chk in checks:
        assert _fails(*chk), "pin %s passed a planted mistake in %s" % (chk[0].__name__, name)
