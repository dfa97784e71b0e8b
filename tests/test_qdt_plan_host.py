"""The library's host planning of the MQDT coarse-mesh interpolation
(rm_qdt_plan_inspect: no GPU) against the oracle's plan (oracle/qdt.py, Section
"namelist stgf MQDT variables": imode = -1, ieq, qetest): segments,
interpolation energies, the valid nodes of every segment and the
interpolation weights of every fine energy, exactly. The channel classes are
the oracle's, fed to both sides."""
import numpy as np
import pytest

from oracle import qdt
from paper_1909_07321_gb300 import rmgb, synth


def _pw():
    pw = synth.random_pw(4711, 4, 60, z=2.0, a=10.0, e_max=1.8, sigma=0.1, l_max=3)
    pw["e_thr"] = np.array([0.0, 0.6, 1.2, 1.8])
    return pw


def _grid(pw):
    E = synth.midpoint_grid(0.05, 2.1, 500)
    E[100] = pw["e_thr"][1]                   # two energies on thresholds
    E[333] = pw["e_thr"][2]
    inside = pw["E_k"][(pw["E_k"] > 0.3) & (pw["E_k"] < 2.0)]
    E[250] = inside[0]                        # and one on a pole
    return np.unique(E)


def _classes(pw, E):
    out = np.empty((E.size, len(pw["e_thr"])), dtype=np.int8)
    for m, x in enumerate(E):
        c = qdt.classes(float(x), pw)
        out[m] = 3 if c is None else c
    return out


@pytest.mark.parametrize("ieq,qetest", [(-1, 0.0), (-7, 0.0), (-25, 0.01), (40, 0.0), (7, 0.002), (1, 0.0)])
def test_plan_matches_oracle(ieq, qetest):
    pw = _pw()
    E = _grid(pw)
    lib = rmgb.rm_qdt_plan_inspect(pw["e_thr"], pw["z"], pw["E_k"], E, _classes(pw, E), ieq, qetest)
    pl = qdt.plan(pw, E, ieq, qetest)
    assert np.array_equal(lib["seg"], pl["seg"])
    assert (pl["seg"] < 0).sum() == 2
    assert np.array_equal(lib["e_int"], pl["e_int"])
    n_seg = len(pl["segments"])
    assert n_seg >= 6 and set(np.unique(lib["node_seg"])) <= set(range(n_seg))
    dropped = 0
    for s, (i0, i1, cls_seg) in enumerate(pl["segments"]):
        xs = np.array([x for x in pl["nodes"][s] if qdt.node_valid(pw, float(x), cls_seg)])
        dropped += len(pl["nodes"][s]) - xs.size
        idx = np.nonzero(lib["node_seg"] == s)[0]
        assert np.array_equal(lib["node_x"][idx], xs), s
        for m in range(i0, i1 + 1):
            if xs.size == 0:
                assert lib["node_a"][m] == -1
                continue
            if xs.size == 1:
                assert lib["node_a"][m] == lib["node_b"][m] == idx[0]
                continue
            j, t = qdt.interpolation_weights(xs, pl["e_int"][m])
            assert (lib["node_a"][m], lib["node_b"][m]) == (idx[j], idx[j + 1]), m
            assert lib["t"][m] == t, m
    assert np.all(lib["node_a"][pl["seg"] < 0] == -1)
    if ieq == -1:
        assert dropped >= 1                   # the pole (and |sin pi nu| < 1e-3 nodes)


def test_plan_rejects_bad_input():
    pw = _pw()
    E = _grid(pw)
    cls = _classes(pw, E)
    with pytest.raises(rmgb.RmError):
        rmgb.rm_qdt_plan_inspect(pw["e_thr"], pw["z"], pw["E_k"], E, cls, 0)
    with pytest.raises(rmgb.RmError):
        rmgb.rm_qdt_plan_inspect(pw["e_thr"], pw["z"], pw["E_k"], E[::-1].copy(), cls[::-1].copy(), -3)


def test_failed_nodes_are_left_out():
    """Node solves that fail are skipped: the weights use the remaining nodes
    of the segment (extrapolating beyond them), and a segment left without
    nodes has none (its energies fail), as in the oracle, where a node whose
    K_u cannot be formed is dropped."""
    pw = _pw()
    E = _grid(pw)
    cls = _classes(pw, E)
    first = rmgb.rm_qdt_plan_inspect(pw["e_thr"], pw["z"], pw["E_k"], E, cls, -9)
    nn = first["node_x"].size
    rng = np.random.default_rng(12)
    ok = (rng.uniform(size=nn) > 0.35).astype(np.int32)
    seg0 = first["node_seg"] == first["node_seg"][0]
    ok[seg0] = 0                               # the first segment loses every node
    lib = rmgb.rm_qdt_plan_inspect(pw["e_thr"], pw["z"], pw["E_k"], E, cls, -9, node_ok=ok)
    assert np.array_equal(lib["node_x"], first["node_x"])
    pl = qdt.plan(pw, E, -9, 0.0)
    for s, (i0, i1, cls_seg) in enumerate(pl["segments"]):
        idx = np.nonzero((lib["node_seg"] == s) & (ok != 0))[0]
        xs = lib["node_x"][idx]
        for m in range(i0, i1 + 1):
            if xs.size == 0:
                assert lib["node_a"][m] == -1
            elif xs.size == 1:
                assert lib["node_a"][m] == lib["node_b"][m] == idx[0]
            else:
                j, t = qdt.interpolation_weights(xs, pl["e_int"][m])
                assert (lib["node_a"][m], lib["node_b"][m], lib["t"][m]) == (idx[j], idx[j + 1], t)
    assert np.all(lib["node_a"][pl["segments"][0][0]:pl["segments"][0][1] + 1] == -1)
