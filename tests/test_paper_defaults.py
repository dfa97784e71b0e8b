"""The library's defaults against the defaults the paper prints for the
corresponding namelist variables (tests/golden/paper_namelist_defaults.txt,
Sections "namelist stgf MQDT variables" and "namelist stgf Advanced options").
Every row is compared with a value the library itself produces (an option
default, the multipole workload, or the host plan of the coarse-mesh
interpolation), so a changed library default fails here."""
import os

import numpy as np

from paper_1909_07321_gb300 import rmgb, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_namelist_defaults.txt")


def _rows():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, paper, lib = line.split()[:3]
        out[name] = (float(paper), float(lib))
    return out


def test_golden_rows():
    assert set(_rows()) == {"fnumin", "iomsw", "lmx", "ieq"}


def test_fnumin_and_iomsw_are_the_option_defaults():
    d = _rows()
    o = rmgb.rm_default_opts()
    assert o.fnumin == d["fnumin"][0] == d["fnumin"][1]
    # iomsw = 1 (full MQDT) leaves out closed channels with nu < l + 0.1
    assert d["iomsw"][0] == 1 and o.nu_margin == d["iomsw"][1]


def test_lmx_is_the_multipole_workloads_order():
    d = _rows()
    _, A, r1, steps, _ = synth.workload_multipole(8)
    assert A.shape[0] == d["lmx"][0] == d["lmx"][1]
    assert np.isfinite(r1) and steps >= 2


def test_ieq_minus_one_makes_every_energy_a_node():
    """ieq = -1 in the library's own host plan: every fine energy is a node
    and is interpolated from itself alone (all weight on its own node), i.e.
    the plain MQDT solve."""
    d = _rows()
    ieq = int(d["ieq"][1])
    assert ieq == d["ieq"][0]
    pw = synth.random_pw(4711, 4, 60, z=2.0, a=10.0, e_max=1.8, sigma=0.1, l_max=3)
    E = synth.midpoint_grid(0.05, 2.1, 200)
    cls = np.where(E[:, None] > pw["e_thr"][None, :], 0, 1).astype(np.int8)
    pl = rmgb.rm_qdt_plan_inspect(pw["e_thr"], pw["z"], pw["E_k"], E, cls, ieq, 0.0)
    assert pl["node_x"].size == E.size
    assert np.array_equal(pl["node_x"], E)
    own = np.arange(E.size)
    a, b, t = pl["node_a"], pl["node_b"], pl["t"]
    assert np.all(((a == own) & (t == 0.0)) | ((b == own) & (t == 1.0)))
