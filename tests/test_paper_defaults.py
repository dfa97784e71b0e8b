"""The library's defaults against the defaults the paper prints for the
corresponding namelist variables (tests/golden/paper_namelist_defaults.txt,
Sections "namelist stgf General calculation parameters", "namelist stgf MQDT
variables" and "namelist stgf Advanced options")."""
import os

import numpy as np

from paper_1909_07321_gb300 import rmgb, synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_namelist_defaults.txt")


def _defaults():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, value = line.split()[:2]
        out[name] = float(value)
    return out


def test_options_mirror_the_paper_defaults():
    d = _defaults()
    o = rmgb.rm_default_opts()
    assert o.fnumin == d["fnumin"]
    assert d["iomsw"] == 1 and o.nu_margin == 0.1      # full MQDT: nu < l + 0.1 omitted
    _, A, r1, steps, _ = synth.workload_multipole(8)
    assert A.shape[0] == d["lmx"]                        # dipole and quadrupole
    assert d["ipert"] == 0 and d["ieq"] == -1 and d["mzpts"] == 3201
    assert 1000 <= steps <= d["mzpts"] and np.isfinite(r1)
