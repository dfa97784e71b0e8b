"""Every energy is solved on its own: a slice of the energies, from a single
energy to slices that end one short of, on, and one past the 128-energy
formation tile, gives bit for bit the K, open counts, statuses and Omega rows
that the same energies get inside one call over all of them (Section
"Overview": R, K and T are per (partial wave, energy); Section "Glossary of
terms": Omega per energy). This covers the ragged tiles of the tensor-core
formation, the solvers' per-energy CTAs and the longest-first CTA order of
the global-memory solver, in the mixed path (bf16x3 formation, FP32 solve)."""
import numpy as np
import pytest

from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu

SLICES = [(0, 1), (777, 1), (5, 127), (300, 128), (1000, 129), (1700, 300)]


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    return torch, rmgb


def _solve(rt, pw, E, solver):
    torch, rmgb = rt
    n = pw["W"].shape[0]
    with rmgb.Context(precision=rmgb.RM_BF16X3, solver=solver, solve_precision=rmgb.RM_FP32) as ctx:
        ctx.load_pw(0, pw)
        Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
        K = torch.zeros((E.size, n * n), dtype=torch.float64, device="cuda")
        no = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        st = torch.zeros(E.size, dtype=torch.int32, device="cuda")
        ctx.solve_energies(0, Ed, rmgb.RM_DIRECT, K, no, st)
        om = ctx.collision_strengths()
    return K.cpu().numpy(), no.cpu().numpy(), st.cpu().numpy(), om


@pytest.mark.parametrize("solver", ["auto", "large"])
def test_energy_slices_equal_the_full_call(rt, solver):
    _, rmgb = rt
    sv = rmgb.RM_SOLVER_AUTO if solver == "auto" else rmgb.RM_SOLVER_LARGE
    pws, E = synth.workload_64ch(2000)
    pw = pws[0]
    K, no, st, om = _solve(rt, pw, E, sv)
    assert (st == rmgb.RM_OK).sum() > 1900
    for o, m in SLICES:
        Ks, nos, sts, oms = _solve(rt, pw, E[o:o + m], sv)
        assert np.array_equal(sts, st[o:o + m]), (o, m)
        assert np.array_equal(nos, no[o:o + m]), (o, m)
        assert np.array_equal(Ks, K[o:o + m]), (o, m)
        assert np.array_equal(oms, om[o:o + m]), (o, m)
