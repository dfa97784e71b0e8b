"""Bounded device waits of the tensor-core formation kernels: with the wait
self-test on (rm_set_wait_probe), every CTA waits on an mbarrier that nothing
arrives at, before it allocates tensor memory or issues any copy or MMA; the
wait gives up after its limit and the host reads RM_ETIMEOUT. The context
stays usable: with the self-test off, the same solve gives the result of a
fresh context."""
import numpy as np
import pytest

from paper_1909_07321_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_07321_gb300 import build, rmgb
    build.build()
    return torch, rmgb


@pytest.mark.parametrize("form", [1, 2], ids=["pair-operand", "per-energy"])
def test_wait_gives_up_and_context_recovers(rt, form):
    torch, rmgb = rt
    pws, E = synth.workload_64ch(2000)
    pw = pws[0]
    with rmgb.Context(precision=2, formulation=form) as ref_ctx:
        ref_ctx.load_pw(0, pw)
        ref_ctx.solve_energies(0, E)
        ref = ref_ctx.collision_strengths()
    with rmgb.Context(precision=2, formulation=form) as ctx:
        ctx.load_pw(0, pw)
        ctx.set_wait_probe(1_000_000)          # 1 ms
        ctx.solve_energies(0, E)
        with pytest.raises(rmgb.RmError) as ei:
            ctx.sync()
        assert ei.value.code == rmgb.RM_ETIMEOUT
        ctx.set_wait_probe(0)
        ctx.collision_strengths(reset=True)    # the flag was cleared by the failed sync
        ctx.solve_energies(0, E)
        om = ctx.collision_strengths()
    np.testing.assert_array_equal(om, ref)


def test_probe_limit_checked(rt):
    torch, rmgb = rt
    with rmgb.Context(precision=2) as ctx:
        with pytest.raises(rmgb.RmError):
            ctx.set_wait_probe(20_000_000_000)
