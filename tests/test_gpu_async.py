"""Streamed read-out of Omega (rm_collision_strengths_async) on the GPU: every
copy equals the blocking read-out of the same step, bit for bit, while the
next steps accumulate into the other device buffer; without reset the next
step waits for the copy."""
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


@pytest.mark.parametrize("precision", [0, 2])
def test_streamed_readout_equals_blocking(rt, precision):
    torch, rmgb = rt
    pws, E = synth.workload_small(2000)
    pw = pws[0]
    E2 = E[::-1].copy()                  # a second grid, so that the buffers differ
    ntri = pw["n_levels"] * (pw["n_levels"] + 1) // 2
    with rmgb.Context(precision=precision) as ctx:
        ctx.load_pw(0, pw)
        ref = []
        for grid in (E, E2):
            ctx.solve_energies(0, grid)
            ref.append(ctx.collision_strengths(reset=True))
        bufs = [torch.empty((E.size, ntri), dtype=torch.float64, pin_memory=True).numpy() for _ in range(5)]
        for b in bufs:
            b.fill(-1.0)
        for i in range(5):
            ctx.solve_energies(0, E if i % 2 == 0 else E2)
            ctx.collision_strengths_async(bufs[i], reset=True)
            assert rmgb.rm_grid_shape(ctx.h) == (0, 0)
        ctx.sync()
        for i in range(5):
            assert np.array_equal(bufs[i], ref[i % 2]), i


def test_readout_without_reset_waits(rt):
    """reset = 0: the copy holds the accumulator as it was when the call was
    made; the next solve, which adds onto the same grid, waits for it."""
    torch, rmgb = rt
    pws, E = synth.workload_small(500)
    pw = pws[0]
    ntri = pw["n_levels"] * (pw["n_levels"] + 1) // 2
    with rmgb.Context() as ctx:
        ctx.load_pw(0, pw)
        ctx.solve_energies(0, E)
        one = ctx.collision_strengths()
        buf = torch.empty((E.size, ntri), dtype=torch.float64, pin_memory=True).numpy()
        buf.fill(-1.0)
        ctx.collision_strengths_async(buf, reset=False)
        ctx.solve_energies(0, E)             # accumulates onto the same grid
        two = ctx.collision_strengths()
        ctx.sync()
    assert np.array_equal(buf, one)
    np.testing.assert_allclose(two, 2.0 * one, rtol=1e-14, atol=0)


def test_async_needs_a_grid(rt):
    torch, rmgb = rt
    with rmgb.Context() as ctx:
        arr = np.zeros((4, 4))
        with pytest.raises(ValueError):
            ctx.collision_strengths_async(arr)
        assert rmgb.lib().rm_collision_strengths_async(ctx.h, arr.ctypes.data, 0) == rmgb.RM_EINVAL
        assert rmgb.lib().rm_collision_strengths_async(ctx.h, None, 0) == rmgb.RM_EINVAL
