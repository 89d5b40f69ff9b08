"""Runtime features through the C ABI: autotuner launch shapes (results
independent of the choice), CUDA-graph replay of RK4 steps, kernel timing,
the host-buffer entry point."""
import numpy as np
import pytest

from paper_1410_1764_gb300 import synth
from helpers import scaled_err, to_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1410_1764_gb300 import api as A
    A.lib()
    return A


@pytest.mark.parametrize("kind,dims", [("bssn", (19, 13, 9)), ("wave", (37, 21, 11)), ("varc", (24, 16, 8))])
def test_every_launch_shape_gives_identical_results(api, orc, kind, dims):
    nx, ny, nz = dims
    rng = np.random.default_rng(1)
    if kind == "bssn":
        K, g = api.BSSN, 3
        st = synth.pad(synth.BSSN_FLAT[:, None, None, None] + 1e-2 * rng.standard_normal((24, nz, ny, nx)), g)
    else:
        K, g = (api.WAVE if kind == "wave" else api.WAVE_VARC), 2
        st = synth.pad(rng.standard_normal((2, nz, ny, nx)), g)
    orc.fill_ghosts(st, g)
    sysm = api.make_system(K, nx, ny, nz, 1.0 / nx)
    if K == api.WAVE_VARC:
        sysm.set_speed(to_gpu(synth.pad(1.0 + 0.1 * rng.uniform(-1, 1, (nz, ny, nx)), g)[0]))
    n = api.lib().chemora_variant_count(K)
    assert n >= 4
    T = to_gpu(st)
    outs = []
    for v in range(n):
        sysm.variant(v)
        outs.append(to_np(sysm.rhs(T)))
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    v, shape, ms = sysm.autotune(T)
    assert 0 <= v < n and ms > 0 and sysm.variant()[0] == v


def test_graph_replay_equals_plain_steps(api, orc):
    n, g = 24, 3
    st, h = synth.bssn_noise(n, n, n, g, seed=4)
    sysm = api.make_system(api.BSSN, n, n, n, h)
    a = to_gpu(st)
    b = to_gpu(st)
    sysm.rk4_step(a, 0.25 * h, 5)           # graph replay
    for _ in range(5):
        sysm.rk4_step(b, 0.25 * h, 1)       # plain launches
    assert np.array_equal(to_np(a), to_np(b))
    sysm.rk4_step(a, 0.125 * h, 3)          # new dt: re-capture
    for _ in range(3):
        sysm.rk4_step(b, 0.125 * h, 1)
    assert np.array_equal(to_np(a), to_np(b))


def test_profile_counts_stage_launches(api):
    n = 16
    st, h = synth.bssn_noise(n, n, n, 3, seed=1)
    sysm = api.make_system(api.BSSN, n, n, n, h)
    t = to_gpu(st)
    sysm.profile(True)
    sysm.rk4_step(t, 0.25 * h, 3)
    ms, launches = sysm.profile_read()
    assert launches == 12 and ms > 0
    sysm.profile(False)


def test_host_buffer_step(api, orc):
    import torch
    n, g = 20, 2
    y0, h = synth.gaussian_pulses(n, g, seed=2, width=0.1)
    sysm = api.make_system(api.WAVE, n, n, n, h)
    host = torch.from_numpy(y0.copy()).pin_memory()
    sysm.rk4_step_host(host, 0.25 * h, 4)
    want = orc.rk4(orc.WAVE, y0, g, h, 0.25 * h, 4)
    assert scaled_err(host.numpy(), want, g) <= 1e-10


def test_nonfinite_sentinel(api):
    n = 12
    st, h = synth.bssn_noise(n, n, n, 3, seed=1)
    sysm = api.make_system(api.BSSN, n, n, n, h)
    t = to_gpu(st)
    assert sysm.nonfinite(t) == 0
    t[5, 3 + 4, 3 + 2, 3 + 7] = float("nan")
    t[9, 3 + 1, 3 + 1, 3 + 1] = float("inf")
    t[0, 0, 0, 0] = float("nan")  # a ghost value is not counted
    assert sysm.nonfinite(t) == 2
    assert b"non-finite" in api.lib().chemora_last_error()


def test_corrupt_worklist_reported_not_faulted(api):
    """A work item naming a patch outside the table is skipped by the
    persistent kernel and reported as an error; the context stays usable."""
    import torch
    from paper_1410_1764_gb300._native import ChemoraError
    dims = [(12, 9, 7), (16, 16, 16)]
    b = api.Batch(dims, 2, 1.0 / 32, kind=api.WAVE)
    assert api.lib().chemora_patches_inject_fault(b.handle, 3) == 0
    with pytest.raises(ChemoraError) as ei:
        b.step(0.01, 1, mode=0)
    assert "outside the patch table" in str(ei.value)
    del b
    # the device still works
    x = torch.ones(4, device="cuda", dtype=torch.float64)
    assert float(x.sum()) == 4.0


def test_persistent_time_limit_reported(api):
    """A persistent stage launch that passes its time limit stops taking work
    items and the step returns CHEMORA_ETIMEOUT (the limit here is a few SM
    cycles, so every block gives up at its first item); the context stays
    usable, and with the limit removed, or generous, the batch steps exactly
    as a batch that never had one."""
    import torch
    from paper_1410_1764_gb300._native import ChemoraError, ETIMEOUT
    dims = [(12, 9, 7), (16, 16, 16), (20, 5, 9)]
    rng = np.random.default_rng(4)
    init = [rng.standard_normal((2, d[2] + 4, d[1] + 4, d[0] + 4)) for d in dims]

    def fresh():
        b = api.Batch(dims, 2, 1.0 / 32, kind=api.WAVE)
        for p, y in enumerate(init):
            b.state(p).copy_(torch.from_numpy(y))
        return b

    ref = fresh()
    ref.step(0.01, 2, mode=0)
    want = [to_np(ref.state(p)) for p in range(len(dims))]
    b = fresh()
    b.set_time_limit(1e-9)
    with pytest.raises(ChemoraError) as ei:
        b.step(0.01, 1, mode=0)
    assert ei.value.code == ETIMEOUT and "time limit" in str(ei.value)
    x = torch.ones(4, device="cuda", dtype=torch.float64)
    assert float(x.sum()) == 4.0
    for limit in (0.0, 10.0):
        b = fresh()
        b.set_time_limit(limit)
        b.step(0.01, 2, mode=0)
        for p in range(len(dims)):
            assert np.array_equal(to_np(b.state(p)), want[p])


@pytest.mark.parametrize("dims,amp", [((32, 9, 7), 3e-2), ((64, 8, 10), 1e-10), ((64, 12, 6), 3e-2), ((32, 16, 6), 3e-2)])
def test_xshare_variants_match_oracle(api, orc, dims, amp):
    """The x-sharing BSSN kernels (neighbour lanes supply x differences and
    the rows of the xy/xz mixed derivatives) against the oracle and the
    direct kernel, on grids whose nx is a multiple of the warp width."""
    nx, ny, nz = dims
    g, h = 3, 1.0 / nx
    rng = np.random.default_rng(21)
    st = synth.pad(synth.BSSN_FLAT[:, None, None, None] + amp * rng.standard_normal((24, nz, ny, nx)), g)
    orc.fill_ghosts(st, g)
    want = orc.bssn_rhs(st, g, h)
    sysm = api.make_system(api.BSSN, nx, ny, nz, h)
    T = to_gpu(st)
    base = to_np(sysm.rhs(T))
    nvar = api.lib().chemora_variant_count(api.BSSN)
    xs = [v for v in range(nvar) if v >= 8]
    assert xs
    for v in xs:
        _, shape = sysm.variant(v)
        if nx % shape[0]:
            continue
        got = to_np(sysm.rhs(T))
        assert scaled_err(got, want, g) <= 1e-12
        assert scaled_err(got, base, g) <= 1e-12
        y = orc.rk4(orc.BSSN, st, g, h, 0.25 * h, 3)
        t2 = to_gpu(st)
        sysm.rk4_step(t2, 0.25 * h, 3)
        assert scaled_err(to_np(t2), y, g) <= 1e-10


def test_xshare_falls_back_on_ragged_x(api):
    n = 19
    st, h = synth.bssn_noise(n, 10, 8, 3, seed=5)
    sysm = api.make_system(api.BSSN, n, 10, 8, h)
    T = to_gpu(st)
    sysm.fill_ghosts(T)
    sysm.variant(0)
    a = to_np(sysm.rhs(T))
    sysm.variant(api.lib().chemora_variant_count(api.BSSN) - 1)
    b = to_np(sysm.rhs(T))
    assert np.array_equal(a, b)
