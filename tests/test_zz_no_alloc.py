"""The allocation-free diagnostics entry point (cfs_diagnostics_static), for callers that cannot
allocate device memory, checked through the C ABI against cfs_diagnostics on the same states and
against the oracle's diagnostics.

Collected last on purpose: it runs after every other test, and also passes alone in a fresh
process."""
import numpy as np
import pytest

from paper_2506_03027_gb300 import cfs
from paper_2506_03027_gb300 import inputs as I

from gpu_util import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    return torch


def state_and_reference(torch, case, nsteps):
    """Advance the case with the regular solver; return its state as a CUDA tensor together with
    cfs_diagnostics (the existing entry point) of that state."""
    s = cfs.Solver(case)
    try:
        s.set_schedule()
        s.set_state(I.initial_state(case))
        s.step(nsteps)
        U = torch.empty((5, case.nz, case.ny, case.nx), dtype=torch.float64, device="cuda")
        s.get_state(U)
        ref = s.diagnostics()
    finally:
        s.close()
    return U, ref


def static_diag(torch, case, U):
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    cfs.cfs_diagnostics_static(U.data_ptr(), case.nx, case.ny, case.nz, (case.dx, case.dy, case.dz), case.order,
                               out.data_ptr(), stream)
    torch.cuda.current_stream().synchronize()
    return out.cpu().numpy()


def test_static_diagnostics_match_context_diagnostics_twice(torch):
    # first call: a ragged 3-D Navier-Stokes state; second call right after: a 2-D vortex state
    c3 = I.tgv_case(30, 3, "SA").replace(ny=28, nz=26)
    c3 = c3.replace(dt=I.cfl_dt(c3, I.tgv_state(c3), 0.3))
    U3, ref3 = state_and_reference(torch, c3, 4)
    c2 = I.vortex_case(48, 2)
    U2, ref2 = state_and_reference(torch, c2, 6)
    got3 = static_diag(torch, c3, U3)
    got2 = static_diag(torch, c2, U2)
    for got, ref in ((got3, ref3), (got2, ref2)):
        np.testing.assert_allclose(got[:7], ref[:7], rtol=1e-12, atol=1e-13)
        assert got[7] == ref[7] == 0.0
    # the scratch keeps the previous call's contents: calling again on the first state must not
    # be affected by the second call
    again = static_diag(torch, c3, U3)
    np.testing.assert_allclose(again[:7], ref3[:7], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("order", [4, 2])
def test_static_diagnostics_match_the_oracle(torch, order):
    """Against the FP64 oracle's diagnostics (the definition of the quantities) on states that no
    solver produced: the Taylor-Green field on a ragged grid and a seeded perturbation of it, with
    the CD4 and the CD2 vorticity."""
    from oracle import oracle as orc
    rng = np.random.default_rng(7 + order)
    c = I.tgv_case(30, 3, "SA", order=order).replace(ny=28, nz=26)
    U = I.tgv_state(c)
    for X in (U, U * (1.0 + 1e-3 * rng.standard_normal(U.shape))):
        got = static_diag(torch, c, torch.from_numpy(np.ascontiguousarray(X)).cuda())
        ref = orc.diagnostics(c, X)
        np.testing.assert_allclose(got[:7], ref[:7], rtol=1e-12, atol=1e-13 * np.abs(ref[:7]).max())
        assert got[7] == ref[7] == 0.0


def test_static_diagnostics_reject_oversized_grid(torch):
    U = torch.zeros((5, 1, 1, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(cfs.CfsError) as e:
        cfs.cfs_diagnostics_static(U.data_ptr(), 512, 256, 256, (1.0, 1.0, 1.0), 4, out.data_ptr())
    assert e.value.status == cfs.CFS_EINVAL
    assert "exceed" in str(e.value)


def test_static_diagnostics_flag_a_non_finite_state(torch):
    """A state with one NaN entry (made on the host): out[7] = 1 -- the asynchronous call returns
    no CFS_ENAN, callers read the flag -- while the totals of the other variables stay those of
    the finite state."""
    c = I.vortex_case(32, 2)
    U = I.vortex_state(c)
    Ud = torch.from_numpy(U).cuda()
    clean = static_diag(torch, c, Ud)
    assert clean[7] == 0.0
    Ubad = U.copy()
    Ubad[4, 0, 5, 7] = np.nan
    got = static_diag(torch, c, torch.from_numpy(Ubad).cuda())
    assert got[7] == 1.0
    np.testing.assert_array_equal(got[2:6], clean[2:6])   # rho, rho u, rho v, rho w untouched
    assert np.isnan(got[6])                                # the total of rho E carries the NaN


@pytest.mark.parametrize("case", ["order", "spacing", "null_U", "null_out", "null_spacing"])
def test_static_diagnostics_reject_bad_arguments(torch, case):
    """Invalid arguments are rejected on the host with CFS_EINVAL before any launch."""
    U = torch.zeros((5, 1, 4, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    up, op, sp, order = U.data_ptr(), out.data_ptr(), (1.0, 1.0, 1.0), 4
    if case == "order":
        order = 3
    elif case == "spacing":
        sp = (1.0, 0.0, 1.0)
    elif case == "null_U":
        up = 0
    elif case == "null_out":
        op = 0
    if case == "null_spacing":
        st = cfs.load().cfs_diagnostics_static(cfs.ctypes.c_void_p(up), 4, 4, 1, None, order,
                                               cfs.ctypes.c_void_p(op), None, None, 0)
        assert st == cfs.CFS_EINVAL
        return
    with pytest.raises(cfs.CfsError) as e:
        cfs.cfs_diagnostics_static(up, 4, 4, 1, sp, order, op)
    assert e.value.status == cfs.CFS_EINVAL
