"""The pressure solve that allocates nothing (erem_pressure_solve_static),
for callers that cannot call cudaMalloc: its work space is a static device
array inside the library.  Checked through the C ABI against the context
entry point pressure_solve and against the oracle's direct solve on the same
inputs, on consecutive calls that share (and inherit) the static array,
within the pressure tolerance the solver tests use; the second call must
leave the device's free memory unchanged.  This file is collected last on
purpose."""
import numpy as np
import pytest

from oracle import fv
from oracle import timestep as ts

pytestmark = pytest.mark.gpu

PRESSURE_TOL = 1e-12  # the CG tolerance of tests/test_gpu_solvers.py


def _bound(g, ph, lnk, T):
    # error bound of a CG result stopped at PRESSURE_TOL (as in test_gpu_solvers.py)
    A, b = fv.pressure_system(g, ph, lnk, T)
    smin = np.linalg.svd(A.toarray(), compute_uv=False).min()
    p = np.linalg.solve(A.toarray(), b)
    return 10.0 * PRESSURE_TOL * np.linalg.norm(b) / smin / np.linalg.norm(p)


def _case(dim, nx, ny, nz, fm, seed):
    rng = np.random.default_rng(seed)
    g = fv.Grid(dim, nx, ny, nz)
    ph = fv.Physics(head_left=1.0, head_right=0.25, fluid_model=fm)
    lnk = rng.normal(0, 1.2, g.n)
    T = rng.uniform(20, 80, g.n) if fm else None
    return g, ph, lnk, T


@pytest.mark.parametrize("dims", [(2, 40, 30, 1, 1), (3, 12, 11, 9, 0)])
def test_static_pressure_solve_matches_pressure_solve(dims):
    import torch

    import paper_1209_5553_gb300 as E

    assert torch.cuda.is_available()
    dim, nx, ny, nz, fm = dims
    g, ph, lnk, T = _case(dim, nx, ny, nz, fm, seed=nx)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    guess = fv.linear_head_guess(g, ph)
    phys = E.Physics(1.0, 1.0, ph.head_left, ph.head_right, 80.0, fm)
    with E.Context(dim, nx, ny, nz, physics=phys) as ctx:
        ctx.set_pressure_precond(1)   # the static solve is the Jacobi CG
        p_ref = t(guess)
        st_ref = ctx.pressure_solve(t(lnk), t(T) if fm else None, p_ref, tol=PRESSURE_TOL)
        ref = p_ref.cpu().numpy()
    bound = _bound(g, ph, lnk, T)
    direct = ts.pressure_solve_direct(g, ph, lnk, T)
    grid = E.erem_grid(dim, nx, ny, nz, 1.0, 1.0, 1.0)
    args = [(t(guess), t(lnk), t(T) if fm else None) for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):  # two calls in a row share the static work space
        p, lk, Tt = args[call]
        free0 = torch.cuda.mem_get_info()[0]
        st = E.erem_pressure_solve_static(grid, phys.c(), lk, Tt, p, tol=PRESSURE_TOL)
        free1 = torch.cuda.mem_get_info()[0]
        if call == 1:  # the first call may load the module (and place the array)
            assert free1 == free0
        got = p.cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= bound, call
        assert np.linalg.norm(got - direct) / np.linalg.norm(direct) <= bound, call
        assert st.lin_resid <= PRESSURE_TOL
        assert st.lin_iters == st_ref.lin_iters
        assert st.flux_in == pytest.approx(st_ref.flux_in, rel=1e-10)
        assert st.vmax == pytest.approx(st_ref.vmax, rel=1e-10)
        assert st.t_ms > 0.0


def test_static_pressure_solve_rejects_grids_beyond_its_limit():
    import torch

    import paper_1209_5553_gb300 as E

    assert torch.cuda.is_available()
    grid = E.erem_grid(2, 300, 300, 1, 1.0, 1.0, 1.0)  # 90,000 cells > 65,536
    x = torch.zeros(300 * 300, dtype=torch.float64, device="cuda")
    with pytest.raises(E.EremError) as ei:
        E.erem_pressure_solve_static(grid, E.Physics().c(), x, None, x.clone())
    assert ei.value.status == E.EREM_EINVAL
    # host arrays are refused too: staging them would allocate
    small = E.erem_grid(2, 8, 8, 1, 1.0, 1.0, 1.0)
    with pytest.raises(E.EremError) as ei:
        E.erem_pressure_solve_static(small, E.Physics().c(), np.zeros(64), None, np.zeros(64))
    assert ei.value.status == E.EREM_EINVAL
    # page-locked host memory too, although the GPU could address it
    pinned = torch.zeros(64, dtype=torch.float64).pin_memory()
    dev = torch.zeros(64, dtype=torch.float64, device="cuda")
    for lk, p in ((pinned, dev), (dev, pinned.clone().pin_memory())):
        with pytest.raises(E.EremError) as ei:
            E.erem_pressure_solve_static(small, E.Physics().c(), lk, None, p)
        assert ei.value.status == E.EREM_EINVAL
