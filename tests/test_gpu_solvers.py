"""GPU parity of the solvers beside the Leja path: the pressure solve
(FP64 CG, Jacobi or with the FP32 Chebyshev polynomial preconditioner) and
the Rosenbrock-type steps ROSM(1), ROSM(1/2) and
ROS2(1) (Jacobi BiCGSTAB stage solves, FP64), against the oracle's direct
solves; plus the error paths of the C ABI.

Linear-solver tolerances are derived from the stopping rule: a relative
residual below tol bounds the error by tol * ||b|| * ||A^{-1}||_2, with
||A^{-1}||_2 taken from the oracle's own matrix (dense SVD on these small
grids); a factor 10 covers the gap between the recursive and the true
residual."""
import numpy as np
import pytest

import cases as C
from oracle import fv, timestep as ts

pytestmark = pytest.mark.gpu

PRESSURE_TOL = 1e-12   # CG stopping tolerance used in these tests
STAGE_TOL = 1e-12      # BiCGSTAB stopping tolerance


@pytest.fixture(scope="module")
def E():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1209_5553_gb300 as E

    return E


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def pressure_error_bound(A, b, p, tol):
    smin = np.linalg.svd(A.toarray(), compute_uv=False).min()
    return 10.0 * tol * np.linalg.norm(b) / smin / np.linalg.norm(p)


@pytest.mark.parametrize("deg", [1, 16, 0])
@pytest.mark.parametrize("dim,nx,ny,nz,fm", [(2, 32, 24, 1, 0), (2, 33, 17, 1, 1), (3, 10, 9, 7, 0)])
def test_pressure_solve_matches_direct_solution(E, dim, nx, ny, nz, fm, deg):
    rng = np.random.default_rng(nx + ny)
    g = fv.Grid(dim, nx, ny, nz)
    ph = fv.Physics(head_left=1.3, head_right=-0.2, fluid_model=fm)
    lnk = rng.normal(0, 1.5, g.n)
    T = rng.uniform(20, 80, g.n) if fm else None
    A, b = fv.pressure_system(g, ph, lnk, T)
    p_ref = ts.pressure_solve_direct(g, ph, lnk, T)
    p0 = fv.linear_head_guess(g, ph)
    with E.Context(dim, nx, ny, nz, physics=E.Physics(1, 1, 1.3, -0.2, 80.0, fm)) as ctx:
        ctx.set_pressure_precond(deg)
        p = _t(p0)
        st = ctx.pressure_solve(_t(lnk), _t(T) if fm else None, p, tol=PRESSURE_TOL, maxit=20000)
        got = p.cpu().numpy()
    assert st.lin_resid <= PRESSURE_TOL
    err = np.linalg.norm(got - p_ref) / np.linalg.norm(p_ref)
    assert err <= pressure_error_bound(A, b, p_ref, PRESSURE_TOL), err
    # net inflow and largest face speed from the oracle's fluxes
    vx, vy, vz = fv.darcy_fluxes(g, ph, lnk, p_ref, T)
    width = g.ly * (g.lz if dim == 3 else 1.0)
    assert st.flux_in == pytest.approx(vx[:, :, 0].sum(), rel=1e-8)
    a = g.face_area
    vmax = max(np.abs(vx).max() / a[0], np.abs(vy).max() / a[1],
               np.abs(vz).max() / a[2] if vz is not None else 0.0)
    assert st.vmax == pytest.approx(vmax, rel=1e-8)
    assert width > 0


def test_polynomial_preconditioner_cuts_the_iterations(E):
    # a heterogeneous 3D field (sigma 2): every degree reaches the direct
    # solution within the residual bound; the outer iterations fall roughly
    # in proportion to the degree (at least by degree / 3 up to 16; on this
    # small grid the count levels off near 14 beyond that)
    rng = np.random.default_rng(5)
    g = fv.Grid(3, 24, 20, 16)
    ph = fv.Physics(head_left=1.0, head_right=0.0, fluid_model=0)
    lnk = rng.normal(0, 2.0, g.n)
    A, b = fv.pressure_system(g, ph, lnk, None)
    p_ref = ts.pressure_solve_direct(g, ph, lnk, None)
    bound = pressure_error_bound(A, b, p_ref, PRESSURE_TOL)
    iters = {}
    with E.Context(3, g.nx, g.ny, g.nz, physics=E.Physics(1, 1, 1.0, 0.0, 80.0, 0)) as ctx:
        for deg in (1, 2, 5, 16, 64):
            ctx.set_pressure_precond(deg)
            p = _t(np.zeros(g.n))
            st = ctx.pressure_solve(_t(lnk), None, p, tol=PRESSURE_TOL, maxit=20000)
            err = np.linalg.norm(p.cpu().numpy() - p_ref) / np.linalg.norm(p_ref)
            assert st.lin_resid <= PRESSURE_TOL and err <= bound, (deg, err, bound)
            iters[deg] = st.lin_iters
        for bad in (-1, 65):
            with pytest.raises(E.EremError) as ei:
                ctx.set_pressure_precond(bad)
            assert ei.value.status == E.EREM_EINVAL
    for deg in (2, 5, 16):
        assert iters[deg] * deg / 3 <= iters[1], iters
    assert iters[64] <= iters[16], iters


@pytest.mark.parametrize("dims", [(2, 96, 80, 1), (2, 67, 41, 1), (3, 40, 33, 21)])
def test_multigrid_preconditioner(E, dims):
    # degree 0: the multigrid V-cycle; the direct solution within the
    # residual bound in a few tens of outer iterations on sigma = 2 fields,
    # with a fraction of the fine-level work of the degree-32 polynomial; odd
    # sizes coarsen with ragged aggregates
    dim, nx, ny, nz = dims
    rng = np.random.default_rng(nx)
    g = fv.Grid(dim, nx, ny, nz)
    ph = fv.Physics(head_left=1.0, head_right=0.0, fluid_model=0)
    lnk = rng.normal(0, 2.0, g.n)
    A, b = fv.pressure_system(g, ph, lnk, None)
    p_ref = ts.pressure_solve_direct(g, ph, lnk, None)
    bound = pressure_error_bound(A, b, p_ref, PRESSURE_TOL) if g.n < 6000 else None
    iters = {}
    with E.Context(dim, nx, ny, nz, physics=E.Physics(1, 1, 1.0, 0.0, 80.0, 0)) as ctx:
        for deg in (32, 0):
            ctx.set_pressure_precond(deg)
            p = _t(np.zeros(g.n))
            st = ctx.pressure_solve(_t(lnk), None, p, tol=PRESSURE_TOL, maxit=20000)
            got = p.cpu().numpy()
            assert st.lin_resid <= PRESSURE_TOL, deg
            err = np.linalg.norm(got - p_ref) / np.linalg.norm(p_ref)
            r = np.linalg.norm(A @ got - b) / np.linalg.norm(b)
            assert r < 10 * PRESSURE_TOL, (deg, r)
            if bound is not None:
                assert err <= bound, (deg, err, bound)
            iters[deg] = st.lin_iters
        with pytest.raises(E.EremError) as ei:
            ctx.set_pressure_multigrid(0, 1.8)
        assert ei.value.status == E.EREM_EINVAL
        with pytest.raises(E.EremError) as ei:
            ctx.set_pressure_multigrid(3, 2.0)
        assert ei.value.status == E.EREM_EINVAL
    # fine-level work: 2 nu + 2 sweep-sized passes per V-cycle against 32
    # sweeps per polynomial application
    assert iters[0] < 40 and iters[0] * (2 * 3 + 2) < 0.5 * iters[32] * 32, iters


@pytest.mark.parametrize("dims", [(2, 1, 1, 1), (2, 7, 1, 1), (2, 1, 9, 1), (2, 3, 2, 1),
                                  (3, 1, 1, 5), (3, 2, 3, 2)])
def test_multigrid_on_degenerate_grids(E, dims):
    # single cells, single rows and tiny boxes: the multigrid levels coarsen
    # to one cell; pressure (CG) and a ROS2(1) step (stage BiCGSTAB) against
    # the direct solutions
    dim, nx, ny, nz = dims
    case = C.random_case(dim, nx, ny, nz, seed=nx * 7 + ny, fluid_model=0)
    g = case.grid
    ph = fv.Physics(head_left=1.0, head_right=0.0, fluid_model=0)
    p_ref = ts.pressure_solve_direct(g, ph, case.lnk, None)
    ref = ts.ros2_step(case.problem(case.T0), case.T0, 0.05)
    with E.Context(dim, nx, ny, nz, physics=case.gpu_physics()) as ctx:
        p = _t(np.zeros(g.n))
        st = ctx.pressure_solve(_t(case.lnk), None, p, tol=PRESSURE_TOL, maxit=2000)
        assert st.lin_resid <= PRESSURE_TOL
        assert np.max(np.abs(p.cpu().numpy() - p_ref)) <= 1e-9 * max(1.0, np.max(np.abs(p_ref)))
        T = _t(case.T0)
        ctx.rosm_step(T, 0.05, E.EREM_ROS2, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam),
                      lin_tol=STAGE_TOL, maxit=2000)
        got = T.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-8 * max(1.0, np.max(np.abs(ref - case.T0)))


def test_pressure_solve_host_pointers_and_maxit(E):
    g = fv.Grid(2, 20, 20)
    ph = fv.Physics()
    lnk = np.random.default_rng(1).normal(0, 1, g.n)
    p_ref = ts.pressure_solve_direct(g, ph, lnk)
    with E.Context(2, 20, 20) as ctx:
        p = fv.linear_head_guess(g, ph).copy()
        ctx.pressure_solve(lnk.copy(), None, p, tol=PRESSURE_TOL)
        assert np.max(np.abs(p - p_ref)) < 1e-9
        p2 = np.zeros(g.n)
        with pytest.raises(E.EremError) as ei:
            ctx.pressure_solve(lnk.copy(), None, p2, tol=1e-14, maxit=2)
        assert ei.value.status == E.EREM_ENOTCONV


def _rosm_case():
    case = C.random_case(2, 18, 14, seed=21, fluid_model=1)
    return case


@pytest.mark.parametrize("scheme", ["rosm1", "rosm_half", "ros2", "ros3p"])
def test_rosm_step_matches_oracle(E, scheme):
    case = _rosm_case()
    prob = case.problem(case.T0)
    tau = 0.05
    gam = {"rosm1": 1.0, "rosm_half": 0.5, "ros2": ts.ROS2_GAMMA, "ros3p": ts.ROS3P_GAMMA}[scheme]
    emb = None
    if scheme == "ros2":
        ref, emb = ts.ros2_step(prob, case.T0, tau, embedded=True)
    elif scheme == "ros3p":
        ref, emb = ts.ros3p_step(prob, case.T0, tau, embedded=True)
    else:
        ref = ts.rosm_step(prob, case.T0, tau, gam)
    A = ts.stage_matrix(prob.J(case.T0), tau, gam)
    smin = np.linalg.svd(A.toarray(), compute_uv=False).min()
    G = prob.G(case.T0)
    inc = ref - case.T0
    # each stage: error <= 10 tol ||rhs|| / smin, rhs ~ G; scaled by the b_i or 1/gamma
    bound = 10 * STAGE_TOL * np.linalg.norm(G) / smin * 3.0 / np.linalg.norm(inc)
    code = {"rosm1": E.EREM_ROSM1, "rosm_half": E.EREM_ROSM_HALF, "ros2": E.EREM_ROS2,
            "ros3p": E.EREM_ROS3P}[scheme]
    with E.Context(2, case.grid.nx, case.grid.ny, physics=case.gpu_physics()) as ctx:
        T = _t(case.T0)
        st = ctx.rosm_step(T, tau, code, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam),
                           lin_tol=STAGE_TOL, maxit=5000)
        got = T.cpu().numpy()
    assert st.lin_iters > 0 and st.lin_resid <= STAGE_TOL
    err = np.linalg.norm((got - case.T0) - inc) / np.linalg.norm(inc)
    assert err <= max(bound, 1e-12), (err, bound)
    if emb is not None:
        # the embedded difference: RMS of y - y_hat (stage errors as above)
        want = np.sqrt(np.mean((ref - emb) ** 2))
        assert st.err_est == pytest.approx(want, rel=max(1e-9, 100 * bound * np.linalg.norm(inc)
                                                          / np.linalg.norm(ref - emb)))
    else:
        assert st.err_est == 0.0


@pytest.mark.parametrize("scheme", ["ros2", "ros3p"])
def test_adaptive_rosenbrock_matches_oracle(E, scheme):
    # the GPU controller takes the oracle's accept/reject decisions and step
    # lengths (the error estimates differ by the stage-solve tolerance only);
    # nonlinear fluid laws (ROS3p's estimate vanishes on the linear model),
    # the Darcy fluxes re-evaluated at T^n every step on both sides
    case = C.random_case(2, 16, 12, seed=23, fluid_model=1)
    t_end, dt0, tol = 0.05, 1e-3, 1e-5
    ref = ts.ros_integrate(lambda T: case.problem(T), case.T0, t_end, dt0, scheme, tol, tol)
    assert ref.rejected + len(ref.dts) > 5
    code = {"ros2": E.EREM_ROS2, "ros3p": E.EREM_ROS3P}[scheme]
    with E.Context(2, case.grid.nx, case.grid.ny, physics=case.gpu_physics()) as ctx:
        T = _t(case.T0)
        ctx.set_state(T, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), dt0)
        st, dts = ctx.rosm_integrate(T, t_end, dt0, code, tol, tol, lin_tol=1e-13, maxit=20000)
        got = T.cpu().numpy()
        assert st.rejected == ref.rejected and st.accepted == len(ref.dts)
        assert np.allclose(dts, ref.dts, rtol=1e-7, atol=0)
        assert st.t_reached == t_end and abs(dts.sum() - t_end) < 1e-15
        # too few attempts: ENOTCONV, T at the last accepted time
        T2 = _t(case.T0)
        ctx.set_state(T2, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), dt0)
        with pytest.raises(E.EremError) as ei:
            ctx.rosm_integrate(T2, t_end, dt0, code, tol, tol, lin_tol=1e-13, max_attempts=2)
        assert ei.value.status == E.EREM_ENOTCONV
        for bad in (dict(scheme=E.EREM_ROSM1), dict(tol_a=0.0, tol_r=0.0), dict(dt0=-1.0)):
            args = dict(t_end=t_end, dt0=dt0, scheme=code, tol_a=tol, tol_r=tol)
            args.update(bad)
            with pytest.raises(E.EremError) as ei:
                ctx.rosm_integrate(T2, **args)
            assert ei.value.status == E.EREM_EINVAL
    assert C.rel_l2(got, ref.T) < 1e-8


@pytest.mark.parametrize("dims", [(2, 70, 52, 1, 1), (3, 20, 17, 11, 0)])
def test_stage_multigrid_matches_jacobi_bicgstab(E, dims):
    # the ROS2(1) and ROS3p steps with the multigrid-preconditioned stage
    # solves equal those with Jacobi BiCGSTAB within the stage-solve bound and
    # take several times fewer iterations
    dim, nx, ny, nz, fm = dims
    case = C.random_case(dim, nx, ny, nz, seed=nx, fluid_model=fm)
    tau = 0.05
    fields = lambda: (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
    out = {}
    with E.Context(dim, nx, ny, nz, physics=case.gpu_physics()) as ctx:
        for scheme in (E.EREM_ROS2, E.EREM_ROS3P):
            for kind in (0, 1):
                ctx.set_stage_precond(kind)
                T = _t(case.T0)
                st = ctx.rosm_step(T, tau, scheme, *fields(), lin_tol=STAGE_TOL, maxit=20000)
                out[(scheme, kind)] = (T.cpu().numpy(), st.lin_iters, st.err_est)
        with pytest.raises(E.EremError) as ei:
            ctx.set_stage_precond(2)
        assert ei.value.status == E.EREM_EINVAL
    for scheme in (E.EREM_ROS2, E.EREM_ROS3P):
        (Tj, ij, ej), (Tm, im, em) = out[(scheme, 0)], out[(scheme, 1)]
        inc = np.linalg.norm(Tj - case.T0)
        assert np.linalg.norm(Tm - Tj) < 1e-9 * inc, scheme
        assert em == pytest.approx(ej, rel=1e-6, abs=1e-12)
        assert 3 * im < ij, (scheme, im, ij)


def test_rosm_then_erem_share_the_context(E):
    case = C.heat2d_rect(24, 20)
    prob = case.problem()
    T1 = ts.ros2_step(prob, case.T0, case.dt)
    T2, res = ts.erem_step(prob, T1, case.dt)
    with E.Context(2, 24, 20, physics=case.gpu_physics()) as ctx:
        T = _t(case.T0)
        ctx.rosm_step(T, case.dt, E.EREM_ROS2, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam),
                      lin_tol=STAGE_TOL)
        ctx.erem_step(T, case.dt, opts=E.leja_opts(replay=res.schedule))
        got = T.cpu().numpy()
    assert C.rel_l2(got, T2) < 1e-10


# ---------------------------------------------------------------------------
# error paths: host-detected arguments and device-detected bad inputs
# ---------------------------------------------------------------------------
def test_error_paths_leave_state_unchanged(E):
    case = C.heat2d_rect(16, 12)
    with E.Context(2, 16, 12, physics=case.gpu_physics()) as ctx:
        T = _t(case.T0)
        out = _t(np.zeros(case.n))
        with pytest.raises(E.EremError) as ei:
            ctx.phi1_apply(T, out)  # no state yet
        assert ei.value.status == E.EREM_EINVAL
        with pytest.raises(E.EremError) as ei:
            ctx.erem_step(T, 0.0, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
        assert ei.value.status == E.EREM_EINVAL
        with pytest.raises(E.EremError) as ei:
            ctx.erem_step(T, 0.05, _t(case.p), None, _t(case.phi), _t(case.lam))
        assert ei.value.status == E.EREM_EINVAL
        # NaN in T: detected by the set-up kernels, T left as it was
        bad = case.T0.copy()
        bad[7] = np.nan
        Tb = _t(bad)
        with pytest.raises(E.EremError) as ei:
            ctx.erem_step(Tb, 0.05, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
        assert ei.value.status == E.EREM_ENONFINITE
        assert np.array_equal(Tb.cpu().numpy(), bad, equal_nan=True)
        # negative conductivity
        lam = case.lam.copy()
        lam[3] = -1.0
        with pytest.raises(E.EremError) as ei:
            ctx.erem_step(T, 0.05, _t(case.p), _t(case.lnk), _t(case.phi), _t(lam))
        assert ei.value.status == E.EREM_EINVAL
        # degree cap without splitting: ENOTCONV, T unchanged
        before = T.cpu().numpy().copy()
        with pytest.raises(E.EremError) as ei:
            ctx.erem_step(T, 0.05, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam),
                          opts=E.leja_opts(m_max=3, max_doublings=0))
        assert ei.value.status == E.EREM_ENOTCONV
        assert np.array_equal(T.cpu().numpy(), before)
        # and the context still works afterwards
        st = ctx.erem_step(T, 0.05)
        assert st.substeps >= 1 and np.all(np.isfinite(T.cpu().numpy()))
        # bad replay
        with pytest.raises(E.EremError) as ei:
            ctx.erem_step(T, 0.05, opts=E.leja_opts(replay=[2, 5]))
        assert ei.value.status == E.EREM_EINVAL
