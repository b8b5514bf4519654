"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances (relative L2): FP64 1e-11 and FP32-bulk 1e-5.  FP64 runs replay
the oracle's Leja schedule (substep count and degrees), because the Leja
truncation at tol 1e-6 is far larger than 1e-11 and a degree taken one term
earlier or later is a legitimate outcome of the stopping test; free-running
FP64 runs are also checked to take the oracle's schedule on these seeds.
"""
import numpy as np
import pytest

import cases as C
from oracle import leja, timestep as ts
from oracle.leja import LejaOptions

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def E():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_1209_5553_gb300 as E

    return E


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _ctx(E, case, precision):
    d, nx, ny, nz = case.dims()
    g = case.grid
    return E.Context(d, nx, ny, nz, physics=case.gpu_physics(), precision=precision,
                     lx=g.lx, ly=g.ly, lz=g.lz)


def _phi1_case(case, tau, seed=5):
    rng = np.random.default_rng(seed)
    prob = case.problem(case.T0)
    J = prob.J(case.T0)
    v = prob.G(case.T0) + rng.normal(0, 1, case.n)
    res = leja.phi1_leja(J, v, tau, float(np.max(np.abs(case.T0))), LejaOptions())
    assert res.converged
    return v, res


CASES_2D = [("heat2d_64", lambda: C.heat2d(64)),
            ("ragged_65x67", lambda: C.heat2d_rect(65, 67)),
            ("tiny_5x3", lambda: C.random_case(2, 5, 3, seed=1)),
            ("single_cell", lambda: C.random_case(2, 1, 1, seed=2)),
            ("row_7x1", lambda: C.random_case(2, 7, 1, seed=3))]
CASES_3D = [("cube_17", lambda: C.random_case(3, 17, 17, 17, seed=4)),
            ("box_24x20x9", lambda: C.random_case(3, 24, 20, 9, seed=5)),
            ("channels_32", lambda: C.channels3d(32, steps=2))]


@pytest.mark.parametrize("name,make", CASES_2D + CASES_3D, ids=[c[0] for c in CASES_2D + CASES_3D])
def test_phi1_apply_fp64_replay(E, name, make):
    case = make()
    tau = case.dt
    v, res = _phi1_case(case, tau)
    with _ctx(E, case, "fp64") as ctx:
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), tau)
        out = _t(np.zeros(case.n))
        st = ctx.phi1_apply(_t(v), out, E.leja_opts(replay=res.schedule))
        got = out.cpu().numpy()
    assert st.schedule == res.schedule
    alpha, beta = res.alpha, res.beta
    assert st.alpha == pytest.approx(alpha, rel=1e-12, abs=1e-12)
    assert st.beta == pytest.approx(beta, rel=1e-9, abs=1e-9 * abs(alpha))
    assert C.rel_l2(got, res.value) < FP64_TOL


@pytest.mark.parametrize("name,make", CASES_2D + CASES_3D, ids=[c[0] for c in CASES_2D + CASES_3D])
def test_phi1_apply_fp64_free_running_takes_oracle_schedule(E, name, make):
    case = make()
    v, res = _phi1_case(case, case.dt)
    with _ctx(E, case, "fp64") as ctx:
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        out = _t(np.zeros(case.n))
        st = ctx.phi1_apply(_t(v), out)
        got = out.cpu().numpy()
    assert st.schedule == res.schedule
    assert C.rel_l2(got, res.value) < FP64_TOL


@pytest.mark.parametrize("name,make", CASES_2D + CASES_3D, ids=[c[0] for c in CASES_2D + CASES_3D])
def test_phi1_apply_fp32_bulk(E, name, make):
    case = make()
    v, res = _phi1_case(case, case.dt)
    with _ctx(E, case, "fp32_bulk") as ctx:
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        out = _t(np.zeros(case.n))
        ctx.phi1_apply(_t(v), out)
        got = out.cpu().numpy()
    assert C.rel_l2(got, res.value) < FP32_TOL


def _oracle_run(case, steps, opts=None):
    prob = case.problem(case.T0)
    T = case.T0.copy()
    scheds = []
    for _ in range(steps):
        if case.phys.fluid_model:
            prob = case.problem(T)
        T, res = ts.erem_step(prob, T, case.dt, opts)
        assert res.converged
        scheds.append(res.schedule)
    return T, scheds


def test_erem_heat2d_64_twenty_steps_fp64(E):
    # the 64x64 workload: 20 steps of 0.05, tol 1e-6
    case = C.heat2d(64)
    T_ref, scheds = _oracle_run(case, 20)
    with _ctx(E, case, "fp64") as ctx:
        T = _t(case.T0)
        ctx.erem_step(T, case.dt, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam),
                      opts=E.leja_opts(replay=scheds[0]))
        for k in range(1, 20):
            ctx.erem_step(T, case.dt, opts=E.leja_opts(replay=scheds[k]))
        got = T.cpu().numpy()
    assert C.rel_l2(got, T_ref) < FP64_TOL
    assert C.rel_l2(got - case.T0, T_ref - case.T0) < 1e-10


def test_erem_heat2d_64_free_running_fp64_and_fp32(E):
    case = C.heat2d(64)
    T_ref, scheds = _oracle_run(case, 20)
    for prec, tol in (("fp64", FP64_TOL), ("fp32_bulk", FP32_TOL)):
        with _ctx(E, case, prec) as ctx:
            T = _t(case.T0)
            got_s = []
            st = ctx.erem_step(T, case.dt, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
            got_s.append(st.schedule)
            for _ in range(19):
                got_s.append(ctx.erem_step(T, case.dt).schedule)
            got = T.cpu().numpy()
        assert C.rel_l2(got, T_ref) < tol, prec
        # the change the 20 steps made, T^20 - T^0, to the same bound
        inc_tol = 10 * tol if prec == "fp64" else tol
        assert C.rel_l2(got - case.T0, T_ref - case.T0) < inc_tol, prec
        if prec == "fp64":
            assert got_s == scheds


@pytest.mark.parametrize("name,make", CASES_3D, ids=[c[0] for c in CASES_3D])
def test_erem_steps_3d(E, name, make):
    case = make()
    steps = 2
    T_ref, scheds = _oracle_run(case, steps)
    for prec, tol in (("fp64", FP64_TOL), ("fp32_bulk", FP32_TOL)):
        with _ctx(E, case, prec) as ctx:
            T = _t(case.T0)
            for k in range(steps):
                fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam)) if k == 0 else (None,) * 4
                opts = E.leja_opts(replay=scheds[k]) if prec == "fp64" else None
                ctx.erem_step(T, case.dt, *fields, opts=opts)
            got = T.cpu().numpy()
        assert C.rel_l2(got, T_ref) < tol, prec
        inc_tol = 10 * tol if prec == "fp64" else tol
        assert C.rel_l2(got - case.T0, T_ref - case.T0) < inc_tol, prec


@pytest.mark.parametrize("name,make", CASES_2D[:2] + CASES_3D,
                         ids=[c[0] for c in CASES_2D[:2] + CASES_3D])
def test_diagonal_free_leja_copy(E, name, make, monkeypatch):
    # FP32-bulk with a divergence-free Darcy flux: the Leja copy keeps the
    # couplings only (4 arrays in 2D, 6 in 3D) and the term forms
    # sum_j J_ij (q_j - q_i) + r_i q_i; against the oracle as every FP32-bulk
    # step, and against the copy with the diagonal (EREM_LEJA_DIAG=1) to FP32
    # rounding
    case = make()
    full = 7 if case.grid.dim == 3 else 5
    steps = 2
    T_ref, _ = _oracle_run(case, steps)
    out = {}
    for keep in ("0", "1"):
        monkeypatch.setenv("EREM_LEJA_DIAG", keep)
        with _ctx(E, case, "fp32_bulk") as ctx:
            T = _t(case.T0)
            for k in range(steps):
                fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam)) if k == 0 else (None,) * 4
                ctx.erem_step(T, case.dt, *fields)
            out[keep] = (ctx.leja_coefficients, T.cpu().numpy())
    assert out["0"][0] == full - 1 and out["1"][0] == full
    for ncoef, got in out.values():
        assert C.rel_l2(got, T_ref) < FP32_TOL, ncoef
        assert C.rel_l2(got - case.T0, T_ref - case.T0) < FP32_TOL, ncoef
    assert C.rel_l2(out["0"][1] - case.T0, out["1"][1] - case.T0) < FP32_TOL


@pytest.mark.parametrize("name,make", [CASES_2D[0], CASES_2D[1], CASES_2D[2], CASES_3D[1], CASES_3D[2]],
                         ids=["heat2d_64", "ragged_65x67", "tiny_5x3", "box_24x20x9", "channels_32"])
def test_lagged_terms_match_the_paired_form(E, name, make, monkeypatch):
    # small grids take each term's stopping test in the next launch (block 0)
    # and add d_{m-1} q_{m-1} to P one launch late: the same schedules and,
    # up to the order of the partial sums, the same steps as one test per
    # launch with the paired running sum (EREM_TERM_LAG=0)
    case = make()
    steps = 2
    for prec in ("fp64", "fp32_bulk"):
        out = {}
        for lag in ("0", "1"):
            monkeypatch.setenv("EREM_TERM_LAG", lag)
            with _ctx(E, case, prec) as ctx:
                T = _t(case.T0)
                scheds = []
                for k in range(steps):
                    fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam)) if k == 0 else (None,) * 4
                    st = ctx.erem_step(T, case.dt, *fields)
                    assert st.terms_lagged == int(lag)
                    scheds.append(st.schedule)
                out[lag] = (scheds, T.cpu().numpy())
        assert out["0"][0] == out["1"][0], prec
        tol = 1e-13 if prec == "fp64" else 1e-6
        assert C.rel_l2(out["1"][1] - case.T0, out["0"][1] - case.T0) < tol, prec


def test_leja_copy_keeps_the_diagonal_for_a_divergent_flux(E, monkeypatch):
    # a pressure that is not the steady solution (the linear head) leaves the
    # interior rows of J with nonzero sums: the copy keeps the diagonal, and
    # the step still matches the oracle on the same pressure
    monkeypatch.delenv("EREM_LEJA_DIAG", raising=False)
    case = C.random_case(3, 17, 13, 11, seed=9)
    g = case.grid
    x = (np.arange(g.nx) + 0.5) / g.nx
    case.p = np.broadcast_to(1.0 - x, (g.nz, g.ny, g.nx)).reshape(-1).copy()
    T_ref, _ = _oracle_run(case, 1)
    with _ctx(E, case, "fp32_bulk") as ctx:
        T = _t(case.T0)
        ctx.erem_step(T, case.dt, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
        assert ctx.leja_coefficients == 7
        got = T.cpu().numpy()
    assert C.rel_l2(got - case.T0, T_ref - case.T0) < FP32_TOL


def test_erem_nonlinear_fluid_reassembles_every_step(E):
    case = C.random_case(2, 24, 18, seed=7, fluid_model=1)
    steps = 3
    T_ref, scheds = _oracle_run(case, steps)
    with _ctx(E, case, "fp64") as ctx:
        T = _t(case.T0)
        for k in range(steps):
            fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam)) if k == 0 else (None,) * 4
            ctx.erem_step(T, case.dt, *fields, opts=E.leja_opts(replay=scheds[k]))
        got = T.cpu().numpy()
    assert C.rel_l2(got, T_ref) < FP64_TOL


@pytest.mark.parametrize("s", [2, 4])
def test_forced_substeps(E, s):
    case = C.random_case(3, 12, 10, 8, seed=9)
    v, _ = _phi1_case(case, case.dt)
    prob = case.problem(case.T0)
    sched = [s] + [40] * s
    ref = leja.phi1_leja(prob.J(case.T0), v, case.dt, float(np.max(np.abs(case.T0))),
                         LejaOptions(replay=sched))
    with _ctx(E, case, "fp64") as ctx:
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        out = _t(np.zeros(case.n))
        st = ctx.phi1_apply(_t(v), out, E.leja_opts(replay=sched))
        got = out.cpu().numpy()
    assert st.schedule == sched
    assert C.rel_l2(got, ref.value) < FP64_TOL


def test_degree_cap_splits_the_step_like_the_oracle(E):
    case = C.random_case(2, 20, 16, seed=11, pe=60.0)
    tau = 0.4
    v, _ = _phi1_case(case, tau)
    prob = case.problem(case.T0)
    ref = leja.phi1_leja(prob.J(case.T0), v, tau, float(np.max(np.abs(case.T0))),
                         LejaOptions(m_max=14))
    assert ref.converged and ref.substeps > 1
    with _ctx(E, case, "fp64") as ctx:
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), tau)
        out = _t(np.zeros(case.n))
        st = ctx.phi1_apply(_t(v), out, E.leja_opts(m_max=14))
        got = out.cpu().numpy()
    assert st.schedule == ref.schedule
    assert C.rel_l2(got, ref.value) < FP64_TOL


def test_substeps_from_the_last_step_like_the_oracle(E):
    # m_max = 14 makes the steps split; starting each step at the count the
    # last one passed with takes the oracle's schedule under the same rule,
    # and skips the failing attempts below it
    case = C.random_case(2, 20, 16, seed=11, pe=60.0)
    tau, steps = 0.4, 4
    prob = case.problem(case.T0)
    T = case.T0.copy()
    scheds, s0 = [], 1
    for _ in range(steps):
        T, res = ts.erem_step(prob, T, tau, LejaOptions(m_max=14, start_substeps=s0))
        assert res.converged
        scheds.append(res.schedule)
        s0 = res.substeps
    assert scheds[0][0] > 1
    with _ctx(E, case, "fp64") as ctx:
        ctx.set_substep_start(E.EREM_SUBSTEPS_FROM_LAST)
        Tg = _t(case.T0)
        got_s = []
        for k in range(steps):
            fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam)) if k == 0 else (None,) * 4
            st = ctx.erem_step(Tg, tau, *fields, opts=E.leja_opts(m_max=14))
            got_s.append(st.schedule)
        got = Tg.cpu().numpy()
        # erem_set_state restarts from one substep: the first step's schedule again
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), tau)
        assert ctx.erem_step(_t(case.T0), tau, opts=E.leja_opts(m_max=14)).schedule == scheds[0]
        with pytest.raises(E.EremError):
            ctx.set_substep_start(2)
    assert got_s == scheds
    assert C.rel_l2(got, T) < FP64_TOL


def test_substeps_from_one_every_step_like_the_oracle(E):
    # the default rule on the same steps: every step restarts at one substep
    # (the next level's divided differences are computed on a host thread
    # while the failing level runs); schedules and values are the oracle's
    case = C.random_case(2, 20, 16, seed=11, pe=60.0)
    tau, steps = 0.4, 4
    prob = case.problem(case.T0)
    T = case.T0.copy()
    scheds = []
    for _ in range(steps):
        T, res = ts.erem_step(prob, T, tau, LejaOptions(m_max=14))
        assert res.converged
        scheds.append(res.schedule)
    assert all(s[0] > 1 for s in scheds)
    with _ctx(E, case, "fp64") as ctx:
        Tg = _t(case.T0)
        got_s = []
        for k in range(steps):
            fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam)) if k == 0 else (None,) * 4
            got_s.append(ctx.erem_step(Tg, tau, *fields, opts=E.leja_opts(m_max=14)).schedule)
        got = Tg.cpu().numpy()
    assert got_s == scheds
    assert C.rel_l2(got, T) < FP64_TOL


def test_host_pointers_match_device_pointers(E):
    case = C.heat2d_rect(40, 24)
    res = []
    for host in (False, True):
        with _ctx(E, case, "fp32_bulk") as ctx:
            if host:
                T = case.T0.copy()
                ctx.erem_step(T, case.dt, case.p.copy(), case.lnk.copy(), case.phi.copy(), case.lam.copy())
                ctx.erem_step(T, case.dt)
                res.append(T)
            else:
                T = _t(case.T0)
                ctx.erem_step(T, case.dt, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
                ctx.erem_step(T, case.dt)
                res.append(T.cpu().numpy())
    assert np.array_equal(res[0], res[1])


def test_runs_are_bitwise_deterministic(E):
    case = C.channels3d(32, steps=2)
    outs = []
    for _ in range(2):
        with _ctx(E, case, "fp32_bulk") as ctx:
            T = _t(case.T0)
            ctx.erem_step(T, case.dt, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
            ctx.erem_step(T, case.dt)
            outs.append(T.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def _phi1_with_env(E, case, v, tau, precision, env, opts=None):
    import os

    old = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(val) for k, val in env.items()})
    try:
        with _ctx(E, case, precision) as ctx:  # tuning overrides are read at creation
            ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), tau)
            out = _t(np.zeros(case.n))
            st = ctx.phi1_apply(_t(v), out, opts)
            return out.cpu().numpy(), st
    finally:
        for k_, val in old.items():
            if val is None:
                os.environ.pop(k_, None)
            else:
                os.environ[k_] = val


@pytest.mark.parametrize("degree", [1, 2, 7, 12, 31])
def test_replayed_degrees_from_one_to_a_chunk_and_beyond(E, degree):
    # a replayed degree runs exactly that many terms, inside one chunk of
    # launches or across several
    case = C.random_case(3, 19, 13, 11, seed=31)
    v, _ = _phi1_case(case, case.dt)
    prob = case.problem(case.T0)
    sched = [1, degree]
    ref = leja.phi1_leja(prob.J(case.T0), v, case.dt, float(np.max(np.abs(case.T0))),
                         LejaOptions(replay=sched))
    got, st = _phi1_with_env(E, case, v, case.dt, "fp64", {}, E.leja_opts(replay=sched))
    assert st.schedule == sched
    assert C.rel_l2(got, ref.value) < FP64_TOL


def test_free_running_degrees_of_both_parities(E):
    # free-running degrees of both parities on several seeds: the result must
    # equal the oracle's at its own degree
    parities = set()
    for seed in range(6):
        case = C.random_case(2, 23, 21, seed=40 + seed, pe=20.0 + 10 * seed)
        v, res = _phi1_case(case, case.dt, seed=seed)
        got, st = _phi1_with_env(E, case, v, case.dt, "fp64", {})
        assert st.schedule == res.schedule
        assert C.rel_l2(got, res.value) < FP64_TOL
        parities.add(res.degrees[0] % 2)
    assert parities == {0, 1}


# ---------------------------------------------------------------------------
# fast (midpoint-candidate) Leja points
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name,make", [CASES_2D[0], CASES_2D[1], CASES_3D[1], CASES_3D[2]],
                         ids=["heat2d_64", "ragged_65x67", "box_24x20x9", "channels_32"])
def test_erem_steps_with_fast_leja_points(E, name, make):
    # the oracle with the same point set: FP64 replayed to 1e-11 and, free
    # running, on the oracle's schedule; FP32-bulk to 1e-5; the point set only
    # changes the polynomial, so exact and fast agree to the Leja tolerance
    case = make()
    steps = 3
    fast = LejaOptions(points="fast")
    T_ref, scheds = _oracle_run(case, steps, fast)
    T_exact, _ = _oracle_run(case, steps)
    assert C.rel_l2(T_ref - case.T0, T_exact - case.T0) < 1e-5
    for prec, tol in (("fp64", FP64_TOL), ("fp32_bulk", FP32_TOL)):
        for replay in ((True, False) if prec == "fp64" else (False,)):
            with _ctx(E, case, prec) as ctx:
                ctx.set_leja_points("fast")
                T = _t(case.T0)
                got_s = []
                for k in range(steps):
                    fields = (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam)) if k == 0 else (None,) * 4
                    opts = E.leja_opts(replay=scheds[k]) if replay else None
                    got_s.append(ctx.erem_step(T, case.dt, *fields, opts=opts).schedule)
                got = T.cpu().numpy()
            assert C.rel_l2(got, T_ref) < tol, (prec, replay)
            if prec == "fp64" and not replay:
                assert got_s == scheds


def test_leja_point_kind_switches_and_errors(E):
    # switching back to the exact points restores the exact-point result
    # bit for bit; bad kinds are EINVAL
    case = C.heat2d(32)
    v = case.problem(case.T0).G(case.T0)
    outs = {}
    with _ctx(E, case, "fp64") as ctx:
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        for kind in ("exact", "fast", "exact"):
            ctx.set_leja_points(kind)
            out = _t(np.zeros(case.n))
            st = ctx.phi1_apply(_t(v), out)
            outs.setdefault(kind, []).append((out.cpu().numpy(), st.schedule))
        for bad in (2, -1):
            with pytest.raises(E.EremError) as ei:
                ctx.set_leja_points(bad)
            assert ei.value.status == E.EREM_EINVAL
    assert np.array_equal(outs["exact"][0][0], outs["exact"][1][0])
    ref = leja.phi1_leja(case.problem(case.T0).J(case.T0), v, case.dt, float(np.max(case.T0)),
                         LejaOptions(points="fast", replay=outs["fast"][0][1]))
    assert C.rel_l2(outs["fast"][0][0], ref.value) < FP64_TOL


@pytest.mark.parametrize("name,make", [("heat2d_64", lambda: C.heat2d(64)),
                                       ("ragged_37x23", lambda: C.heat2d_rect(37, 23)),
                                       ("box_24x20x9", lambda: C.random_case(3, 24, 20, 9, seed=5))])
def test_host_T_in_place_equals_device_T(E, name, make):
    # erem_step with T in page-locked host memory read and written in place by
    # the kernels, staged through copies, or on the device: bitwise equal
    import torch

    case = make()
    fields = lambda: (_t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam))
    outs = []
    for kind in ("device", "pinned_in_place", "pinned_staged", "pageable"):
        with _ctx(E, case, "fp32_bulk") as ctx:
            if kind == "pinned_staged":
                ctx.set_host_access(0)
            if kind == "device":
                T = _t(case.T0)
            elif kind == "pageable":
                T = case.T0.copy()
            else:
                T = torch.from_numpy(case.T0.copy()).pin_memory()
            for k in range(3):
                ctx.erem_step(T, case.dt, *(fields() if k == 0 else (None,) * 4))
            outs.append(T.cpu().numpy() if hasattr(T, "cpu") else T.copy())
        if kind == "pinned_staged":
            with _ctx(E, case, "fp32_bulk") as ctx:
                with pytest.raises(E.EremError) as ei:
                    ctx.set_host_access(2)
                assert ei.value.status == E.EREM_EINVAL
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
