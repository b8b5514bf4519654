"""Batched ensemble (erem_ensemble_*) against the oracle.

Seven independent 2D members of different shapes (ragged widths, a 5 x 3
grid, members that span every CTA of a cluster) and two members whose first step
has to be split into 2 and 4 substeps and whose later steps need fewer, so
that the two substep policies take different schedules.  Every member's
fields come from the oracle side (workloads + the oracle's direct pressure
solve); member k draws its ln K with seed 20120925 + 4 + 1000 + k like the
512-member workload.

The two substep members run at Peclet 5.  At Peclet 50 and Leja degrees
above 100 the FP64 result of a step responds to unit-roundoff changes of
T^n by up to 1e-8 (relative), so no two FP64 evaluations with different
rounding orders agree to 1e-11 there; at Peclet 5 the response stays near
1e-15 and the 1e-11 bound applies to every member.
"""
import dataclasses

import numpy as np
import pytest

import cases as C
import workloads as W
from oracle import leja, timestep as ts

pytestmark = pytest.mark.gpu

# (nx, ny, sigma of ln K, dt, Peclet)
SPEC = [
    (13, 11, 0.5, 0.05, 50.0),
    (96, 50, 2.5, 0.05, 50.0),
    (37, 61, 1.5, 0.05, 50.0),
    (5, 3, 1.0, 0.05, 50.0),
    (200, 160, 2.0, 0.02, 5.0),
    (120, 100, 2.0, 0.2, 5.0),
    (64, 64, 1.0, 0.05, 50.0),
]
SUBSTEP_MEMBERS = (4, 5)
STEPS = 3
FP64_TOL = 1e-11
FP32_TOL = 1e-5


def _member_case(k):
    nx, ny, sigma, dt, peclet = SPEC[k]
    wl = W.heat2d_rect(nx, ny, sigma=sigma, seed=W.SEED_BASE + 4 + 1000 + k, steps=STEPS)
    case = C.from_workload(dataclasses.replace(wl, peclet=peclet, dt=dt))
    return case


@pytest.fixture(scope="module")
def ref():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    members = []
    for k in range(len(SPEC)):
        case = _member_case(k)
        pb = case.problem()
        T = case.T0.copy()
        traj, scheds = [T.copy()], []
        for _ in range(STEPS):
            T, res = ts.erem_step(pb, T, case.dt)
            traj.append(T.copy())
            scheds.append(res.schedule)
        members.append((case, pb, traj, scheds))
    return E, members


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _ensemble(E, members, precision, policy=None, **cfg):
    ens = E.Ensemble([(m[0].grid.nx, m[0].grid.ny, m[0].gpu_physics()) for m in members], precision)
    ens.configure(policy=E.EREM_ENS_RESTART_SUBSTEPS if policy is None else policy, **cfg)
    for k, (case, _, _, _) in enumerate(members):
        ens.set_member(k, _t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
    return ens


def _get(ens, k):
    import torch

    out = torch.empty(ens.sizes[k], dtype=torch.float64, device="cuda")
    ens.get_member(k, out)
    return out.cpu().numpy()


def _check_schedule(sched, free, err_est):
    """The stopping decisions the ensemble took, against the oracle's.

    At degrees near 100 the Leja error estimates amplify rounding differences
    (a relative change of 1e-15 in T^n moves them by about 1e-4 at m = 120),
    so a stop that sits at the threshold can fall one term earlier or later
    than the oracle's.  The substep count must agree; each degree must lie
    within two of the oracle's own; and the oracle, replaying the ensemble's
    schedule, must find the stopping test met at that degree up to 10 %."""
    assert sched[0] == free[0], (sched, free)
    assert all(abs(a - b) <= 2 for a, b in zip(sched[1:], free[1:])), (sched, free)
    assert 100.0 * err_est < 1.1, (sched, err_est)


def test_fp64_restart_policy_matches_oracle(ref):
    # step by step: the oracle replays the schedule each step took and the
    # temperatures agree to 1e-11; the schedule is checked against the
    # oracle's free-running step from the same state
    E, members = ref
    with _ensemble(E, members, "fp64") as ens:
        T = [m[0].T0.copy() for m in members]
        for step in range(STEPS):
            rs = ens.run(1)
            assert rs.members_failed == 0 and rs.clusters >= 1 and rs.passes > 0
            for k, (case, pb, traj, scheds) in enumerate(members):
                st = ens.member_stats(k)
                assert st.status == 0 and st.steps_done == 1
                free = ts.erem_step(pb, T[k], case.dt)[1].schedule
                T[k], res = ts.erem_step(pb, T[k], case.dt, leja.LejaOptions(replay=st.schedule))
                _check_schedule(st.schedule, free, res.err_est)
                assert st.terms >= st.degree_total
                assert C.rel_l2(_get(ens, k), T[k]) < FP64_TOL, (k, step)
        for k, (case, _, traj, _) in enumerate(members):
            assert C.rel_l2(_get(ens, k), traj[-1]) < FP32_TOL


def test_fp64_keep_policy_matches_oracle_replay(ref):
    # KEEP starts each step at the substep count of the previous one: step by
    # step, the oracle replays the schedule the ensemble reports
    E, members = ref
    with _ensemble(E, members, "fp64", policy=E.EREM_ENS_KEEP_SUBSTEPS) as ens:
        T = [m[0].T0.copy() for m in members]
        for step in range(STEPS):
            ens.run(1)
            for k, (case, pb, traj, scheds) in enumerate(members):
                sched = ens.member_stats(k).schedule
                free = ts.erem_step(pb, T[k], case.dt)[1].schedule
                assert sched[0] >= free[0]
                T[k], res = ts.erem_step(pb, T[k], case.dt, leja.LejaOptions(replay=sched))
                if step == 0:
                    _check_schedule(sched, free, res.err_est)
                assert 100.0 * res.err_est < 1.1
                assert C.rel_l2(_get(ens, k), T[k]) < FP64_TOL, (k, step)
        # the members that could go back to fewer substeps did not
        for k in SUBSTEP_MEMBERS:
            assert ens.member_stats(k).substeps > members[k][3][-1][0] > 0
        # and the schedule change stays within the Leja tolerance
        for k, (case, _, traj, _) in enumerate(members):
            assert C.rel_l2(_get(ens, k), traj[-1]) < FP32_TOL


def test_fp32_bulk_matches_oracle(ref):
    # the members' fluxes are divergence-free (the oracle's direct pressure
    # solves), so their FP32 Leja copies hold the couplings only
    E, members = ref
    with _ensemble(E, members, "fp32_bulk", policy=E.EREM_ENS_KEEP_SUBSTEPS) as ens:
        ens.run(STEPS)
        for k, (case, _, traj, _) in enumerate(members):
            assert ens.member_stats(k).leja_coefficients == 4, k
            assert C.rel_l2(_get(ens, k), traj[-1]) < FP32_TOL, k
    with _ensemble(E, members[:1], "fp64") as ens:
        assert ens.member_stats(0).leja_coefficients == 5


def test_cluster_sizes_agree(ref):
    # the per-cell arithmetic does not depend on the cluster size; only the
    # order of the norm partial sums does
    E, members = ref
    runs = []
    for cs in (2, 4, 8, 16):
        with _ensemble(E, members, "fp64", cluster_ctas=cs) as ens:
            rs = ens.run(STEPS)
            assert rs.cluster_ctas == cs and rs.members_failed == 0
            runs.append(([ens.member_stats(k).schedule for k in range(len(members))],
                         [_get(ens, k) for k in range(len(members))]))
    for sch, Ts in runs[1:]:
        assert sch == runs[0][0]
        for a, b in zip(Ts, runs[0][1]):
            assert C.rel_l2(a, b) < 1e-14


def test_member_result_does_not_depend_on_the_batch(ref):
    # a member's bits are the same alone, in the batch, with one cluster
    # taking every member in turn, and on a second run from the same state
    E, members = ref
    out = []
    for kw in ({}, {"max_clusters": 1}):
        for rep in range(2):
            with _ensemble(E, members, "fp32_bulk", **kw) as ens:
                rs = ens.run(STEPS)
                assert rs.members_failed == 0
                if kw:
                    assert rs.clusters == 1
                out.append(([_get(ens, k) for k in range(len(members))],
                            [ens.member_stats(k).terms for k in range(len(members))]))
    for k in (1, 4):
        with _ensemble(E, [members[k]], "fp32_bulk") as ens:
            ens.run(STEPS)
            alone = _get(ens, 0)
            assert np.array_equal(alone, out[0][0][k]), k
            assert ens.member_stats(0).terms == out[0][1][k]
    for Ts, terms in out[1:]:
        assert terms == out[0][1]
        for x, y in zip(Ts, out[0][0]):
            assert np.array_equal(x, y)


def test_runs_in_pieces_equal_one_run(ref):
    E, members = ref
    with _ensemble(E, members, "fp32_bulk") as one, _ensemble(E, members, "fp32_bulk") as three:
        assert one.run(STEPS).graph == 1
        for _ in range(STEPS):
            assert three.run(1).graph == 1  # the first run captures, the others replay
        for k in range(len(members)):
            assert np.array_equal(_get(one, k), _get(three, k))


def test_graph_replay_equals_direct_launches(ref, monkeypatch):
    # the captured run (uploads, the persistent launch, the read-back) gives
    # the bits of the same operations launched directly, over several runs and
    # a change of cluster shape (a new capture)
    E, members = ref
    out = {}
    for graph in ("1", "0"):
        monkeypatch.setenv("EREM_ENS_GRAPH", graph)
        res = []
        with _ensemble(E, members, "fp32_bulk", cluster_ctas=4) as ens:
            for cs in (4, 4, 2):
                ens.configure(policy=E.EREM_ENS_RESTART_SUBSTEPS, cluster_ctas=cs)
                rs = ens.run(1)
                assert rs.graph == int(graph) and rs.cluster_ctas == cs and rs.members_failed == 0
                res.append([_get(ens, k) for k in range(len(members))])
        out[graph] = res
    for a, b in zip(out["1"], out["0"]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_matches_single_context_steps(ref):
    E, members = ref
    with _ensemble(E, members, "fp64") as ens:
        ens.run(STEPS)
        for k, (case, _, _, _) in enumerate(members):
            g = case.grid
            with E.Context(2, g.nx, g.ny, physics=case.gpu_physics()) as ctx:
                T = _t(case.T0)
                ctx.set_state(T, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
                for _ in range(STEPS):
                    ctx.erem_step(T, case.dt)
                assert C.rel_l2(_get(ens, k), T.cpu().numpy()) < 1e-13, k


def test_autotune_restores_state_and_learns_substeps(ref):
    E, members = ref
    with _ensemble(E, members, "fp32_bulk", policy=E.EREM_ENS_KEEP_SUBSTEPS) as ens:
        before = [_get(ens, k) for k in range(len(members))]
        ens.autotune(1)
        for k in range(len(members)):
            assert np.array_equal(_get(ens, k), before[k])
        rs = ens.run(1)
        assert rs.cluster_ctas in (2, 4, 8, 16)
        for k, (case, _, traj, scheds) in enumerate(members):
            st = ens.member_stats(k)
            # started at the count doubling reached: no failed attempt
            assert st.attempts == 0 and st.substeps == scheds[0][0]
            assert st.terms == st.degree_total
            assert C.rel_l2(_get(ens, k), traj[1]) < FP32_TOL


def test_member_failure_is_isolated(ref):
    # m_max = 40 and one doubling: each member converges or fails as the
    # oracle with the same options does; failed members keep T^n
    E, members = ref
    opts_o = leja.LejaOptions(m_max=40, max_doublings=1)
    with _ensemble(E, members, "fp64") as ens:
        ens.configure(E.leja_opts(m_max=40, max_doublings=1), policy=E.EREM_ENS_RESTART_SUBSTEPS)
        with pytest.raises(E.EremError) as ei:
            ens.run(1)
        assert ei.value.status == E.EREM_ENOTCONV
        n_fail = 0
        for k, (case, pb, _, _) in enumerate(members):
            T1, res = ts.erem_step(pb, case.T0, case.dt, opts_o)
            st = ens.member_stats(k)
            if res.converged:
                assert st.status == 0 and st.steps_done == 1
                assert C.rel_l2(_get(ens, k), T1) < FP64_TOL
            else:
                n_fail += 1
                assert st.status == E.EREM_ENOTCONV and st.steps_done == 0
                assert np.array_equal(_get(ens, k), case.T0)
        assert 0 < n_fail < len(members)
        assert ens.run_stats().members_failed == n_fail


def test_fp32_estimate_overflow_splits_the_step(ref):
    # member 1 of the 512-member workload (190^2 cells, sigma 1.73, Pe 50):
    # the Newton vectors q_m grow past 1.8e19 at m = 86 whatever the substep
    # length (the scaled operator does not depend on it), so their FP32
    # squares overflow before the oracle's 4-substep schedule (101, 72, 63,
    # 61 terms) stops; the non-finite estimate counts as a failed attempt and
    # the step is split further, in the ensemble and in a single context
    E, _ = ref
    case = C.from_workload(W.ensemble_member(1))
    T1, res = ts.erem_step(case.problem(), case.T0, case.dt)
    assert res.schedule[0] == 4 and res.schedule[1] > 86
    g = case.grid
    for policy in (E.EREM_ENS_RESTART_SUBSTEPS, E.EREM_ENS_KEEP_SUBSTEPS):
        with E.Ensemble([(g.nx, g.ny, case.gpu_physics())], "fp32_bulk") as ens:
            ens.configure(policy=policy)
            ens.set_member(0, _t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam),
                           case.dt)
            ens.run(1)
            st = ens.member_stats(0)
            assert st.status == 0 and st.steps_done == 1 and st.substeps > 4
            assert max(st.degrees[:st.substeps]) <= 86
            assert C.rel_l2(_get(ens, 0), T1) < FP32_TOL
    with E.Context(2, g.nx, g.ny, physics=case.gpu_physics(), precision="fp32_bulk") as ctx:
        T = _t(case.T0)
        ctx.set_state(T, _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        st = ctx.erem_step(T, case.dt)
        assert st.substeps > 4
        assert C.rel_l2(T.cpu().numpy(), T1) < FP32_TOL


def test_member_pass_bound_returns_timeout(ref, monkeypatch):
    # every member is bounded in passes; with a bound of 40 passes a step
    # (a test hook) the members whose first step needs more stop with
    # ETIMEOUT and keep T^n, the others take their step
    E, members = ref
    monkeypatch.setenv("EREM_ENS_PASSES_PER_STEP", "40")
    with _ensemble(E, members, "fp64") as ens:
        with pytest.raises(E.EremError) as ei:
            ens.run(1)
        assert ei.value.status == E.EREM_ETIMEOUT
        n_out = 0
        for k, (case, _, traj, scheds) in enumerate(members):
            st = ens.member_stats(k)
            if st.status == E.EREM_ETIMEOUT:
                n_out += 1
                assert st.steps_done == 0 and st.terms + st.passes == 40
                assert np.array_equal(_get(ens, k), case.T0)
            else:
                assert st.status == 0 and st.terms + st.passes <= 40
                assert C.rel_l2(_get(ens, k), traj[1]) < FP64_TOL
        assert 0 < n_out < len(members)
    monkeypatch.delenv("EREM_ENS_PASSES_PER_STEP")
    with _ensemble(E, members, "fp64") as ens:  # and the next ensemble runs normally
        ens.run(1)
        assert C.rel_l2(_get(ens, 0), members[0][2][1]) < FP64_TOL


def test_set_temperature_restarts_from_a_saved_state(ref):
    # save after one step, run two more, restore the saved state (from host
    # memory for one member, device memory for the rest) and run two again
    E, members = ref
    with _ensemble(E, members, "fp32_bulk") as ens:
        ens.run(1)
        saved = [_get(ens, k) for k in range(len(members))]
        ens.run(2)
        after = [_get(ens, k) for k in range(len(members))]
        for k in range(len(members)):
            ens.set_temperature(k, saved[k] if k == 0 else _t(saved[k]))
            assert np.array_equal(_get(ens, k), saved[k])
        ens.run(2)
        for k in range(len(members)):
            assert np.array_equal(_get(ens, k), after[k])


def test_host_output_and_argument_errors(ref):
    E, members = ref
    with _ensemble(E, members[:2], "fp64") as ens:
        ens.run(1)
        host = np.zeros(ens.sizes[1])
        ens.get_member(1, host)
        assert np.array_equal(host, _get(ens, 1))
        for bad in (lambda: ens.run(0), lambda: E.erem_ensemble_get_member(ens._h, 2, None, host),
                    lambda: ens.configure(E.leja_opts(replay=[1, 5]))):
            with pytest.raises(E.EremError) as ei:
                bad()
            assert ei.value.status == E.EREM_EINVAL
    case = members[0][0]
    with E.Ensemble([(case.grid.nx, case.grid.ny, case.gpu_physics())] * 2, "fp64") as ens:
        ens.set_member(0, _t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), 0.05)
        with pytest.raises(E.EremError) as ei:
            ens.run(1)  # member 1 has no state
        assert ei.value.status == E.EREM_EINVAL
