"""The 512-member ensemble at full size, in the configuration bench.py times
(FP32-bulk, tile size and substep levels from the autotuner, KEEP policy):
every member's fields, pressure and heat capacity come from the oracle side
(the oracle's direct pressure solves run in a spawned process pool), one
batched step of all 51.4 M cells runs through the C ABI, then the 29 more
that make the workload's 30, and sampled members (the smallest, the
largest, member 1 whose FP32 Leja estimate overflows, and seeded picks) are
compared with the oracle's own steps after the first and after the 30th, on
the state and on the increment.  Every member must finish with finite
values."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import cases as C
import workloads as W
from oracle import timestep as ts

pytestmark = pytest.mark.gpu

MEMBERS = 512
STEPS = 30
FP32_TOL = 1e-5


def _pressure_and_capacity(e):
    """Oracle side of member e: the steady pressure and (rho c) for Pe 50."""
    case = C.from_workload(W.ensemble_member(e, MEMBERS))
    return e, case.p, case.phys.rhoc_f


@pytest.fixture(scope="module")
def full():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    procs = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_pressure_and_capacity, range(MEMBERS), chunksize=4)
    res.sort(key=lambda r: r[0])
    wls = [W.ensemble_member(e, MEMBERS) for e in range(MEMBERS)]
    return E, wls, [r[1] for r in res], [r[2] for r in res]


def _oracle_run(args):
    """Oracle side of a sampled member: T^1 and T^STEPS (and the first step's
    schedule) from its own steps."""
    e, p, rc = args
    wl = W.ensemble_member(e, MEMBERS)
    case = C.Case(C.fv.Grid(2, wl.nx, wl.ny), C.fv.Physics(rc, rc, wl.head_drop, 0.0, wl.T_inflow, 0),
                  wl.lnk, wl.phi, wl.lam, wl.T0.copy(), p, wl.dt, STEPS)
    prob = case.problem()
    T, first = case.T0.copy(), None
    for k in range(STEPS):
        T, res = ts.erem_step(prob, T, case.dt)
        assert res.converged
        if k == 0:
            first = (T.copy(), res.schedule)
    return e, first[0], first[1], T


def _sample(wls):
    sizes = np.array([wl.nx for wl in wls])
    rng = np.random.default_rng(20120925 + 4)
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes)), 1}
    picks.update(int(e) for e in rng.choice(MEMBERS, 3, replace=False))
    return sorted(picks)


@pytest.mark.timeout(3000)
def test_full_ensemble_steps_match_oracle_on_sampled_members(full):
    E, wls, ps, rcs = full
    picks = _sample(wls)
    # the sampled members' oracle runs go on in spawned processes meanwhile
    pool = mp.get_context("spawn").Pool(len(picks))
    pending = pool.map_async(_oracle_run, [(e, ps[e], rcs[e]) for e in picks])
    members = [(wl.nx, wl.ny, E.Physics(rc, rc, wl.head_drop, 0.0, wl.T_inflow, 0))
               for wl, rc in zip(wls, rcs)]
    outs = []
    with E.Ensemble(members, "fp32_bulk") as ens:
        ens.configure(E.leja_opts(tol=wls[0].tol), policy=E.EREM_ENS_KEEP_SUBSTEPS)
        for e, (wl, p) in enumerate(zip(wls, ps)):
            ens.set_member(e, wl.T0, p, wl.lnk, wl.phi, wl.lam, wl.dt)
        ens.autotune(1)
        for steps in (1, STEPS - 1):
            rs = ens.run(steps)
            assert rs.members_failed == 0 and rs.cells == sum(wl.n for wl in wls)
            stats = [ens.member_stats(e) for e in range(MEMBERS)]
            assert all(s.status == 0 and s.steps_done == steps for s in stats)
            out = {}
            for e in range(MEMBERS):
                T = np.zeros(wls[e].n)
                ens.get_member(e, T)
                assert np.isfinite(T).all(), e
                if e in picks:
                    out[e] = T
            outs.append((out, stats))
    ref = {r[0]: r[1:] for r in pending.get(timeout=2400)}
    pool.close()
    pool.join()
    (out1, stats1), (outN, _) = outs
    for e in picks:
        T0 = wls[e].T0
        T1, sched1, TN = ref[e]
        assert stats1[e].substeps >= sched1[0], (e, stats1[e].schedule, sched1)
        assert C.rel_l2(out1[e], T1) < FP32_TOL, e
        assert C.rel_l2(out1[e] - T0, T1 - T0) < FP32_TOL, e
        assert C.rel_l2(outN[e], TN) < FP32_TOL, e
        assert C.rel_l2(outN[e] - T0, TN - T0) < FP32_TOL, e
