"""The 512-member ensemble at full size, in the configuration bench.py times
(FP32-bulk, tile size and substep levels from the autotuner, KEEP policy):
every member's fields, pressure and heat capacity come from the oracle side
(the oracle's direct pressure solves run in a spawned process pool), one
batched step of all 51.4 M cells runs through the C ABI, and sampled members
(the smallest, the largest, member 1 whose FP32 Leja estimate overflows, and
seeded picks) are compared with the oracle's own step.  Every member must
finish its step with finite values."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import cases as C
import workloads as W
from oracle import timestep as ts

pytestmark = pytest.mark.gpu

MEMBERS = 512
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


def _sample(wls):
    sizes = np.array([wl.nx for wl in wls])
    rng = np.random.default_rng(20120925 + 4)
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes)), 1}
    picks.update(int(e) for e in rng.choice(MEMBERS, 3, replace=False))
    return sorted(picks)


@pytest.mark.timeout(2400)
def test_full_ensemble_step_matches_oracle_on_sampled_members(full):
    E, wls, ps, rcs = full
    members = [(wl.nx, wl.ny, E.Physics(rc, rc, wl.head_drop, 0.0, wl.T_inflow, 0))
               for wl, rc in zip(wls, rcs)]
    with E.Ensemble(members, "fp32_bulk") as ens:
        ens.configure(E.leja_opts(tol=wls[0].tol), policy=E.EREM_ENS_KEEP_SUBSTEPS)
        for e, (wl, p) in enumerate(zip(wls, ps)):
            ens.set_member(e, wl.T0, p, wl.lnk, wl.phi, wl.lam, wl.dt)
        ens.autotune(1)
        rs = ens.run(1)
        assert rs.members_failed == 0 and rs.cells == sum(wl.n for wl in wls)
        stats = [ens.member_stats(e) for e in range(MEMBERS)]
        assert all(s.status == 0 and s.steps_done == 1 for s in stats)
        out = {}
        for e in range(MEMBERS):
            T = np.zeros(wls[e].n)
            ens.get_member(e, T)
            assert np.isfinite(T).all(), e
            out[e] = T
    for e in _sample(wls):
        wl = wls[e]
        case = C.Case(C.fv.Grid(2, wl.nx, wl.ny), C.fv.Physics(rcs[e], rcs[e], wl.head_drop, 0.0,
                                                               wl.T_inflow, 0),
                      wl.lnk, wl.phi, wl.lam, wl.T0.copy(), ps[e], wl.dt, 1)
        T1, res = ts.erem_step(case.problem(), case.T0, case.dt)
        assert stats[e].substeps >= res.substeps, (e, stats[e].schedule, res.schedule)
        assert C.rel_l2(out[e], T1) < FP32_TOL, e
