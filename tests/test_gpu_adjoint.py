"""Gradients of a temperature misfit through the C ABI's adjoint and the
torch.autograd.Function of ``paper_1209_5553_gb300.autograd``: against the
oracle's adjoint (oracle/adjoint.py) with the GPU's Leja schedules frozen in
both, against central finite differences of the GPU forward itself (h =
1e-4, schedules replayed, spectral interval held), and across checkpoint
intervals."""
import numpy as np
import pytest

import cases as C
from oracle import adjoint as OA, fv, leja, timestep as ts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch

    assert torch.cuda.is_available()
    import paper_1209_5553_gb300 as E

    return E


def _t(a, dtype=None):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda() if dtype is None else \
        torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def _setup(shape, steps, seed=0):
    case = C.heat2d_rect(*shape) if len(shape) == 2 else C.random_case(3, *shape, seed=seed)
    rng = np.random.default_rng(seed + 9)
    obs = np.sort(rng.choice(case.n, size=min(16, case.n), replace=False))
    data = case.T0[obs] + 5.0 * rng.standard_normal(obs.size)
    return case, obs, data, steps


def _model(E, case, obs, data, steps, precision, checkpoint=10, replay=None, interval=None,
           tape=True):
    import torch

    from paper_1209_5553_gb300.autograd import MisfitModel

    g = case.grid
    return MisfitModel(g.dim, g.nx, g.ny, g.nz, case.gpu_physics(), _t(case.phi), _t(case.lam),
                       case.dt, steps, _t(obs, torch.int64), _t(data), precision=precision,
                       checkpoint=checkpoint, replay=replay, interval=interval, tape=tape)


def _grads(E, case, obs, data, steps, precision, checkpoint=10, replay=None, tape=True):
    import torch

    from paper_1209_5553_gb300.autograd import misfit

    m = _model(E, case, obs, data, steps, precision, checkpoint, replay, tape=tape)
    lnk = _t(case.lnk).requires_grad_(True)
    T0 = _t(case.T0).requires_grad_(True)
    L = misfit(lnk, T0, m)
    L.backward()
    out = (float(L.detach()), lnk.grad.cpu().numpy(), T0.grad.cpu().numpy(), list(m.schedules),
           m.interval)
    m.close()
    return out


def _oracle(case, obs, data, steps, schedules):
    g, ph = case.grid, case.phys
    J = case.problem().J(case.T0)
    alpha, beta = leja.gershgorin_interval(J, case.dt)
    frozen = [OA.FrozenStep(list(s), alpha, beta) for s in schedules]
    L, gT0, glnk, _ = OA.gradients(g, ph, case.lnk, case.phi, case.lam, case.T0, case.dt, steps,
                                   obs, data, frozen=frozen)
    return L, glnk, gT0


@pytest.mark.parametrize("shape", [(14, 11), (6, 5, 4)])
def test_fp64_gradients_match_oracle(E, shape):
    case, obs, data, steps = _setup(shape, 4)
    L, glnk, gT0, sched, _ = _grads(E, case, obs, data, steps, "fp64")
    Lo, glnk_o, gT0_o = _oracle(case, obs, data, steps, sched)
    assert abs(L - Lo) < 1e-10 * Lo
    assert C.rel_l2(gT0, gT0_o) < 1e-9
    assert C.rel_l2(glnk, glnk_o) < 1e-8


def test_fp32_bulk_gradients_match_oracle(E):
    case, obs, data, steps = _setup((20, 16), 5)
    L, glnk, gT0, sched, _ = _grads(E, case, obs, data, steps, "fp32_bulk")
    Lo, glnk_o, gT0_o = _oracle(case, obs, data, steps, sched)
    assert abs(L - Lo) < 1e-5 * Lo
    assert C.rel_l2(gT0, gT0_o) < 1e-4
    assert C.rel_l2(glnk, glnk_o) < 1e-4


def test_gradients_match_central_differences_of_the_gpu_forward(E):
    import torch

    from paper_1209_5553_gb300.autograd import misfit

    # schedules replayed and the interval held: the map the adjoint
    # differentiates, to the O(h^2) and rounding of the differences
    case, obs, data, steps = _setup((16, 16), 6)
    L, glnk, gT0, sched, interval = _grads(E, case, obs, data, steps, "fp64")
    m = _model(E, case, obs, data, steps, "fp64", replay=sched, interval=interval)
    rng = np.random.default_rng(21)
    h = 1e-4
    with torch.no_grad():
        for _ in range(8):
            dk = rng.standard_normal(case.n)
            dT = rng.standard_normal(case.n)
            Lp = float(misfit(_t(case.lnk + h * dk), _t(case.T0 + h * dT), m))
            Lm = float(misfit(_t(case.lnk - h * dk), _t(case.T0 - h * dT), m))
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - (glnk @ dk + gT0 @ dT)) < 1e-7 * max(abs(fd), 1e-3 * L)
    m.close()


def test_held_interval_is_the_forward_interval(E):
    # (schedule replayed) holding the forward's own interval changes the step
    # by rounding only; holding another one changes it, and releasing the
    # hold restores the assembled interval
    import torch

    case, obs, data, steps = _setup((16, 12), 1)
    g = case.grid
    outs = []
    with E.Context(2, g.nx, g.ny, physics=case.gpu_physics()) as ctx:
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        st = ctx.erem_step(_t(case.T0), case.dt)
        lo, hi = st.alpha / case.dt, st.beta / case.dt
        for iv in (None, (lo, hi), (1.5 * lo, hi), None):
            ctx.hold_interval(iv)
            ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam),
                          case.dt)
            T = _t(case.T0)
            s2 = ctx.erem_step(T, case.dt, opts=E.leja_opts(replay=st.schedule))
            outs.append(T.cpu().numpy())
            if iv is not None:
                assert abs(s2.alpha - case.dt * iv[0]) <= 1e-15 * abs(s2.alpha)
        for bad in ((1.0, 0.0), (float("nan"), 0.0)):
            with pytest.raises(E.EremError) as ei:
                ctx.hold_interval(bad)
            assert ei.value.status == E.EREM_EINVAL
    scale = np.max(np.abs(outs[0] - case.T0))
    assert np.max(np.abs(outs[1] - outs[0])) <= 1e-13 * scale
    assert np.max(np.abs(outs[2] - outs[0])) > 1e-12 * scale
    assert np.array_equal(outs[3], outs[0])


def test_checkpoint_interval_does_not_change_the_gradients(E):
    case, obs, data, steps = _setup((12, 9), 7)
    a = _grads(E, case, obs, data, steps, "fp32_bulk", checkpoint=1)
    b = _grads(E, case, obs, data, steps, "fp32_bulk", checkpoint=3)
    assert a[3] == b[3] and a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("precision", ["fp32_bulk", "fp64"])
def test_tape_gives_the_same_gradients(E, precision):
    # the Newton vectors and substep starts recorded by the segment replay are
    # the bits the adjoint would recompute: the gradients are bitwise equal;
    # two steps forced to two and three substeps exercise the w_k records
    case, obs, data, steps = _setup((18, 14), 7)
    free = _grads(E, case, obs, data, steps, precision)[3]
    sched = [list(s) for s in free]
    sched[2] = [2, free[2][1] + 4, free[2][1] + 2]
    sched[5] = [3] + [free[5][1] + 3] * 3
    a = _grads(E, case, obs, data, steps, precision, checkpoint=3, replay=sched, tape=False)
    b = _grads(E, case, obs, data, steps, precision, checkpoint=3, replay=sched, tape=True)
    assert a[3] == b[3] == sched
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


@pytest.mark.parametrize("precision", ["fp32_bulk", "fp64"])
def test_full_tape_gives_the_same_gradients(E, precision):
    # the forward run tapes every step and keeps every state; the backward pass
    # replays nothing and its gradients are those of the recomputing adjoint
    case, obs, data, steps = _setup((18, 14), 7)
    free = _grads(E, case, obs, data, steps, precision)[3]
    sched = [list(s) for s in free]
    sched[2] = [2, free[2][1] + 4, free[2][1] + 2]
    sched[5] = [3] + [free[5][1] + 3] * 3
    a = _grads(E, case, obs, data, steps, precision, checkpoint=3, replay=sched, tape=False)
    b = _grads(E, case, obs, data, steps, precision, replay=sched, tape="full")
    assert a[3] == b[3] == sched
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_full_tape_free_run_matches_oracle(E):
    # stopping-test forward (no replay) taped as it runs: FP64 gradients
    # against the oracle's adjoint of the same frozen schedules
    case, obs, data, steps = _setup((14, 11), 4)
    L, glnk, gT0, sched, _ = _grads(E, case, obs, data, steps, "fp64", tape="full")
    Lo, glnk_o, gT0_o = _oracle(case, obs, data, steps, sched)
    assert abs(L - Lo) < 1e-10 * Lo
    assert C.rel_l2(gT0, gT0_o) < 1e-9
    assert C.rel_l2(glnk, glnk_o) < 1e-8


def test_full_tape_that_does_not_fit_falls_back(E):
    case, obs, data, steps = _setup((12, 10), 4)
    ref = _grads(E, case, obs, data, steps, "fp32_bulk", tape=False, replay=None)
    from paper_1209_5553_gb300.autograd import misfit

    m = _model(E, case, obs, data, steps, "fp32_bulk", tape="full")
    m.full_tape_reserve = lambda: 1024   # far too small: nothing is taped
    lnk = _t(case.lnk).requires_grad_(True)
    T0 = _t(case.T0).requires_grad_(True)
    L = misfit(lnk, T0, m)
    L.backward()
    assert m.schedules == ref[3]
    assert np.allclose(lnk.grad.cpu().numpy(), ref[1], rtol=1e-12, atol=0)
    assert np.allclose(T0.grad.cpu().numpy(), ref[2], rtol=1e-12, atol=0)
    m.close()


def test_tape_that_does_not_fit_falls_back(E):
    # a tape too small for a segment records nothing; the adjoint recomputes
    import torch

    case, obs, data, steps = _setup((12, 10), 4)
    ref = _grads(E, case, obs, data, steps, "fp32_bulk", tape=False)
    m = _model(E, case, obs, data, steps, "fp32_bulk")
    m.tape_bytes = lambda scheds: 1024   # far too small
    from paper_1209_5553_gb300.autograd import misfit

    lnk = _t(case.lnk).requires_grad_(True)
    T0 = _t(case.T0).requires_grad_(True)
    L = misfit(lnk, T0, m)
    L.backward()
    assert float(L.detach()) == ref[0]
    assert np.array_equal(lnk.grad.cpu().numpy(), ref[1]) and np.array_equal(T0.grad.cpu().numpy(), ref[2])
    m.close()


def test_adjoint_argument_errors(E):
    case, obs, data, steps = _setup((8, 6), 1)
    g = case.grid
    with E.Context(2, g.nx, g.ny, physics=case.gpu_physics()) as ctx:
        lam = _t(np.zeros(case.n))
        with pytest.raises(E.EremError) as ei:
            ctx.adjoint_step(_t(case.T0), lam, [1, 5])   # no state yet
        assert ei.value.status == E.EREM_EINVAL
        ctx.set_state(_t(case.T0), _t(case.p), _t(case.lnk), _t(case.phi), _t(case.lam), case.dt)
        ctx.adjoint_begin()
        for bad in ([2, 5], [0], [1, 0]):
            with pytest.raises(E.EremError) as ei:
                ctx.adjoint_step(_t(case.T0), lam, bad)
            assert ei.value.status == E.EREM_EINVAL
