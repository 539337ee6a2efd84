"""Resident problems and the request queue (continuous batching) on the GPU.

Every result that goes through the queue must equal the same request solved
alone through cal_pmchwt_solve, within the far-field tolerance of the solve
(1e-4 relative), whatever else ran beside it.
"""
import numpy as np
import pytest

from gpu_common import EPS, mesh, rel
from paper_2008_04772_gb300 import cal, meshgen

pytestmark = pytest.mark.gpu

FAR_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    from paper_2008_04772_gb300 import build
    build.build()
    return cal.Context(0)


def _inc(n, seed=0):
    d = meshgen.fibonacci_directions(n + seed)[seed:]
    return np.concatenate([d, meshgen.perpendicular_polarisation(d)], 1)


# (mesh, k, eps, nrhs, options): sizes, wavenumbers, materials, preconditioners
# and right-hand-side counts all differ
MIX = [
    ("sphere1", 2.0, EPS, 1, dict(precond="D")),
    ("sphere2", 3.0, 2.5 + 0.01j, 3, dict(precond="D")),
    ("prisms2", 4.0, 3.3 + 0.01j, 2, dict(precond="Di", near_cutoff_P=2.0)),
    ("cubes", 2.5, EPS, 1, dict(precond="D")),
    ("sphere2", 1.5, 3.5 + 0.01j, 5, dict(precond="Si", near_cutoff_P=3.0)),
    ("bipyr14", 2.0, 2.8 + 0.01j, 2, dict(precond="D")),
]
DIRS = meshgen.fibonacci_directions(24)


def _opts(o):
    return cal.solve_opts(precision=cal.FP32, tol=1e-6, **o)


@pytest.fixture(scope="module")
def solo(ctx):
    """Each request of MIX solved alone through cal_pmchwt_solve."""
    out = []
    for i, (name, k, eps, nrhs, o) in enumerate(MIX):
        m = mesh(name)
        gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
        s = cal.pmchwt_solve(ctx, gm, k, eps, _inc(nrhs, i), opts=_opts(o))
        out.append(s.far_field(DIRS))
    return out


def test_problem_solves_equal_the_one_shot_solve(ctx, solo):
    name, k, eps, nrhs, o = MIX[1]
    m = mesh(name)
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    prob = cal.Problem(ctx, gm, k, eps, opts=_opts(o))
    del gm  # the problem no longer needs the mesh
    info = prob.info()
    assert info.n_unknowns == 960
    assert info.bytes_A > 0 and info.bytes_P > 0 and info.bytes_G > 0
    # the same columns as the one-shot solve, then a different batch width
    F = prob.solve(_inc(nrhs, 1)).far_field(DIRS)
    assert rel(F, solo[1]) < 1e-5
    F1 = prob.solve(_inc(nrhs, 1)[1:2]).far_field(DIRS)
    assert rel(F1[0], solo[1][1]) < FAR_TOL
    assert prob.info().batch_width == 1
    # another context on the same device may run the solves
    ctx2 = cal.Context(0)
    F2 = prob.solve(_inc(nrhs, 1), ctx=ctx2).far_field(DIRS)
    assert rel(F2, solo[1]) < 1e-5
    # per-solve solver settings: a cap of two iterations does not converge,
    # and the problem's own settings apply again on the next solve
    s = prob.solve(_inc(1), solver=cal.solve_opts(tol=1e-12, maxit=2, refine=0), allow_not_converged=True)
    assert s.rc == cal.ENOTCONV and s.info().iterations <= 2
    assert prob.solve(_inc(nrhs, 1)).rc == cal.OK


def _submit(q, i):
    name, k, eps, nrhs, o = MIX[i]
    m = mesh(name)
    return q.submit(m.verts, m.tris, m.domain, k, eps, _inc(nrhs, i), DIRS, opts=_opts(o))


def test_queue_results_equal_solo_results_in_the_mix(ctx, solo):
    q = cal.Queue(0, slots=3)
    tickets = [_submit(q, i) for i in range(len(MIX))]
    for i, t in enumerate(tickets):
        res, F = q.wait(t, timeout=600)
        assert res.status == cal.OK, (i, res.status)
        assert res.t_submit <= res.t_start <= res.t_done
        assert rel(F, solo[i]) < FAR_TOL, (i, rel(F, solo[i]))
    st = q.stats()
    assert st.completed == len(MIX) and st.pending == 0 and st.running == 0
    # requests ran side by side on the worker streams
    assert st.peak_running >= 2
    assert st.peak_reserved_bytes <= st.budget_bytes
    q.close()


def test_queue_merges_pending_requests_of_one_problem(ctx, solo):
    # one slot: while a larger request runs, three requests of another problem
    # wait and are then solved as one lockstep batch of 3 + 1 + 1 columns
    q = cal.Queue(0, slots=1)
    b = mesh("sphere3")
    t0 = q.submit(b.verts, b.tris, b.domain, 3.0, EPS, _inc(1), DIRS, opts=_opts(dict(precond="D")))
    name, k, eps, nrhs, o = MIX[4]
    m = mesh(name)
    inc = _inc(nrhs, 4)
    parts = [inc[0:3], inc[3:4], inc[4:5]]
    ts = [q.submit(m.verts, m.tris, m.domain, k, eps, p, DIRS, opts=_opts(o)) for p in parts]
    res0, F0 = q.wait(t0, timeout=600)
    assert res0.status == cal.OK and res0.batch_rhs == 1
    Fs = []
    for t in ts:
        res, F = q.wait(t, timeout=600)
        assert res.status == cal.OK
        assert res.batch_rhs == 5
        Fs.append(F)
    assert rel(np.concatenate(Fs), solo[4]) < FAR_TOL
    assert q.stats().merged >= 2
    q.close()


def test_queue_poll_reports_states_without_waiting(ctx, solo):
    """cal_queue_poll: a submitted request is pending or running, then done; a
    done request's wait returns at once with its result, and the released
    ticket is unknown to poll."""
    import time
    q = cal.Queue(0, slots=1)
    t0, t1 = _submit(q, 1), _submit(q, 0)
    states = {q.poll(t0), q.poll(t1)}
    assert states <= {cal.REQ_PENDING, cal.REQ_RUNNING, cal.REQ_DONE}
    deadline = time.monotonic() + 600
    while q.poll(t1) != cal.REQ_DONE and time.monotonic() < deadline:
        time.sleep(0.01)
    assert q.poll(t1) == cal.REQ_DONE
    r1, F1 = q.wait(t1, timeout=0)
    assert r1.status == cal.OK and rel(F1, solo[0]) < FAR_TOL
    with pytest.raises(cal.CalError) as e:
        q.poll(t1)
    assert e.value.code == cal.EINVAL
    r0, F0 = q.wait(t0, timeout=600)
    assert rel(F0, solo[1]) < FAR_TOL
    q.close()


def test_queue_keeps_operators_resident(ctx, solo):
    q = cal.Queue(0, slots=2)
    r1, F1 = q.wait(_submit(q, 0), timeout=600)
    r2, F2 = q.wait(_submit(q, 0), timeout=600)
    assert r1.reused == 0 and r2.reused == 1
    assert rel(F2, solo[0]) < FAR_TOL
    st = q.stats()
    assert st.problems_created == 1 and st.problem_hits == 1
    q.close()


def test_queue_admission_by_footprint(ctx):
    # three problems of equal size and a budget that holds one of them: they
    # run one after the other although three slots are free (each admission
    # evicts the previous, idle problem), and every result stays correct
    m = mesh("sphere2")
    gm = cal.Mesh(ctx, m.verts, m.tris, m.domain)
    ks = (1.5, 2.0, 2.5)
    o = _opts(dict(precond="D"))
    fps = []
    for k in ks:
        r, keep = cal.make_request(m.verts, m.tris, m.domain, k, EPS, _inc(2), DIRS, opts=o)
        fps.append(sum(cal.request_footprint(r)))
    budget = int(1.05 * max(fps))
    assert all(a + b > budget for a in fps for b in fps)
    q = cal.Queue(0, budget_bytes=budget, slots=3)
    ts = [q.submit(m.verts, m.tris, m.domain, k, EPS, _inc(2), DIRS, opts=o) for k in ks]
    for k, t in zip(ks, ts):
        res, F = q.wait(t, timeout=600)
        assert res.status == cal.OK
        ref = cal.pmchwt_solve(ctx, gm, k, EPS, _inc(2), opts=o).far_field(DIRS)
        assert rel(F, ref) < FAR_TOL
    st = q.stats()
    assert st.peak_reserved_bytes <= budget
    assert st.peak_running == 1
    assert st.evictions >= 2
    # a request that cannot fit the budget on its own is refused at submit
    big = meshgen.icosphere(4)
    with pytest.raises(cal.CalError) as e:
        q.submit(big.verts, big.tris, big.domain, 2.0, EPS, _inc(1), DIRS, opts=o)
    assert e.value.code == cal.ENOMEM
    q.close()


def test_queue_isolates_failing_requests(ctx, solo):
    q = cal.Queue(0, slots=2)
    good = _submit(q, 0)
    name, k, eps, nrhs, o = MIX[0]
    m = mesh(name)
    # a material the solver rejects, and a solve capped before convergence
    bad = q.submit(m.verts, m.tris, m.domain, k, float("nan"), _inc(1), DIRS, opts=_opts(o))
    capped = q.submit(m.verts, m.tris, m.domain, k, eps, _inc(1, 7), DIRS,
                      opts=cal.solve_opts(precision=cal.FP32, tol=1e-12, maxit=2, refine=0, precond="D"))
    res_bad, F_bad = q.wait(bad, timeout=600)
    assert res_bad.status == cal.EINVAL and F_bad is None
    res_cap, F_cap = q.wait(capped, timeout=600)
    assert res_cap.status == cal.ENOTCONV and F_cap is not None
    res, F = q.wait(good, timeout=600)
    assert res.status == cal.OK and rel(F, solo[0]) < FAR_TOL
    # waiting on a request that cannot have finished yet times out and keeps it
    t = _submit(q, 1)
    with pytest.raises(cal.CalError) as e:
        q.wait(t, timeout=0.0)
    assert e.value.code == cal.ETIMEOUT
    res, F = q.wait(t, timeout=600)
    assert res.status == cal.OK and rel(F, solo[1]) < FAR_TOL
    with pytest.raises(cal.CalError):
        q.wait(t, timeout=1.0)  # the ticket was released
    q.close()
