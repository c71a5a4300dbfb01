"""GPU tests of the request server (rsrr_server_*): continuous batching of
whole RSRR solves.  Each request's result in a mixed, overlapping stream is
the result of the same request run alone through rsrr_create / rsrr_sample /
rsrr_project / rsrr_solve; admission respects the memory budget; kept
handles stay resident until released; a failing request does not disturb
the others."""
import ctypes as C
import time

import numpy as np
import pytest

import workloads as W
from util import match_eigs

pytestmark = pytest.mark.gpu

EIG_TOL = 1e-9   # relative eigenvalue agreement, as against the oracle
RES_TOL = 1e-10  # normalised residual of every returned eigenpair


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return rsrr


# (name, problem, NQ): the families of the eigen-parity tests, sparse and dense
MIX = [
    ("diag_quadratic", lambda: W.diag_quadratic(), 256),
    ("diag_rational", lambda: W.diag_rational(), 256),
    ("diag_delay", lambda: W.diag_delay(), 256),
    ("quadratic_c0b", lambda: W.config("c0b"), 500),
    ("grid_g30", lambda: W.rational_grid(g=30, N=64, L=8), 500),
    ("helmholtz_n64", lambda: W.helmholtz_sphere(n=64, N=32, L=16), 256),
    ("helmholtz_n128", lambda: W.helmholtz_sphere(n=128, N=32, L=16), 256),
]


def alone(rs, p, NQ):
    s = rs.Solver(p, rs.default_opts(NQ=NQ))
    s.sample()
    s.check()
    s.project()
    out = s.solve()
    out["k"] = s.stats()["k"]
    s.close()
    return out


@pytest.fixture(scope="module")
def lone_results(rs):
    return {name: alone(rs, make(), NQ) for name, make, NQ in MIX}


def check_same(ref, rep):
    assert rep["status"] in (0, 1), rep["error"]  # OK or WGAP
    assert rep["count"] == len(ref["lam"]) > 0
    assert match_eigs(ref["lam"], rep["lam"]) <= EIG_TOL
    assert rep["res"].max() <= RES_TOL


def overlapping_pairs(reps):
    iv = sorted((r["t_admit"], r["t_done"]) for r in reps)
    return sum(1 for i in range(len(iv)) for j in range(i + 1, len(iv)) if iv[j][0] < iv[i][1])


def test_each_result_in_the_mix_equals_the_result_alone(rs, lone_results):
    rng = np.random.default_rng(5000)
    sv = rs.Server(slots=4)
    ids = []
    # every family three times, in a shuffled order, with Poisson-like gaps
    order = [i for i in range(len(MIX)) for _ in range(3)]
    rng.shuffle(order)
    for i in order:
        name, make, NQ = MIX[i]
        ids.append((name, sv.submit(make(), rs.default_opts(NQ=NQ))))
        time.sleep(float(rng.exponential(0.01)))
    reps = []
    for name, rid in ids:
        rep = sv.wait(rid, timeout=600.0)
        assert rep is not None, name
        check_same(lone_results[name], rep)
        assert rep["t_submit"] <= rep["t_admit"] <= rep["t_done"]
        reps.append(rep)
        sv.release(rid)
    st = sv.stats()
    sv.close()
    assert st["completed"] == len(ids) and st["failed"] == 0
    # requests were on the device together
    assert st["peak_active"] >= 2
    assert overlapping_pairs(reps) >= 1
    assert st["used_bytes"] == 0


def test_admission_respects_the_memory_budget(rs, lone_results):
    probs = [(name, make(), NQ) for name, make, NQ in MIX[:3]]  # requests of similar size
    est = [rs.estimate_bytes(p, rs.default_opts(NQ=NQ)) for _, p, NQ in probs]
    budget = int(max(est) * 1.2)  # room for one request at a time
    assert min(est) * 2 > budget
    sv = rs.Server(slots=4, mem_budget_bytes=budget)
    ids = [(name, sv.submit(p, rs.default_opts(NQ=NQ))) for name, p, NQ in probs]
    reps = []
    for name, rid in ids:
        rep = sv.wait(rid, timeout=600.0)
        check_same(lone_results[name], rep)
        reps.append(rep)
        sv.release(rid)
    st = sv.stats()
    sv.close()
    assert st["peak_bytes"] <= budget
    assert st["peak_active"] == 1
    assert overlapping_pairs(reps) == 0
    assert [r["device_bytes"] for r in reps] == est


def test_request_larger_than_the_budget_is_refused(rs):
    sv = rs.Server(slots=2, mem_budget_bytes=1 << 20)
    with pytest.raises(rs.RSRRError) as e:
        sv.submit(W.diag_quadratic(), rs.default_opts(NQ=256))
    assert e.value.status == rs.RSRR_ENOMEM
    sv.close()


def test_kept_handle_stays_resident_until_release(rs, lone_results):
    name, make, NQ = MIX[4]
    p = make()
    sv = rs.Server(slots=2, keep=True)
    rid = sv.submit(p, rs.default_opts(NQ=NQ))
    rep = sv.wait(rid, timeout=600.0)
    check_same(lone_results[name], rep)
    assert sv.stats()["used_bytes"] == rep["device_bytes"] > 0
    h = sv.handle(rid)
    assert h
    st = rs.rsrr_stats()
    assert rs.rsrr_get_stats(h, C.byref(st)) == rs.RSRR_OK
    assert st.k == rep["k"] == lone_results[name]["k"]
    Q = np.empty((st.k, p.n), dtype=np.complex128)
    assert rs.rsrr_get_Q(h, Q.ctypes.data_as(C.c_void_p), 0, None) == rs.RSRR_OK
    Q = Q.T
    assert np.abs(Q.conj().T @ Q - np.eye(st.k)).max() <= 1e-12
    sv.release(rid)
    assert sv.stats()["used_bytes"] == 0
    assert not sv.handle(rid)
    sv.close()


def test_failed_request_does_not_disturb_the_others(rs, lone_results):
    sv = rs.Server(slots=3)
    good = [(name, sv.submit(make(), rs.default_opts(NQ=NQ))) for name, make, NQ in MIX[:3]]
    # no refinement sweep: the complex64 solve stops near eta ~ 1e-6 > 1e-10
    bad = sv.submit(W.diag_rational(), rs.default_opts(NQ=256, max_refine=0))
    rb = sv.wait(bad, timeout=600.0)
    assert rb["status"] == rs.RSRR_ENOCONV and "refinement" in rb["error"]
    for name, rid in good:
        check_same(lone_results[name], sv.wait(rid, timeout=600.0))
    st = sv.stats()
    sv.close()
    assert st["failed"] == 1 and st["completed"] == 3 and st["used_bytes"] == 0


def test_timeout_in_one_request_stays_with_that_request(rs, lone_results):
    """A bounded device wait that runs out in one request (injected on the
    host side: a wait on a barrier nothing completes, counted in that
    request's own status word) makes that request return ETIMEOUT; the
    requests running beside it return OK with their lone results."""
    sv = rs.Server(slots=4)
    good = [(name, sv.submit(make(), rs.default_opts(NQ=NQ))) for name, make, NQ in MIX[:3]]
    bad = sv.submit(W.diag_quadratic(),
                    rs.default_opts(NQ=256, flags=rs.RSRR_FLAG_INJECT_TIMEOUT))
    more = [(name, sv.submit(make(), rs.default_opts(NQ=NQ))) for name, make, NQ in MIX[3:5]]
    rb = sv.wait(bad, timeout=600.0)
    assert rb["status"] == rs.RSRR_ETIMEOUT, rb["error"]
    for name, rid in good + more:
        rep = sv.wait(rid, timeout=600.0)
        assert rep["status"] == rs.RSRR_OK, rep["error"]
        check_same(lone_results[name], rep)
    st = sv.stats()
    sv.close()
    assert st["failed"] == 1 and st["completed"] == 5 and st["used_bytes"] == 0
