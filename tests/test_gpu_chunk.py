"""Sampling under a device-memory budget (RSRR_FLAG_CHUNK_POINTS), through
the C ABI: when the band factors of all N points do not fit the budget, the
handle holds the factors of a chunk of points and factors, solves and
refines the points chunk by chunk.  A point's factorisation, solves and
refinement sweeps do not depend on the other points, so the samples are
bitwise those of the unchunked handle; the handle stays within its budget,
the eigenpairs match the oracle, and two-stage sampling (rsrr_add_points)
works through the chunks too."""
import numpy as np
import pytest

import oracle
import workloads as W
from util import match_eigs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return rsrr


def chunk_budget(rs, p, frac, **kw):
    """A budget that holds everything but the band storage, and about frac
    of the band storage of all N points (from the estimates with all points
    and with chunks of one point)."""
    need = rs.estimate_bytes(p, rs.default_opts(**kw))
    need1 = rs.estimate_bytes(p, rs.default_opts(chunk_points=1, **kw))
    return need, int(need1 + frac * (need - need1))


def sampled(rs, p, **kw):
    s = rs.Solver(p, rs.default_opts(**kw))
    s.sample()
    s.check()
    return s


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_chunked_samples_equal_the_unchunked_ones(rs, prec):
    p = W.rational_grid(g=60, N=32, L=8)
    precision = rs.RSRR_PREC_MIXED if prec == "mixed" else rs.RSRR_PREC_FP64
    full = sampled(rs, p, precision=precision)
    need, budget = chunk_budget(rs, p, 0.3, precision=precision)
    ch = sampled(rs, p, precision=precision, flags=rs.RSRR_FLAG_CHUNK_POINTS, mem_budget_bytes=budget)
    assert ch.stats()["device_bytes"] <= budget < need
    assert np.array_equal(ch.samples(), full.samples())
    assert np.array_equal(ch.eta(), full.eta())
    seven = sampled(rs, p, precision=precision, chunk_points=7)   # explicit chunks, last one of 4
    assert seven.stats()["device_bytes"] < full.stats()["device_bytes"]
    assert np.array_equal(seven.samples(), full.samples())
    seven.close()
    for s in (full, ch):
        s.project()
    a, b = full.solve(), ch.solve()
    assert np.array_equal(a["lam"], b["lam"])
    ref = oracle.rsrr(p)
    assert len(b["lam"]) == len(ref["lam"]) > 0 and match_eigs(ref["lam"], b["lam"]) <= 1e-9
    full.close()
    ch.close()


def test_without_the_flag_the_budget_still_refuses(rs):
    p = W.rational_grid(g=40, N=16, L=4)
    need = rs.estimate_bytes(p)
    with pytest.raises(rs.RSRRError) as e:
        rs.Solver(p, rs.default_opts(mem_budget_bytes=need // 2))
    assert e.value.status == rs.RSRR_ENOMEM
    with pytest.raises(rs.RSRRError) as e:   # not even one point fits
        rs.Solver(p, rs.default_opts(mem_budget_bytes=1 << 16, flags=rs.RSRR_FLAG_CHUNK_POINTS))
    assert e.value.status == rs.RSRR_ENOMEM


def test_two_stage_sampling_through_chunks(rs):
    p = W.diag_rational(N=12)
    _, budget = chunk_budget(rs, p, 0.3)
    opts = dict(flags=rs.RSRR_FLAG_CHUNK_POINTS, mem_budget_bytes=budget, NQ=256, res_tol=1e-2,
                eta_tol=1e-13, max_refine=16)
    outs = []
    for kw in (dict(eta_tol=1e-13, max_refine=16, NQ=256, res_tol=1e-2), opts):
        s = sampled(rs, p, **kw)
        s.project()
        lam1 = s.solve()["lam"]
        s.add_points(lam1)
        assert s.check_status() == rs.RSRR_OK
        outs.append((s.samples(), s.points()))
        s.close()
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][0], outs[1][0])
