"""rsrr_sample_batch: several band-path problems of uneven size (grid sides,
bandwidths, N, L, precisions) sampled with ONE persistent grouped band LU
launch per precision.  Each handle's samples equal bit for bit those of its
own rsrr_sample with the one-CTA-per-point LU (the same arithmetic on every
element), and reach the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return rsrr


PROBLEMS = [
    (lambda: W.rational_grid(g=30, N=8, L=4), 1),
    (lambda: W.rational_grid(g=55, N=16, L=8), 1),
    (lambda: W.random_banded(n=900, kl=240, ku=30, N=3, L=3, seed=13), 1),
    (lambda: W.random_banded(n=500, kl=5, ku=9, N=6, L=5, seed=14), 0),
    (lambda: W.rational_grid(g=40, N=5, L=3), 0),
]


def test_batch_equals_each_lone_sample_bitwise(rs):
    probs = [(make(), prec) for make, prec in PROBLEMS]
    lone = []
    for p, prec in probs:
        s = rs.Solver(p, rs.default_opts(precision=prec, flags=rs.RSRR_FLAG_ONE_CTA_LU))
        s.sample()
        assert s.check_status() == rs.RSRR_OK
        lone.append(s.samples())
        s.close()
    solvers = [rs.Solver(p, rs.default_opts(precision=prec)) for p, prec in probs]
    rs.sample_batch(solvers)
    for sv, ref, (p, prec) in zip(solvers, lone, probs):
        assert sv.check_status() == rs.RSRR_OK
        S = sv.samples()
        assert np.array_equal(S, ref)
        z = oracle.sample_points(p.region, p.N)
        X0 = oracle.resolvent_samples(p, z[:1])[0]
        assert oracle.backward_error_inf(p, z[0], S[:, :p.L]).max() <= (1e-10 if prec == 1 else 1e-14)
        assert np.abs(S[:, :p.L] - X0).max() <= 1e-6 * np.abs(X0).max()
    for sv in solvers:
        sv.close()


def test_batch_refuses_dense_handles(rs):
    a = rs.Solver(W.rational_grid(g=20, N=4, L=2))
    b = rs.Solver(W.helmholtz_sphere(n=64, N=4, L=2))
    with pytest.raises(rs.RSRRError) as e:
        rs.sample_batch([a, b])
    assert e.value.status == rs.RSRR_EINVAL
    a.close()
    b.close()
