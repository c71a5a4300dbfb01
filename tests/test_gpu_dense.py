"""GPU parity of the dense kernel path (T(z)_ij = exp(i z r_ij)/(4 pi r_ij)):
samples X_j = T(z_j)^{-1} U, the Taylor projection P_p = Q^H A_p Q and the
eigenpairs, through the C ABI, against the FP64 oracle."""
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


# gemm 0: the residual products T X in native FP64 at these sizes; gemm 2:
# forced onto the FP64-accurate tensor-core slices (the large sizes' default)
@pytest.mark.parametrize("n,N,L,prec,gemm", [(256, 6, 8, "mixed", 0), (300, 4, 5, "mixed", 0),
                                             (70, 3, 3, "mixed", 0), (256, 4, 8, "fp64", 0),
                                             (300, 4, 5, "mixed", 2), (200, 3, 7, "fp64", 2)])
def test_dense_samples_match_oracle(rs, n, N, L, prec, gemm):
    p = W.helmholtz_sphere(n=n, N=N, L=L)
    o = rs.default_opts(precision=rs.RSRR_PREC_MIXED if prec == "mixed" else rs.RSRR_PREC_FP64,
                        gemm=gemm)
    s = rs.Solver(p, o)
    s.sample()
    assert s.check_status() == rs.RSRR_OK
    S, eta, z = s.samples(), s.eta(), s.points()
    s.close()
    zo = oracle.sample_points(p.region, p.N)
    assert np.abs(z - zo).max() <= 1e-13 * np.abs(zo).max()
    ref = oracle.resolvent_samples_dense(p, zo)
    tol_eta = 1e-10 if prec == "mixed" else 1e-14
    for j, Xr in enumerate(ref):
        Xg = S[:, j * L:(j + 1) * L]
        e = oracle.backward_error_inf_dense(p, zo[j], Xg)
        assert e.max() <= tol_eta
        assert np.allclose(eta[j * L:(j + 1) * L], e, rtol=1e-3, atol=max(1e-3 * tol_eta, 1e-14))
        assert np.abs(Xg - Xr).max() <= (1e-6 if prec == "mixed" else 1e-9) * np.abs(Xr).max()


@pytest.mark.parametrize("n", [64, 128])
def test_dense_eigenpairs_match_oracle(rs, n):
    p = W.helmholtz_sphere(n=n, N=32, L=16)
    ref = oracle.rsrr_dense(p, NQ=256)
    s = rs.Solver(p, rs.default_opts(NQ=256))
    s.sample()
    s.check()
    s.project()
    out = s.solve()
    Q = s.Q()
    P = s.projected()
    st = s.stats()
    s.close()
    assert len(out["lam"]) == len(ref["lam"]) > 0
    assert match_eigs(ref["lam"], out["lam"]) <= 1e-9
    assert out["res"].max() <= 1e-10
    for lam, v in zip(out["lam"], out["V"].T):
        assert oracle.residual_dense(p, lam, v) <= 1e-10
    # projected Taylor coefficients equal Q^H A_p Q for the GPU's own Q
    A = oracle.taylor_coefficients(p)
    assert st["m"] == len(A)
    for q in (0, 1, 5, len(A) - 1):
        Pr = Q.conj().T @ A[q] @ Q
        assert np.abs(P[q] - Pr).max() <= 1e-12 * max(np.abs(A[q]).sum(axis=0).max(), 1e-300)


@pytest.mark.parametrize("n,N,L", [(300, 4, 5), (160, 3, 8), (129, 2, 3)])
def test_tensor_core_dense_update_matches_the_fma_update(rs, n, N, L):
    """The complex64 LU's trailing updates on the tensor cores (3xTF32) and on
    FP32 FMAs: one solve from each factor agrees to complex64 rounding, and
    both refine to the oracle."""
    p = W.helmholtz_sphere(n=n, N=N, L=L)
    out = {}
    for name, flags in (("tc", 0), ("simt", rs.RSRR_FLAG_SIMT_DENSE_UPDATE)):
        s = rs.Solver(p, rs.default_opts(max_refine=0, flags=flags))
        s.sample()
        S0 = s.samples()
        s.close()
        s = rs.Solver(p, rs.default_opts(flags=flags))
        s.sample()
        assert s.check_status() == rs.RSRR_OK
        out[name] = (S0, s.samples(), s.eta())
        s.close()
    a0, b0 = out["tc"][0], out["simt"][0]
    assert np.abs(a0 - b0).max() <= 1e-4 * np.abs(b0).max()
    zo = oracle.sample_points(p.region, p.N)
    ref = oracle.resolvent_samples_dense(p, zo)
    for name in out:
        S, eta = out[name][1], out[name][2]
        assert eta.max() <= 1e-10
        for j, Xr in enumerate(ref):
            assert np.abs(S[:, j * L:(j + 1) * L] - Xr).max() <= 1e-6 * np.abs(Xr).max()
