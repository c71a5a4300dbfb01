"""rsrr_solve_band_noalloc, the allocation-free banded solve for callers that
cannot call cudaMalloc (plug-ins whose host application has reserved the
device memory through its own pool, loops that must stay out of the
allocator).  Its solutions are checked against the regular entry point
(rsrr_create + rsrr_sample, FP64 path) on two calls in a row; the second
call uses a smaller problem, so anything left in the shared scratch by the
first call would show up.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return torch, rsrr


def lapack_band(p, z):
    """T(z) in the LAPACK general band layout (kl+ku+1) x n, column major."""
    kl, ku = p.bandwidths()
    T = oracle.assemble(p, z).tocoo()
    ab = np.zeros((kl + ku + 1, p.n), dtype=np.complex128)
    ab[ku + T.row - T.col, T.col] = T.data
    return np.asfortranarray(ab), kl, ku


def regular_entry_point(rsrr, p, z):
    """X = T(z)^{-1} U through rsrr_create / rsrr_sample (FP64 path)."""
    q = W.Problem(p.name, p.n, p.row_ptr, p.col_idx, p.values, p.fns,
                  W.Region(p.region.center, p.region.a, p.region.b, kind="points",
                           points=np.array([z])), 1, p.L, p.U)
    s = rsrr.Solver(q, rsrr.default_opts(precision=rsrr.RSRR_PREC_FP64))
    s.sample()
    s.check()
    X = s.samples()
    s.close()
    return X


def noalloc(torch, rsrr, p, z):
    ab, kl, ku = lapack_band(p, z)
    dev = torch.device("cuda")
    band = torch.from_numpy(ab.T.copy()).to(dev)          # column-major (kl+ku+1) x n
    U = torch.from_numpy(np.ascontiguousarray(p.U.T)).to(dev)  # column-major n x L
    X = torch.empty_like(U)
    stream = torch.cuda.current_stream()
    st = rsrr.rsrr_solve_band_noalloc(p.n, kl, ku, ctypes.c_void_p(band.data_ptr()), p.L,
                                      ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))
    assert st == rsrr.RSRR_OK, rsrr.rsrr_last_error(None).decode()
    return X.cpu().numpy().T


def test_noalloc_matches_the_regular_entry_point_twice(env):
    torch, rsrr = env
    cases = [(W.random_banded(n=700, kl=9, ku=6, N=1, L=5, seed=7), 0.3 + 0.2j),
             (W.random_banded(n=150, kl=3, ku=4, N=1, L=3, seed=8), -0.1 + 0.05j)]
    for p, z in cases:
        X_new = noalloc(torch, rsrr, p, z)
        X_ref = regular_entry_point(rsrr, p, z)
        # the FP64-path tolerance of the sampling parity tests
        assert np.abs(X_new - X_ref).max() <= 1e-9 * np.abs(X_ref).max()


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch(env):
    torch, rsrr = env
    dev = torch.device("cuda")
    dummy = torch.zeros(4, dtype=torch.complex128, device=dev)
    ptr = ctypes.c_void_p(dummy.data_ptr())
    st = rsrr.rsrr_solve_band_noalloc(1 << 20, 100, 100, ptr, 1, ptr, ptr, None)
    assert st == rsrr.RSRR_EINVAL
    assert b"fixed maximum" in rsrr.rsrr_last_error(None)
