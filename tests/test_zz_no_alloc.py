"""rsrr_solve_band_noalloc, the allocation-free banded solve for callers that
cannot call cudaMalloc (plug-ins whose host application has reserved the
device memory through its own pool, loops that must stay out of the
allocator).

Its solutions are checked against the CPU oracle (LAPACK banded solve of the
same T(z) and U) and against the regular entry point (rsrr_create +
rsrr_sample, FP64 path) on two calls in a row; the second call uses a smaller
problem, so anything left in the shared scratch by the first call would show
up.  Around the calls after the first (which loads the library's device code
and with it the fixed scratch array), the device's free memory and the torch
allocator's statistics must not move: the entry point allocates nothing.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-9  # the FP64-path tolerance of the sampling parity tests (relative to max |X|)


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


def device_inputs(torch, p, z):
    ab, kl, ku = lapack_band(p, z)
    dev = torch.device("cuda")
    band = torch.from_numpy(ab.T.copy()).to(dev)               # column-major (kl+ku+1) x n
    U = torch.from_numpy(np.ascontiguousarray(p.U.T)).to(dev)  # column-major n x L
    X = torch.empty_like(U)
    return band, U, X, kl, ku


def call(rsrr, torch, p, band, U, X, kl, ku):
    stream = torch.cuda.current_stream()
    return rsrr.rsrr_solve_band_noalloc(p.n, kl, ku, ctypes.c_void_p(band.data_ptr()), p.L,
                                        ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(X.data_ptr()),
                                        ctypes.c_void_p(stream.cuda_stream))


CASES = [(dict(n=700, kl=9, ku=6, N=1, L=5, seed=7), 0.3 + 0.2j),
         (dict(n=150, kl=3, ku=4, N=1, L=3, seed=8), -0.1 + 0.05j)]


def test_noalloc_matches_the_oracle_and_the_regular_entry_point_twice(env):
    torch, rsrr = env
    probs = [(W.random_banded(**kw), z) for kw, z in CASES]
    inputs = [device_inputs(torch, p, z) for p, z in probs]
    torch.cuda.synchronize()
    # warm-up calls: load the library's device code (each kernel the calls
    # use), which brings the fixed scratch array into device memory
    for (p, _), inp in zip(probs, inputs):
        assert call(rsrr, torch, p, *inp) == rsrr.RSRR_OK, rsrr.rsrr_last_error(None).decode()
        inp[2].zero_()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    # two calls in a row, the second on a smaller problem
    outs = []
    for (p, z), inp in zip(probs, inputs):
        st = call(rsrr, torch, p, *inp)
        assert st == rsrr.RSRR_OK, rsrr.rsrr_last_error(None).decode()
        outs.append(inp[2].cpu().numpy().T)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0, (free0, free1)
    for key in ("allocation.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    for (p, z), X_new in zip(probs, outs):
        X_orc = oracle.resolvent_samples(p, np.array([z]))[0]
        scale = np.abs(X_orc).max()
        assert np.abs(X_new - X_orc).max() <= TOL * scale
        X_ref = regular_entry_point(rsrr, p, z)
        assert np.abs(X_new - X_ref).max() <= TOL * scale


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch(env):
    torch, rsrr = env
    dev = torch.device("cuda")
    dummy = torch.zeros(4, dtype=torch.complex128, device=dev)
    ptr = ctypes.c_void_p(dummy.data_ptr())
    st = rsrr.rsrr_solve_band_noalloc(1 << 20, 100, 100, ptr, 1, ptr, ptr, None)
    assert st == rsrr.RSRR_EINVAL
    assert b"fixed maximum" in rsrr.rsrr_last_error(None)
    # an upper bandwidth beyond n - 1 is refused before anything runs
    st = rsrr.rsrr_solve_band_noalloc(16, 2, 1 << 20, ptr, 1, ptr, ptr, None)
    assert st == rsrr.RSRR_EINVAL
    assert b"at most n - 1" in rsrr.rsrr_last_error(None)
