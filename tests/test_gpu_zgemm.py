"""The projection's dense complex products through rsrr_zgemm, for both
methods: native FP64 and the sliced bf16 tensor-core (Ozaki) scheme.

Checks that hold independently of either implementation:
  * integer inputs small enough that every FP64 sum is exact: both methods
    must return the exact product bit for bit (numpy's complex128 product of
    the same integers is exact too);
  * random inputs with rows and columns scaled over a wide exponent range:
    the error against an extended-precision product stays below
    4 K 2^-53 max|a_i.| max|b_.j| (the scheme's bound, up to a factor);
  * Hermitian Gram matrices come back exactly Hermitian;
  * chunking K (small work space) and splitting K across CTAs do not change
    the result beyond FP64 rounding of the partial sums.
Shapes are ragged on purpose (M, N, K not multiples of the 64 x 64 tiles or
of the 16-deep K steps)."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1605_07951_gb300 import rsrr
    return torch, rsrr


def dev(torch, X):
    """column-major complex128 device copy of X (as a transposed C-order tensor)"""
    return torch.from_numpy(np.ascontiguousarray(X.T)).to("cuda")


def zgemm(env, A, B, conjA, method, C0=None, alpha=1.0, beta=0.0, hermitian=False, ws=0):
    torch, rsrr = env
    M = A.shape[1] if conjA else A.shape[0]
    K = A.shape[0] if conjA else A.shape[1]
    N = B.shape[1]
    dA = dev(torch, A)
    dB = dA if (hermitian and B is A) else dev(torch, B)
    dC = dev(torch, C0 if C0 is not None else np.full((M, N), np.nan + 1j * np.nan))
    st = rsrr.rsrr_zgemm(M, N, K, int(conjA), ctypes.c_void_p(dA.data_ptr()), A.shape[0],
                         ctypes.c_void_p(dB.data_ptr()), B.shape[0], ctypes.c_void_p(dC.data_ptr()),
                         M, alpha, beta, method, int(hermitian), ws, None)
    assert st == rsrr.RSRR_OK, rsrr.rsrr_last_error(None).decode()
    return dC.cpu().numpy().T


def rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def exact_product(A, B, conjA):
    """extended-precision reference product (long double accumulation)"""
    a = (A.conj().T if conjA else A)
    ar, ai = a.real.astype(np.longdouble), a.imag.astype(np.longdouble)
    br, bi = B.real.astype(np.longdouble), B.imag.astype(np.longdouble)
    return ar @ br - ai @ bi, ar @ bi + ai @ br


METHODS = [(1, "fp64"), (2, "ozaki_tcgen05"), (3, "ozaki_mma")]
SHAPES = [(1, 1, 1), (37, 53, 29), (130, 70, 301), (64, 128, 1000), (200, 9, 777)]


@pytest.mark.parametrize("method", [m for m, _ in METHODS], ids=[n for _, n in METHODS])
@pytest.mark.parametrize("conjA", [False, True], ids=["A", "AH"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{m}x{n}x{k}" for m, n, k in SHAPES])
def test_integer_products_are_exact(env, method, conjA, shape):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    ints = lambda *s: (rng.integers(-1000, 1001, s) + 1j * rng.integers(-1000, 1001, s)).astype(np.complex128)
    A = ints(K, M) if conjA else ints(M, K)
    B = ints(K, N)
    # scale rows of op(A) and columns of B by powers of two: still exact
    B = B * (2.0 ** rng.integers(-40, 40, N))[None, :]
    ref = (A.conj().T if conjA else A) @ B
    got = zgemm(env, A, B, conjA, method)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("method", [m for m, _ in METHODS], ids=[n for _, n in METHODS])
@pytest.mark.parametrize("conjA", [False, True], ids=["A", "AH"])
@pytest.mark.parametrize("shape", SHAPES[1:], ids=[f"{m}x{n}x{k}" for m, n, k in SHAPES[1:]])
def test_scaled_random_products_within_the_bound(env, method, conjA, shape):
    M, N, K = shape
    rng = np.random.default_rng(1000 + M + N + K)
    A = rand(rng, K, M) if conjA else rand(rng, M, K)
    if conjA:
        A *= (2.0 ** rng.integers(-300, 300, M))[None, :]
    else:
        A *= (2.0 ** rng.integers(-300, 300, M))[:, None]
    B = rand(rng, K, N) * (2.0 ** rng.integers(-300, 300, N))[None, :]
    A[rng.random(A.shape) < 0.05] = 0.0       # scattered zeros
    got = zgemm(env, A, B, conjA, method)
    rr, ri = exact_product(A, B, conjA)
    a = A.conj().T if conjA else A
    amax = np.maximum(np.abs(a.real), np.abs(a.imag)).max(axis=1)
    bmax = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=0)
    bound = 4 * K * 2.0 ** -53 * np.outer(amax, bmax)
    err_r = np.abs(got.real.astype(np.longdouble) - rr).astype(np.float64)
    err_i = np.abs(got.imag.astype(np.longdouble) - ri).astype(np.float64)
    assert np.all(err_r <= bound) and np.all(err_i <= bound)


@pytest.mark.parametrize("method", [2, 3], ids=["ozaki_tcgen05", "ozaki_mma"])
@pytest.mark.parametrize("shape", [(64, 5000), (100, 3001), (192, 20000), (320, 1024)])
def test_hermitian_gram_is_exactly_hermitian(env, shape, method):
    N, K = shape
    rng = np.random.default_rng(N + K)
    S = rand(rng, K, N)
    S /= np.linalg.norm(S, axis=0)
    G = zgemm(env, S, S, True, method, hermitian=True)
    assert np.array_equal(G, G.conj().T)
    rr, ri = exact_product(S, S, True)
    ref = (rr + 1j * ri).astype(np.complex128)
    amax = np.maximum(np.abs(S.real), np.abs(S.imag)).max(axis=0)
    bound = 4 * K * 2.0 ** -53 * np.outer(amax, amax)
    assert np.all(np.abs(G - ref) <= bound + 1e-300)


@pytest.mark.parametrize("method", [2, 3], ids=["ozaki_tcgen05", "ozaki_mma"])
def test_chunked_and_split_K_agree_with_the_whole_product(env, method):
    torch, rsrr = env
    rng = np.random.default_rng(5)
    M, N, K = 40, 24, 20000   # few tiles, long K: split across CTAs
    A = rand(rng, K, M)
    B = rand(rng, K, N)
    whole = zgemm(env, A, B, True, method)
    # a work space for a fraction of K forces chunks of K
    chunked = zgemm(env, A, B, True, method, ws=14 * (128 + 64) * 2 * 4096 + 4096)
    scale = np.abs(A).max() * np.abs(B).max() * K
    assert np.abs(whole - chunked).max() <= 8 * K * 2.0 ** -53 * np.abs(A).max() * np.abs(B).max()
    rr, ri = exact_product(A, B, True)
    assert np.abs(whole.real - rr.astype(np.float64)).max() <= 4 * 2.0 ** -53 * scale


def test_alpha_beta_and_empty_depth(env):
    rng = np.random.default_rng(9)
    M, N, K = 70, 33, 450
    A = rand(rng, M, K)
    B = rand(rng, K, N)
    C0 = rand(rng, M, N)
    for method in (1, 2, 3):
        got = zgemm(env, A, B, False, method, C0=C0, alpha=-1.0, beta=1.0)
        ref = C0 - A @ B
        assert np.abs(got - ref).max() <= 1e-12 * (np.abs(A) @ np.abs(B)).max()
        # K = 0: C = beta C
        torch, rsrr = env
        dC = dev(torch, C0)
        st = rsrr.rsrr_zgemm(M, N, 0, 0, None, M, None, 1, ctypes.c_void_p(dC.data_ptr()), M,
                             1.0, 0.5, method, 0, 0, None)
        assert st == rsrr.RSRR_OK
        assert np.array_equal(dC.cpu().numpy().T, 0.5 * C0)


def test_bad_arguments_are_rejected(env):
    torch, rsrr = env
    x = torch.zeros(4, dtype=torch.complex128, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    assert rsrr.rsrr_zgemm(2, 2, 2, 0, p, 1, p, 2, p, 2, 1.0, 0.0, 2, 0, 0, None) == rsrr.RSRR_EINVAL
    assert rsrr.rsrr_zgemm(2, 2, 2, 0, p, 2, p, 2, p, 2, 1.0, 0.0, 7, 0, 0, None) == rsrr.RSRR_EINVAL
    # hermitian needs A^H A
    assert rsrr.rsrr_zgemm(2, 2, 2, 0, p, 2, p, 2, p, 2, 1.0, 0.0, 2, 1, 0, None) == rsrr.RSRR_EINVAL


@pytest.mark.parametrize("shape", [(256, 128, 3000), (130, 70, 5001)])
def test_tcgen05_and_mma_slice_products_agree(env, shape):
    """The two kernels sum the same exact slice products; only the rounded
    sixth group (relative weight <= 2^-40) may differ."""
    M, N, K = shape
    rng = np.random.default_rng(M * N + K)
    A = rand(rng, K, M)
    B = rand(rng, K, N)
    a = zgemm(env, A, B, True, 2)
    b = zgemm(env, A, B, True, 3)
    amax = np.maximum(np.abs(A.real), np.abs(A.imag)).max(axis=0)
    bmax = np.maximum(np.abs(B.real), np.abs(B.imag)).max(axis=0)
    assert np.all(np.abs(a - b) <= 2 * K * 2.0 ** -53 * np.outer(amax, bmax))


def test_bounded_wait_runs_out_and_the_context_stays_usable(env):
    """Failure detection without a GPU fault: a bounded wait on a barrier that
    nothing completes gives up, is counted and reported as ETIMEOUT; products
    and whole solves afterwards succeed."""
    torch, rsrr = env
    assert rsrr.rsrr_check_wait_timeout(256, None) == rsrr.RSRR_ETIMEOUT
    assert b"ran out" in rsrr.rsrr_last_error(None)
    assert rsrr.rsrr_check_wait_timeout(0, None) == rsrr.RSRR_EINVAL
    torch.cuda.synchronize()
    # the counter is compared around each call: a later product is not blamed
    rng = np.random.default_rng(5)
    A = rng.integers(-9, 10, (256, 512)) + 1j * rng.integers(-9, 10, (256, 512))
    B = rng.integers(-9, 10, (512, 64)) + 1j * rng.integers(-9, 10, (512, 64))
    C = zgemm(env, A, B, False, 2)
    assert np.array_equal(C, A @ B)
