"""The synthetic inputs are the stated recipe: seeded and reproducible, with the
shapes, sizes and structure of the benchmark workloads (no method arithmetic
here; these are the inputs both the oracle and the GPU path receive)."""
import numpy as np

import workloads as W


def test_benchmark_grid_workload_has_the_stated_shape():
    p = W.config("c1")
    assert (p.n, p.N, p.L, p.m) == (40000, 64, 32, 3)
    rows = np.repeat(np.arange(p.n), np.diff(p.row_ptr))
    cols = np.asarray(p.col_idx)
    assert np.abs(rows - cols).max() == 200  # natural ordering: half-bandwidth g
    K, M, E = (np.asarray(v) for v in p.values)
    assert np.count_nonzero(K) == 199_200  # 5-point stencil on a 200 x 200 grid
    assert np.array_equal(M != 0, rows == cols) and np.all(M[rows == cols] == 1.0)  # M = I
    assert np.count_nonzero(E) == 400 and np.all((E != 0) <= (rows == cols))  # 1% of the diagonal
    assert np.allclose(K[rows == cols], 4.0 * 201 ** 2)
    assert p.U.shape == (40000, 32) and p.U.flags.f_contiguous
    reg = p.region
    assert (reg.center, reg.a, reg.b) == (100.0, 80.0, 20.0)


def test_inputs_are_reproducible_from_their_seeds():
    a, b = W.config("c1", g=40), W.config("c1", g=40)
    assert np.array_equal(a.U, b.U)
    assert all(np.array_equal(x, y) for x, y in zip(a.values, b.values))
    c = W.config("c1", g=40, seed_u=7)
    assert not np.array_equal(a.U, c.U)


def test_probe_entries_are_standard_complex_normal():
    U = W.probe(20000, 4, 123)
    z = U.ravel()
    # (g1 + i g2)/sqrt(2): E|u|^2 = 1, real and imaginary parts each of variance 1/2
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.02
    assert abs(np.var(z.real) - 0.5) < 0.01 and abs(np.var(z.imag) - 0.5) < 0.01
    assert abs(np.mean(z)) < 0.01


def test_dense_workload_points_lie_on_the_unit_sphere():
    p = W.helmholtz_sphere(n=512, N=8, L=4)
    r = np.linalg.norm(p.points, axis=1)
    assert np.abs(r - 1.0).max() < 1e-12
    d = np.linalg.norm(p.points[:, None] - p.points[None, :], axis=2)
    np.fill_diagonal(d, np.inf)
    h = d.min(axis=1).mean()
    assert abs(p.diag - 1.0 / (2.0 * h)) <= 1e-12 * p.diag  # diagonal 1/(2h)
