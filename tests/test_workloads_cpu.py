"""The seeded input generators: determinism, shapes and the stated ranges."""
import numpy as np

import bench
import workloads as wl


def test_generators_are_deterministic():
    a, b = wl.kron_diag("x", [6, 5], [0.2, 0.3], 0.1, 0.2, 2, 1e-8, 9), \
        wl.kron_diag("x", [6, 5], [0.2, 0.3], 0.1, 0.2, 2, 1e-8, 9)
    assert np.array_equal(a.B, b.B) and np.array_equal(a.extra["d"], b.extra["d"])
    m1, m2 = wl.multitask(3, 4, 10), wl.multitask(3, 4, 10)
    assert all(np.array_equal(x, y) for x, y in zip(m1.B + m1.K, m2.B + m2.K))
    assert np.array_equal(wl.bipoisson(8, 2).B, wl.bipoisson(8, 2).B)


def test_stated_ranges_and_shapes():
    w = wl.kron_diag("x", [6, 5], [0.2, 0.3], 0.1, 0.2, 2, 1e-8, 9)
    d = w.extra["d"]
    assert d.shape == (30,) and d.min() >= 0.1 and d.max() <= 0.2 and w.B.shape == (2, 30)
    h = wl.config2_hetero(n=8, nrhs=3)
    assert h.N == 512 and h.extra["d"].min() >= 0.005 and h.extra["d"].max() <= 0.015
    m = wl.multitask(3, 4, 10)
    assert m.N == 40 and len(m.coeffs) == 3
    for b in m.B:   # a a^T + diag(k) with positive loadings: entrywise positive, SPD
        assert np.all(b > 0) and np.all(np.linalg.eigvalsh(b) > 0)
    p = wl.bipoisson(8, 2)
    assert p.N == 64 and p.B.shape == (2, 64) and p.tol == 1e-11
    assert np.array_equal(p.L, wl.dirichlet_laplacian(8))


def test_optional_bench_section_reports_errors():
    assert bench.optional_section(lambda: {"ok": 1}, True) == {"ok": 1}
    assert bench.optional_section(lambda: 1 / 0, False) is None
    err = bench.optional_section(lambda: 1 / 0, True)
    assert err["error"].startswith("ZeroDivisionError")
