"""The batched launch plan's integer tables (cola_batch_tile_table, the table
cola_cg_solve_batched uploads) against the oracle's definition, bit for bit,
and the oracle against a brute-force enumeration of tiles.  No GPU needed."""
import ctypes

import numpy as np
import pytest

import workloads as wl
from oracle import plan


@pytest.fixture(scope="module")
def lib():
    from paper_2309_03060_gb300 import build, _abi
    build.build()
    return _abi.load()


def _enumerate(problems, cap):
    """Every (problem, rhs, row tile, chunk) in problem-major order."""
    out = []
    for i, (n_out, rest, nrhs) in enumerate(problems):
        n16 = -(-n_out // 16) * 16
        nch = 1
        while -(-n16 // nch) > cap:
            nch += 1
        for r in range(nrhs):
            for m0 in range(0, rest, 128):
                for c in range(nch):
                    out.append(i)
    return out


def test_oracle_plan_matches_enumeration():
    rng = np.random.default_rng(7)
    probs = [(int(rng.integers(1, 300)), int(rng.integers(1, 700)), int(rng.integers(1, 9)))
             for _ in range(40)]
    for cap in (64, 128):
        first, tp = plan.tile_table(probs, cap)
        assert tp == _enumerate(probs, cap)
        assert first == [tp.index(i) for i in range(len(probs))]


def _call(lib, probs, cap, capacity=None):
    n = len(probs)
    n_out = (ctypes.c_int32 * n)(*[p[0] for p in probs])
    rest = (ctypes.c_int64 * n)(*[p[1] for p in probs])
    nrhs = (ctypes.c_int64 * n)(*[p[2] for p in probs])
    first = (ctypes.c_int64 * max(n, 1))()
    total = ctypes.c_int64()
    cap_n = capacity if capacity is not None else sum(
        plan.problem_tiles(*p, cap) for p in probs)
    tp = (ctypes.c_int32 * max(cap_n, 1))()
    st = lib.cola_batch_tile_table(n, n_out, rest, nrhs, cap, first, tp, cap_n,
                                   ctypes.byref(total))
    return st, list(first)[:n], list(tp)[:total.value], total.value


@pytest.mark.parametrize("cap", [64, 128])
def test_batch_tile_table_bit_exact_on_the_batched_workload(lib, cap):
    """The 512-system batched workload's two mode steps (rest = the other factor's side)."""
    w4 = wl.config4()
    for step in (0, 1):
        probs = []
        for s in w4.systems:
            n1, n2 = s.factors[0].shape[0], s.factors[1].shape[0]
            n_out, rest = (n1, n2) if step == 0 else (n2, n1)
            probs.append((n_out, rest, s.B.shape[0]))
        st, first, tp, total = _call(lib, probs, cap)
        assert st == 0
        f_ref, tp_ref = plan.tile_table(probs, cap)
        assert total == len(tp_ref)
        assert first == f_ref
        assert tp == tp_ref


def test_batch_tile_table_edge_cases(lib):
    # one-row problems, widths at chunk boundaries, empty plan
    probs = [(1, 1, 1), (16, 128, 1), (17, 129, 2), (128, 256, 3), (129, 1, 1), (8192, 5, 1)]
    st, first, tp, total = _call(lib, probs, 128)
    f_ref, tp_ref = plan.tile_table(probs, 128)
    assert st == 0 and first == f_ref and tp == tp_ref
    st, _, _, total = _call(lib, [], 128)
    assert st == 0 and total == 0
    # capacity too small: error, total still reported
    st, _, _, total = _call(lib, probs, 128, capacity=3)
    assert st == 1 and total == len(tp_ref)
    # invalid chunk cap
    st, *_ = _call(lib, probs, 96)
    assert st == 1
