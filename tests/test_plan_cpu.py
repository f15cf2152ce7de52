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


def test_oracle_plan_covers_every_output_once_with_fewest_tiles():
    """Properties any valid table must have, found by search rather than by
    the plan's own formula: problem i owns one contiguous run of tiles in
    problem order; that run, spread evenly over its right-hand sides, is the
    product of the fewest 128-row tiles covering `rest` rows and the fewest
    chunks of at most `cap` columns (each a multiple of 16, the MMA's N step)
    covering the n_out output columns, so every output element lies in
    exactly one tile and no tile is empty."""
    rng = np.random.default_rng(11)
    probs = [(int(rng.integers(1, 520)), int(rng.integers(1, 900)), int(rng.integers(1, 9)))
             for _ in range(60)] + [(16, 128, 1), (17, 129, 2), (128, 256, 1), (129, 1, 3)]

    def fewest(total, width):
        k = 1
        while k * width < total:
            k += 1
        return k

    for cap in (64, 128):
        first, tp = plan.tile_table(probs, cap)
        assert tp == sorted(tp)
        for i, (n_out, rest, nrhs) in enumerate(probs):
            count = tp.count(i)
            assert first[i] == (tp.index(i) if count else len(tp))
            assert count % nrhs == 0
            n16 = next(w for w in range(n_out, n_out + 16) if w % 16 == 0)
            # the fewest chunks whose width (a multiple of 16, <= cap) covers n16
            chunks = next(k for k in range(1, n16 + 1)
                          if -(-(-(-n16 // k)) // 16) * 16 <= cap)
            assert count // nrhs == fewest(rest, 128) * chunks
            assert chunks == fewest(n16, cap)
