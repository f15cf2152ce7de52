"""The table-driven batched launch plan by its definition.  Test infrastructure only.

The batched solve runs one mode step of many Kronecker systems in a single
launch that walks a global tile table (no counterpart in the paper; it is how
the uneven systems share the GPU).  A tile is 128 consecutive rows of one
right-hand side's current layout times one chunk of output columns.  The
output width is padded to a multiple of 16 and split into the fewest equal
chunks of at most ``cap`` columns.  Problem i owns a contiguous run of tiles,
in problem order.
"""
from __future__ import annotations


def output_chunks(n_out: int, cap: int) -> int:
    n16 = (n_out + 15) // 16 * 16
    return (n16 + cap - 1) // cap


def problem_tiles(n_out: int, rest: int, nrhs: int, cap: int) -> int:
    return (rest + 127) // 128 * nrhs * output_chunks(n_out, cap)


def tile_table(problems, cap: int):
    """problems: [(n_out, rest, nrhs)].  Returns (first, tile_prob)."""
    first, tile_prob = [], []
    for i, (n_out, rest, nrhs) in enumerate(problems):
        first.append(len(tile_prob))
        tile_prob.extend([i] * problem_tiles(n_out, rest, nrhs, cap))
    return first, tile_prob
