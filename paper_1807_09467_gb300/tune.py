"""Launch-shape autotuner of the batched form.

The one launch-shape knob of the fused passes that can change at run time is
how many 256-row tiles each block owns (``Solver(tiles_per_block=...)``): the
sliced-ELL slice height (32 rows, one lane per row of a warp) and the tile (the
sorting window of the slices, eight slices, one per warp of a 256-thread block)
are fixed by the kernels' layout, and the blocks a multiprocessor holds are
fixed per build.  More tiles a block means fewer blocks a system: alone, a
system wants every SM; in a batch, systems that each take fewer blocks leave
room for more of them at once.  The tuner measures instead of guessing: the
caller supplies a trial that runs representative work with a given cap on the
blocks of any one system and returns its time, and the tuner keeps the fastest
cap.  Host logic only; the trials run the library's kernels.
"""
from __future__ import annotations

TILE = 256


def tiles_per_block(n: int, max_blocks: int | None) -> int:
    """The tiles_per_block that keeps a system of n rows within max_blocks
    blocks (0: the library's automatic choice, i.e. no cap)."""
    if not max_blocks:
        return 0
    ntile = (n + TILE - 1) // TILE
    return max(1, -(-ntile // max_blocks))


def blocks(n: int, tpb: int, auto_blocks: int) -> int:
    """Blocks of a system of n rows with tiles_per_block tpb (auto_blocks: the
    grid cap of the automatic choice, blocks per SM x SMs)."""
    ntile = (n + TILE - 1) // TILE
    if tpb <= 0:
        nb = max(1, min(ntile, auto_blocks))
        tpb = -(-ntile // nb)
    tpb = min(tpb, ntile)
    return -(-ntile // tpb)


def tune(trial, candidates, repeats: int = 1):
    """Run trial(c) for each candidate c (repeats times, keeping the fastest
    time of each) and return (best candidate, {candidate: ms}).  Ties keep the
    earlier candidate, so list the default first."""
    if not candidates:
        raise ValueError("no candidates")
    times = {}
    for c in candidates:
        ms = min(float(trial(c)) for _ in range(max(1, repeats)))
        if not ms >= 0.0:
            raise ValueError(f"trial({c!r}) returned {ms!r}")
        times[c] = ms
    best = min(candidates, key=lambda c: (times[c], candidates.index(c)))
    return best, times
