"""Autotuner for the batched path's tile parameters.

The results of integration do not depend on the tile parameters (segment
length in dominant-axis steps, blocks per SM of the walk kernel), only the
speed does.  The tuner builds scratch maps with the caller's parameters, runs
a few representative steps per candidate through a captured CUDA graph, times
them with CUDA events and returns the fastest candidate.  The caller's own
maps are never touched.
"""
import itertools

import torch

from . import ohm

DEFAULT_SEGMENT_STEPS = (6, 10, 16, 24)
DEFAULT_WALK_BLOCKS = (2, 3, 4)


def time_batch_steps(batch: "ohm.Batch", steps, stream, warmup=2):
    """Mean device milliseconds per step of `steps` (lists of per-map ray sets)."""
    for s in steps[:warmup]:
        with torch.cuda.stream(stream):
            batch.integrate(s, graph=True)
    batch.sync(stream)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for s in steps:
        with torch.cuda.stream(stream):
            batch.integrate(s, graph=True)
    end.record(stream)
    batch.sync(stream)
    return start.elapsed_time(end) / len(steps)


def autotune_batch(map_params, sample_steps, segment_steps=DEFAULT_SEGMENT_STEPS,
                   walk_blocks=DEFAULT_WALK_BLOCKS, stream=None):
    """Pick (segment_steps, walk_blocks_per_sm) for maps built from
    `map_params` (a list of parameter dicts) on the step inputs
    `sample_steps`.  Returns (best, table) where table maps each candidate to
    its mean milliseconds per step."""
    stream = stream or torch.cuda.Stream()
    table = {}
    for S, B in itertools.product(segment_steps, walk_blocks):
        maps = [ohm.Map(**p) for p in map_params]
        batch = ohm.Batch(maps)
        batch.tune(S, B)
        table[(S, B)] = time_batch_steps(batch, sample_steps, stream)
        batch.close()
        for m in maps:
            m.close()
    best = min(table, key=table.get)
    return best, table
