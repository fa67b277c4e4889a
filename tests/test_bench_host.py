"""Host-side logic of bench.py: the ALU work model counted from a trace (one
recurrence term per distinct index selected before), and the seeded block
samples of the CPU baselines."""
import os
import sys
import types

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2207_01205_gb300 import synth  # noqa: E402

TRACE = np.dtype([("u1", "<i2"), ("u2", "<i2"), ("re", "<f4"), ("im", "<f4")])


def test_alu_work_counts_distinct_prefix_terms():
    specs = [synth.PlanSpec(16, 16, 64, 0.8, 0.5, 6), synth.PlanSpec(8, 8, 32, 0.8, 0.5, 4)]
    tr = np.zeros((2, 6), dtype=TRACE)
    # block 0: picks 0,0,5,0,5,7 -> distinct before each: 0,1,1,2,2,2 = 8 terms
    for it, (a, b) in enumerate([(0, 0), (0, 0), (0, 5), (0, 0), (0, 5), (1, 7)]):
        tr[0, it] = (a, b, 0, 0)
    # block 1 (4 iterations): picks (2,3) four times -> 0,1,1,1 = 3 terms
    for it in range(4):
        tr[1, it] = (2, 3, 0, 0)
    blocks = np.array([[0, 0, 0], [0, 0, 1]], dtype=np.int32)
    ops, terms = bench.alu_work(tr, blocks, specs)
    assert terms == 8 + 3
    bins64, bins32 = 64 * 64 // 2 + 2, 32 * 32 // 2 + 2
    assert ops == (6 * bins64 + 4 * bins32) * bench.OPS_PER_BIN_ITER + bench.OPS_PER_RECURRENCE_TERM * 11


def test_cpu_samples_are_seeded_subsets():
    wl = types.SimpleNamespace(blocks=np.arange(300, dtype=np.int32).reshape(100, 3))
    a = bench._sample(wl, 10)
    b = bench._sample(wl, 10)
    assert np.array_equal(a, b) and len(a) == 10
    rows = {tuple(r) for r in wl.blocks}
    assert all(tuple(r) in rows for r in a)
    assert len({tuple(r) for r in a}) == 10
    assert bench._sample(wl, None) is wl.blocks
    assert bench._sample(wl, 1000) is wl.blocks


def test_volume_cpu_legs_on_a_small_video():
    """The video workload's CPU legs: a seeded oracle sample (the same blocks
    every run) and the transform-domain form over all blocks, which takes the
    oracle's paths."""
    wl = synth.small_video(5, plan=synth.VolumePlanSpec(8, 4, 1, 16, 4, 0.8, 0.5, 20))
    pick, ora, dt = bench.volume_oracle_sample(wl, 6, threads=2)
    pick2, _, _ = bench.volume_oracle_sample(wl, 6, threads=2)
    assert np.array_equal(pick, pick2) and len(pick) == 6 and dt > 0
    assert (ora.status == 0).all()
    fd = bench.cpu_volume_transform_domain(wl, threads=2)
    assert fd["unit"] == "blocks/s" and fd["value"] > 0 and fd["cores"] == 2
    import oracle
    full = oracle.run_batch_volume(wl.video, wl.avail, wl.blocks, wl.plan, transform_domain=True)
    assert np.array_equal(full.path[pick], ora.path)
