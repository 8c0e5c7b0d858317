"""The bench's block-parallel oracle baseline on the host cores (CPU only):
one spawned process per core, the field shared through shared memory."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_block_parallel_oracle_baseline():
    sys.path.insert(0, ROOT)
    import bench
    x = np.random.default_rng(0).standard_normal(1 << 18).astype(np.float32)
    msgs = [(np.random.default_rng(i).standard_normal(5000).astype(np.float32), 1e-3)
            for i in range(3)]
    r = bench.cpu_parallel(x, msgs, x.size)
    assert r["unit"] == "GB/s" and r["value"] > 0
    assert r["cores"] == (os.cpu_count() or 1)
    assert "%d segments" % r["cores"] in r["sample"]
