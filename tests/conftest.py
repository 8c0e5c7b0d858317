import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    """Parse a golden stream fixture: '# key: value' metadata, 'hex:' lines and a
    'decoded:' line of the reconstructed values."""
    meta, hexs, decoded = {}, [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line.startswith("# input:"):
                for kv in line[len("# input:"):].split():
                    k, v = kv.split("=", 1)
                    meta[k] = v
            elif line.startswith("hex:"):
                hexs.append(line[4:].replace(" ", ""))
            elif line.startswith("decoded:"):
                decoded = [float(t) for t in line[len("decoded:"):].split()]
    return meta, bytes.fromhex("".join(hexs)), decoded
