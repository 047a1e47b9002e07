import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_golden(name):
    """Parse a tests/golden fixture: '# key: value' headers + 8 rows of x y z."""
    meta, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line:
                continue
            if line.startswith("#"):
                body = line[1:].strip()
                if ":" in body:
                    k, v = body.split(":", 1)
                    if k.strip() in ("kind", "truth", "cubic"):
                        meta[k.strip()] = v.strip()
                continue
            rows.append([float(x) for x in line.split()])
    assert len(rows) == 8 and all(len(r) == 3 for r in rows)
    q = np.array(rows, dtype=np.float64).reshape(24)
    meta["kind"] = 0 if meta["kind"] == "VF" else 1
    meta["truth"] = int(meta["truth"])
    return q, meta


@pytest.fixture
def golden():
    return load_golden
