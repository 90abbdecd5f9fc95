import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


def read_golden(name: str) -> dict:
    """Parse a tests/golden fixture: '# section: NAME' headers split whitespace rows."""
    sections: dict[str, list[list[str]]] = {"rows": []}
    cur = "rows"
    with open(os.path.join(TESTS, "golden", name)) as f:
        for line in f:
            s = line.strip()
            if s.startswith("# section:"):
                cur = s.split(":", 1)[1].strip()
                sections[cur] = []
                continue
            s = s.split("#", 1)[0].strip()
            if s:
                sections[cur].append(s.split())
    return sections


@pytest.fixture(scope="session")
def tiny_graph():
    from invariants import csr_from_edges
    g = read_golden("tiny_graph.txt")
    edges = [(int(a), int(b)) for a, b, _ in g["edges"]]
    ws = [int(c) for _, _, c in g["edges"]]
    row_ptr, col, w = csr_from_edges(7, edges, ws)
    level = np.array([int(x) for x in g["level"][0]], np.int32)
    dist = np.array([int(x) for x in g["dist"][0]], np.uint64).astype(np.uint32)
    return row_ptr, col, w, level, dist
