"""Host-side sizing rules of the build, checked on CPU.

The build sizes the lexicographic triangle-key buffer of small complexes
before it knows the triangle count, from the bound on the number of triangles
of a graph with E edges, T <= (sqrt 2 / 3) E^(3/2) (a consequence of the
Kruskal-Katona theorem; complete graphs approach it), and the max-edge key
buffer from the wedge bound T <= sum_v C(deg v, 2) / 3.  These tests check the
capacity formulas the build uses against exact triangle counts."""
import math

import numpy as np
import pytest


def capacity(E):
    """The build's buffer capacity for E kept edges."""
    return math.ceil(math.sqrt(2.0) / 3.0 * E ** 1.5) + 1


def triangles(adj):
    a = adj.astype(np.int64)
    return int(np.trace(a @ a @ a)) // 6


@pytest.mark.parametrize("n", [3, 4, 5, 10, 40, 120])
def test_complete_graphs(n):
    adj = np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64)
    E = n * (n - 1) // 2
    T = n * (n - 1) * (n - 2) // 6
    assert triangles(adj) == T
    assert T <= capacity(E)
    # the bound is tight up to lower-order terms
    assert T >= 0.7 * (math.sqrt(2.0) / 3.0) * E ** 1.5 or n < 10


@pytest.mark.parametrize("seed", range(6))
def test_random_and_clustered_graphs(seed):
    g = np.random.default_rng(seed)
    n = int(g.integers(20, 200))
    p = float(g.uniform(0.05, 0.9))
    m = g.random((n, n)) < p
    adj = np.triu(m, 1)
    # a dense block (clique) inside makes the count lopsided
    k = int(g.integers(3, n // 2))
    adj[:k, :k] = True
    adj = np.triu(adj, 1)
    adj = (adj | adj.T).astype(np.int64)
    E = int(adj.sum()) // 2
    assert triangles(adj) <= capacity(E)


def wedge_capacity(adj):
    """The max-edge key buffer's capacity: every triangle holds three of the
    sum_v C(deg v, 2) wedges (pairs of edges at a vertex), so
    T <= sum_v C(deg v, 2) / 3; the build takes that plus one."""
    deg = adj.sum(1)
    return int((deg * (deg - 1) // 2).sum()) // 3 + 1


@pytest.mark.parametrize("seed", range(8))
def test_wedge_bound(seed):
    g = np.random.default_rng(100 + seed)
    n = int(g.integers(5, 160))
    pts = g.normal(size=(n, 3))
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    r2 = float(np.quantile(d2, g.uniform(0.05, 1.0)))
    adj = ((d2 <= r2) & ~np.eye(n, dtype=bool)).astype(np.int64)
    assert triangles(adj) <= wedge_capacity(adj)


@pytest.mark.parametrize("n", [3, 4, 7, 30])
def test_wedge_bound_tight_on_complete_graphs(n):
    """Complete graphs meet it: C(n, 3) = n C(n - 1, 2) / 3."""
    adj = np.ones((n, n), dtype=np.int64) - np.eye(n, dtype=np.int64)
    assert wedge_capacity(adj) == n * (n - 1) * (n - 2) // 6 + 1


def test_small_cases():
    assert capacity(0) == 1
    assert capacity(1) >= 1
    assert capacity(3) >= 1  # one triangle


def test_cloud_descriptor_bytes():
    """The batch bench counts the per-cloud descriptor the batch path copies
    each way; its byte count must match the struct in the CUDA source (fields
    of 4 and 8 bytes only, so no padding beyond a trailing pair)."""
    import os
    import re
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "paper_1809_04424_b300", "csrc", "batch.cu")).read()
    body = src[src.index("struct CloudDesc {"):]
    body = body[: body.index("};")]
    size = {"int64_t": 8, "uint64_t": 8, "double": 8, "int32_t": 4, "float": 4}
    total = 0
    for line in body.splitlines()[1:]:
        line = line.split("//")[0].strip()
        if not line:
            continue
        m = re.match(r"(\w+)\s+(.*);", line)
        total += size[m.group(1)] * len(m.group(2).split(","))
    assert total % 8 == 0
    sys.path.insert(0, root)
    import bench
    assert bench.CLOUD_DESC_BYTES == total
