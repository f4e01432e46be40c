"""The bench's byte accounting on CPU: per-launch method and intermediate
bytes of the roofline regions for each triangle path the build reports
(vr_build_stats.tri_order), and the whole build's method bytes."""
import numpy as np

import bench
import synth


class _Cloud:
    def __init__(self, n, d):
        self.n = n
        self.points = np.zeros((n, d), np.float32)


def test_final_write_bytes_by_triangle_path():
    c = _Cloud(4000, 32)
    E, T = 399_899, 19_760_896
    lex = bench.roofline_bytes(c, E, T, 0, E + 1, tri_order=1)
    counted = bench.roofline_bytes(c, E, T, 0, E + 1, tri_order=2)
    claimed = bench.roofline_bytes(c, E, T, 0, E + 1, tri_order=3)
    for r in (lex, counted, claimed):
        assert r["tri_final"][0] == 36 * T          # outputs: verts 12, grade 4, rowidx 12, colptr 8
    assert lex["tri_final"][1] == 8 * T             # 64-bit lex keys
    assert counted["tri_final"][1] == 4 * T         # 32-bit max-edge keys: E <= 2^20 beside a 12-bit vertex
    assert claimed["tri_final"][1] == 2 * T         # 16-bit third vertices
    assert claimed["tri_gen"] == (0, 2 * T + 8 * E)  # plus each edge's count and run start


def test_counted_keys_widen_when_edges_do_not_fit():
    c = _Cloud(6200, 32)                            # 13-bit vertex: 19 bits left for the edge index
    E = (1 << 19) + 1
    assert bench.roofline_bytes(c, E, 10, tri_order=2)["tri_final"][1] == 80


def test_build_method_bytes():
    c = synth.config1()
    counts = [64, 2016, 41664]
    b = bench.method_bytes_per_step(c, counts)
    assert b == c.points.nbytes + 76 * 2016 + 36 * 41664
