"""Host logic of bench.py: the K bench steps always cover exactly one whole load path, and
both arms name the same workload."""
import argparse

import bench


def test_bench_steps_cover_one_whole_path():
    for K in (1, 3, 7, 20, 100):
        b = bench.chunks(K)
        assert b[0] == 0 and b[-1] == bench.STEPS_PER_PATH and len(b) == K + 1
        assert all(b[i] < b[i + 1] for i in range(K))
    assert bench.chunks(20) == list(range(0, 101, 5))
    assert bench.chunks(0) == [0, 100] and bench.chunks(500)[-1] == 100


def test_both_arms_name_the_same_workload():
    a = argparse.Namespace(grid=512, max_stag=20000, scheme="S1")
    name = bench.workload_name(a, bench.workload(512).l)
    assert name.startswith("tensile notched square 512x512 Q1, l=0.0075 mm")
    assert "whole load paths" in name
