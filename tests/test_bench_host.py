"""Host-side checks of bench.py: the batched workload's recipe (seeded, 64
instances inside the configured ranges) and the source hash that ties the
recorded DRAM traffic to the slab kernel's sources."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as wl  # noqa: E402


def test_batched_workload_is_seeded_and_in_range():
    a, b = bench.batch_workloads(), bench.batch_workloads()
    assert len(a) == bench.BATCH == 64
    assert [(w.n1, w.n2, w.n3, w.r, w.observed, w.seed) for w in a] == \
        [(w.n1, w.n2, w.n3, w.r, w.observed, w.seed) for w in b]
    for w in a:
        assert 64 <= w.n1 <= 1024 and 96 <= w.n2 <= 288 and 28 <= w.n3 <= 168 and 4 <= w.r <= 32
        assert 0.1 <= w.observed <= 0.6
        assert w.period == w.n2          # one day per mode-2 length
    assert len({w.seed for w in a}) == 64
    # the mix covers small and large ranks and both tube-length parities
    rs = np.array([w.r for w in a])
    assert (rs > 16).any() and (rs <= 16).any()
    assert len({w.n3 % 2 for w in a}) == 2


def test_source_hash_covers_the_slab_kernel_sources():
    h = bench.src_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    csrc = os.path.join(ROOT, "paper_2005_09838_gb300", "csrc")
    for f in bench.SLAB_SOURCES:
        assert os.path.exists(os.path.join(csrc, f)), f


def test_roofline_bytes_follow_the_per_iteration_model():
    # the bench's algorithmic bytes for the 144 x 288 x 168 FP32 workload:
    # B_iter = s N + N/8 + 3 (2 s n1 n2 S) = 113.3 MB per iteration, of which
    # the fused transform / W-step / residual kernel carries G, the mask bits
    # and one write of the residual spectrum (56.94 MB)
    import bench
    w = wl.c2(0.2)
    assert abs(bench.iteration_bytes(w) - 113.3e6) < 0.05e6
    alg = bench.algorithmic_bytes(w)
    assert abs(alg["slab"] - 56.94e6) < 0.01e6
    # the slab kernel's design bytes add the read of the stored Z~ spectrum
    assert bench.design_bytes(w)["slab"] - alg["slab"] > 28e6
