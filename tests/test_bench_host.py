"""Host-side pieces of bench.py (no GPU): its synthetic paper network and FP64 reference
agree with the test suite's, the input layout holds one [x, x] window per prediction,
and the CPU-baseline extrapolation counts the operations the paper states."""
import os
import sys

import numpy as np

from tests import netref

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_paper_network_and_reference_match_the_tests():
    n = 768
    layers, pw = bench.paper_layers_for(n)
    w, W1, W2, W2s = netref.paper_net_weights(n)
    assert np.array_equal(pw[0], w) and np.array_equal(pw[1], W1) and np.array_equal(pw[2], W2)
    assert [ly[0] for ly in layers] == ["conv1d", "dense", "replicate", "poly3", "avgpool", "dense"]
    assert np.array_equal(layers[5][1], W2s)
    assert bench.RELU_APPROX == netref.relu_coeffs()
    x = np.random.default_rng(3).uniform(-1, 1, n)
    assert np.max(np.abs(bench.paper_fp64(pw, x) - netref.paper_net_fp64(x, w, W1, W2, netref.relu_coeffs()))) < 1e-12


def test_input_windows_layout():
    N, t0 = 8192, 1024
    xs, slots = bench.inputs_for(N, [768], 3, t0, windows=2)
    assert xs.shape == (3, 2, 768) and slots.shape == (3, N // 2)
    for b in range(3):
        for j in range(2):
            base = 2 * t0 * j
            assert np.array_equal(slots[b, base:base + 768], xs[b, j])
            assert np.array_equal(slots[b, base + t0:base + t0 + 768], xs[b, j])
            assert not slots[b, base + 768:base + t0].any()


def test_operation_plan_follows_the_papers_counts():
    # dense t x t by Eq. (bsgs): t1 + t2 - 2 rotations and t products; conv f = 9: 8
    # rotations and 9 products; avgpool 3: 2 rotations; the paper's depth 6
    plan = bench.op_plan(bench.WORKLOADS["paper_p1"])
    rots = sum(p[0] for p in plan)
    assert rots == 8 + 62 + 1 + 2 + 2 + 62  # conv, dense, replicate, ReLU (2 relins), pool, dense
    assert [p[3] for p in plan] == [7, 6, 5, 5, 4, 3, 2]
    # the batched network in the rectangular form: 1024->256 (t1 = t2 = 16, fold of 2 rotations
    # plus the [y, y] one), x^2, 256->256 (30 + replicate), x^2, 256->64 (t1 = t2 = 8, fold 2)
    plan = bench.op_plan(dict(bench.WORKLOADS["batched"], dense_form="rect"))
    assert sum(p[0] for p in plan) == (30 + 3) + 1 + (30 + 1) + 1 + (14 + 2)
    assert sum(p[1] for p in plan) == 256 + 1.5 + 256 + 1.5 + 64
    # the lazy-ModDown split: t1 = 32, t2 = 8 for t = 256; t1 = 16, t2 = 4 for t = 64
    plan = bench.op_plan(bench.WORKLOADS["batched"])
    assert bench.WORKLOADS["batched"]["dense_form"] == "rect_lazy"
    assert sum(p[0] for p in plan) == (38 + 3) + 1 + (38 + 1) + 1 + (18 + 2)
    sq = dict(bench.WORKLOADS["batched"], dense_form="square")
    plan = bench.op_plan(sq)
    assert sum(p[0] for p in plan) == 62 + 1 + 1 + 30 + 1 + 1 + 30
    assert sum(p[1] for p in plan) == 1024 + 1.5 + 256 + 1.5 + 256


def test_cpu_baseline_runs_a_whole_oracle_forward_on_small_rings():
    wl = dict(bench.WORKLOADS["single4096"])
    wl.update(N=256, dims=[16, 8])  # the same network shape (dense, then x^2), small enough for a unit test
    smp = bench.OracleSample(wl)
    secs = smp.step()
    assert secs > 0 and smp.fraction == 1.0 and smp.err < 1e-4


def test_cpu_baseline_sample_is_a_fraction_of_the_forward():
    # larger rings: a step is one rotation, one product and one rescale, a known share of a
    # forward; the forward is at least as long as one rotation per key switch at the lowest level
    wl = dict(bench.WORKLOADS["batched"])
    wl.update(N=1024)
    smp = bench.OracleSample(wl, whole=False)
    secs = smp.step()
    t_rot, t_pt, t_rs = smp.parts
    fwd = smp.forward_seconds(t_rot, t_pt, t_rs)
    n_ks = sum(p[0] for p in bench.op_plan(wl))
    assert 0 < smp.fraction < 1 and abs(smp.fraction - secs / fwd) < 1e-12
    assert fwd > n_ks * t_rot * (2 * 6) / (4 * 10) * 0.99  # lowest level of the plan: 4 primes, 2 digits, 6 limbs


def test_both_arms_print_the_same_config():
    wl = bench.WORKLOADS["batched"]
    assert bench.shared_config(wl, 1) == bench.shared_config(wl, 1)
    assert set(bench.shared_config(wl, 2, cuda_graph=True)) >= {"workload", "batch_per_gpu", "N", "parallelism"}
