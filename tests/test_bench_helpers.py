"""The benchmark's roofline bookkeeping (no GPU): DRAM traffic is reported only for the
kernel sources it was captured on, per launch in proportion to the moves, and the
tensor-core training kernel's FLOP count follows the products it issues."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_only_for_the_captured_sources(monkeypatch):
    h = bench.kernel_sources_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    monkeypatch.setitem(bench.KINETIC_TRAFFIC, "w", {"sources": h, "bytes_per_move": 2000.0})
    assert bench.kinetic_traffic("w", 1000) == 2000.0 * 1000
    assert bench.kinetic_traffic("w", 0) == 0.0
    monkeypatch.setitem(bench.KINETIC_TRAFFIC, "w", {"sources": "0" * 16 if h != "0" * 16 else "1" * 16,
                                                     "bytes_per_move": 2000.0})
    assert bench.kinetic_traffic("w", 1000) is None  # another kernel: no traffic
    assert bench.kinetic_traffic("no such workload", 1000) is None


def test_sources_hash_follows_every_kernel_file(tmp_path, monkeypatch):
    """The hash covers every .cu / .cuh of the library: a change in any of them (a
    header the kinetic kernel includes, or the host file that launches it) turns the
    recorded traffic off."""
    import shutil
    pkg = tmp_path / "paper_2308_06484_gb300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2308_06484_gb300", "csrc"), pkg,
                    ignore=shutil.ignore_patterns("*.o", "*.so"))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_hash()
    assert h0 == bench.kernel_sources_hash()
    for name in sorted(os.listdir(pkg)):
        if not name.endswith((".cu", ".cuh")):
            continue
        f = pkg / name
        text = f.read_bytes()
        f.write_bytes(text + b"\n")
        assert bench.kernel_sources_hash() != h0, name
        f.write_bytes(text)
    assert bench.kernel_sources_hash() == h0


def test_tensor_training_flops_per_tile():
    """Hand count of k_mlp_grad_tc's BF16 products per 128-row tile: five row products
    with three parts each (layer 1: N 64, K 32; layer 2: 64, 64; layer 3: 32, 64;
    dOut W3: 64, 32; dZ2 W2: 64, 64), G_a (128 x 112 over the 128 rows, three
    products) and G_b (128 x 32, two)."""
    m = 128
    rows = 3 * 2 * m * (64 * 32 + 64 * 64 + 32 * 64 + 64 * 32 + 64 * 64)
    grads = 3 * 2 * 128 * 112 * m + 2 * 2 * 128 * 32 * m
    assert bench._tc_grad_flops_per_tile() == rows + grads == 24117248
    # the network's own work per row stays the CUDA-core kernel's count
    assert bench.MLP_FLOPS_PER_ROW == 2 * 7424 * 3 + 2 * 18 * 64 + 2 * 64 * 64
