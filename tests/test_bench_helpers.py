"""Host-side measurement helpers of bench.py (no GPU).

The DRAM traffic that a bench line reports as roofline.traffic comes from
profiles/rk4_step_traffic.json only while the step kernel's sources are the
ones the ncu capture was taken from; the FP32 error per result is a relative
L2 norm against the FP64 result."""
import json
import os
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

RECORD = os.path.join(ROOT, "profiles", "rk4_step_traffic.json")


def test_traffic_record_is_tied_to_the_kernel_sources(monkeypatch):
    rec = json.load(open(RECORD))
    key = "reservoir_2048_fp32"
    entry = rec[key]["tiles"]["7"]
    monkeypatch.setattr(bench, "kernel_hash", lambda: rec[key]["kernel_sources"])
    assert bench.recorded_traffic("reservoir_2048", 32, 7) == entry["dram_bytes_per_launch"]
    # a tile configuration without a record, or other kernel sources: no figure
    assert bench.recorded_traffic("reservoir_2048", 32, 99) is None
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("reservoir_2048", 32, 7) is None
    assert bench.recorded_traffic("no_such_workload", 32, 7) is None


def test_traffic_records_are_well_formed():
    """Every record: read + write = the per-launch figure, a positive duration,
    and the one-pass ncu command on bench.py that produced it, with the GPU's
    clocks left alone."""
    rec = json.load(open(RECORD))
    n = 0
    for key, e in rec.items():
        if key == "note":
            continue
        assert len(e["kernel_sources"]) == 16
        for tile, t in e["tiles"].items():
            n += 1
            assert t["dram_bytes_per_launch"] == pytest.approx(t["dram_read"] + t["dram_write"])
            assert t["duration_s"] > 0
            cmd = t["command"]
            assert cmd.startswith("ncu ") and "--clock-control none" in cmd
            assert "python bench.py " in cmd and "--tile %s" % tile in cmd
            assert "-c 1" in cmd
    assert n >= 3


def test_kernel_hash_covers_the_step_kernel_sources():
    csrc = os.path.join(ROOT, "paper_2411_18341_gb300", "csrc")
    for f in bench.STEP_KERNEL_SOURCES:
        assert os.path.isfile(os.path.join(csrc, f)), f
    h = bench.kernel_hash()
    assert len(h) == 16 and h == bench.kernel_hash()


def test_precision_error_is_relative_l2():
    rng = np.random.default_rng(3)
    psi64 = torch.tensor(rng.normal(size=(1, 8, 9)) + 1j * rng.normal(size=(1, 8, 9)))
    n64 = torch.tensor(rng.uniform(1, 2, size=(1, 8, 9)))
    d = torch.tensor(1e-3 * (rng.normal(size=(1, 8, 9)) + 1j * rng.normal(size=(1, 8, 9))))
    psi32 = (psi64 + d).to(torch.complex64)
    n32 = (n64 * (1 + 1e-4)).to(torch.float32)
    out = bench.precision_error(psi32, n32, psi64, n64, "test")
    want = np.linalg.norm(psi32.numpy().astype(np.complex128) - psi64.numpy()) / \
        np.linalg.norm(psi64.numpy())
    assert out["psi_rel_l2"] == pytest.approx(want, rel=1e-12)
    want_n = np.linalg.norm(n32.numpy().astype(np.float64) - n64.numpy()) / np.linalg.norm(n64.numpy())
    assert out["n_rel_l2"] == pytest.approx(want_n, rel=1e-12)
    assert "n_rel_l2" not in bench.precision_error(psi32, None, psi64, None, "test")
