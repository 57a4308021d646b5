"""Host-side arithmetic of bench.py (no GPU): the contact-value fit of the
pressure route, the shared-memory roofline's algorithmic bytes, the FP64 pipe
in warp-instructions, the latency ceiling and the all-cores batch CPU
baseline."""
import math
from types import SimpleNamespace

import numpy as np
import pytest

import bench
import ecmc_workloads as W


def test_contact_value_recovers_a_quadratic_exactly():
    r = 1.0 + 0.01 * (np.arange(10) + 0.5)
    g = 6.5 - 40.0 * (r - 1.0) + 300.0 * (r - 1.0) ** 2
    assert bench.contact_value(r, g) == pytest.approx(6.5, abs=1e-9)


def test_smem_roofline_counts_the_strip_that_can_hold_the_first_hit():
    w = SimpleNamespace(N=1048576, L=W.box_side(1048576, 0.72))
    c = SimpleNamespace(sum_disp=0.05 * 1000.0, events=900.0)
    per, disks, lam0 = bench.smem_bytes_per_event(w, c, 1000, 1)
    rho = w.N / w.L**2
    assert lam0 == pytest.approx(0.05)
    assert disks == pytest.approx(rho * 2.0 * (1.0 + 0.05))
    assert per == pytest.approx(disks * 8.0 + 16.0)
    assert bench.smem_bytes_per_event(w, c, 1000, 0)[0] == pytest.approx(disks * 16.0 + 16.0)
    # the roofline divides the algorithmic bytes of one launch by that
    # launch's average time (not by the step time)
    kt = SimpleNamespace(phase_ms=3.0, phase_launches=3)
    out = bench.chain_roofline(w, None, c, 1000, kt, 1, 40000.0, 1, True)
    assert out["events_per_launch"] == pytest.approx(300.0)
    assert out["launch_ms"] == pytest.approx(1.0)
    assert out["achieved"] == pytest.approx(per * 300.0 / 1e-3 / 1e9)
    assert out["frac"] == pytest.approx(out["achieved"] / 40000.0)
    assert out["bound"] == "smem" and out["unit"] == "GB/s"
    assert out["traffic"] == pytest.approx(bench.FUSED_DRAM_BYTES_CAPTURE * w.N
                                           / bench.FUSED_CAPTURE_N)
    assert bench.chain_roofline(w, None, c, 1000, kt, 1, 40000.0, 1, False)["traffic"] is None
    assert bench.chain_roofline(w, [1], c, 1000, kt, 1, 40000.0, 1, True) is None
    # the counters follow the frame mode the run used; frame mode 0 (falsy)
    # still selects its own capture, an uncaptured mode gives none
    out0 = bench.chain_roofline(w, None, c, 1000, kt, 1, 40000.0, 1, 0)
    assert out0["traffic"] == pytest.approx(bench.FUSED_CAPTURES[0]["dram_bytes"] * w.N
                                            / bench.FUSED_CAPTURE_N)
    assert bench.chain_roofline(w, None, c, 1000, kt, 1, 40000.0, 1, 2)["traffic"] is None


def test_fp64_pipe_counts_warp_instructions():
    kt = SimpleNamespace(phase_ms=2.0, phase_launches=2)
    iters = 2 * bench.FUSED_ITERATIONS_CAPTURE
    out = bench.fp64_pipe(iters, kt, 152, 2000.0, 1024.0, 1, True)
    winst = bench.FUSED_FP64_WINST_CAPTURE  # per launch: the captured count at these iterations
    cyc = 152 * 2000e6 / (1024e9 / 64.0)
    assert out["warp_instructions_per_launch"] == pytest.approx(winst)
    assert out["cycles_per_warp_instruction"] == pytest.approx(cyc)
    assert out["frac"] == pytest.approx(winst * cyc / (152 * 2000e6 * 1e-3))
    assert bench.fp64_pipe(iters, kt, 152, 2000.0, 1024.0, 1, False) is None
    out0 = bench.fp64_pipe(iters, kt, 152, 2000.0, 1024.0, 1, 0)
    assert out0["warp_instructions_per_launch"] == pytest.approx(bench.FUSED_CAPTURES[0]["fp64_winst"])


def test_latency_ceiling_arithmetic():
    class FakeHandle:
        def get_param(self, key):
            return 9120.0

    c = SimpleNamespace(events=2.4e6)
    kt = SimpleNamespace(phase_ms=2.6, phase_launches=2)
    out = bench.latency_ceiling(FakeHandle(), None, 240, c, kt, {"sm_mhz": 2000.0}, 2070.0)
    cyc = 1.3e-3 * 2000e6 * 9120 / 1.2e6
    assert out["cycles_per_event_per_chain"] == pytest.approx(cyc)
    assert out["ceiling_all_active_cells"] == pytest.approx(14400 * 2000e6 / cyc)


def test_batch_cpu_baseline_uses_all_cores():
    descs = []
    for r, d in enumerate(W.replica_batch(R=4)):
        descs.append(dict(N=min(d["N"], 4096), L=W.box_side(min(d["N"], 4096), d["eta"]),
                          cells_x=4, cells_y=4, ell=2.0, n_m=2, seed=d["seed"], replica=r))
    out = bench.cpu_baseline_batch(descs, 0.5)
    assert out["kind"] == "oracle" and out["value"] > 0
    assert 1 <= out["cores"] <= 4 and "processes" in out["sample"]
