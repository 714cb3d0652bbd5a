"""Host logic of bench.py's measurement legs without a GPU: the Cartesian
leg and the checkpointed accuracy leg run against a stand-in solver (plain
numpy state, fixed event times), so the JSON they produce can be checked
for its keys and arithmetic."""
import types

import numpy as np
import pytest
import torch

import bench
from paper_1507_05988_gb300 import workloads as W


class _Event:
    def __init__(self, **kw):
        pass

    def record(self):
        pass

    def elapsed_time(self, other):
        return 10.0                      # ms


class _Solver:
    """Stand-in with the SolverXY/Solver surface bench.py uses."""

    def __init__(self, grid, phys, precision=0):
        self.p = precision
        self.a = None

    def set_field(self, a):
        self.a = np.array(a)

    def step(self, dz, n, graph=True):
        # FP32 drifts by 1e-7 per step, FP64 stays
        self.a = self.a * (1 + (1e-7 if self.p else 0.0)) ** n

    def get_field(self):
        return self.a

    def get_field_device(self, t):
        t.copy_(torch.from_numpy(np.asarray(self.a, np.complex128)))
        return t

    def set_field_device(self, t):
        self.a = t.numpy().copy()

    def diag(self):
        return {"energy": float(np.sum(np.abs(self.a) ** 2))}

    def variants(self):
        return (1, 6)

    def profile(self, on):
        pass

    def profile_read(self, reset=True):
        return {"row_head": (0.07, 1), "row_mid": (19.9, 199), "row_tail": (0.11, 1),
                "line_x": (17.2, 200), "line_y": (17.3, 200)}

    def close(self):
        pass


@pytest.fixture
def fake_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    monkeypatch.setattr(bench, "PERTURB_DEVICE", "cpu")


def test_cartesian_leg_reports_throughput_kernels_roofline_accuracy(fake_cuda):
    wl = W.small_xy(15, 13, 16).with_(nsteps=200)
    fcn = types.SimpleNamespace(FCN_FP32_MIXED=1, FCN_FP64=0, SolverXY=_Solver)
    Wm = types.SimpleNamespace(cartesian_config1=lambda: wl)
    out = bench.cartesian_leg(fcn, Wm, None, 1, accuracy=True, cpu=False)
    # 200 steps in 10 ms
    assert out["fp32"]["value"] == pytest.approx(wl.points * 200 / 10e-3)
    assert out["fp32"]["ms_per_step"] == pytest.approx(0.05)
    assert out["gpu_launches"] == 601
    k = out["kernels"]["line_x"]
    assert k["avg_us"] == pytest.approx(86.0)
    assert k["alg_GBps"] == pytest.approx(200 * 2 * wl.points * 8 / 17.2e-3 / 1e9)
    r = out["roofline"]
    assert r["kernel"] == "row_mid" and r["bound"] == "hbm"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    acc = out["accuracy_vs_fp64"]
    assert [c["steps"] for c in acc["checkpoints"]] == [25, 50, 100, 150, 200]
    # the stand-in's FP32 drift after 200 steps
    assert acc["field_rel_l2"] == pytest.approx((1 + 1e-7) ** 200 - 1, rel=1e-6)
    # the reference is perturbed by 6e-8 xi after every step: a random walk
    # of ~6e-8 / sqrt(3) per step
    c0, c4 = acc["checkpoints"][0], acc["checkpoints"][4]
    assert 1e-8 < c0["fp64_perturbed_field_rel_l2"] < 6e-8 * 25 ** 0.5
    assert c4["fp64_perturbed_field_rel_l2"] > c0["fp64_perturbed_field_rel_l2"]
    assert c4["fp32_over_reference"] == pytest.approx(
        c4["fp32_field_rel_l2"] / c4["fp64_perturbed_field_rel_l2"])


def test_weak_scaling_counts_every_rank():
    assert bench.weak_scaling_value(4, 1000, 10, 2.0) == pytest.approx(4 * 1000 * 10 / 2e-3)
