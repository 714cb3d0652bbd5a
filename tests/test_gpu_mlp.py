"""The learned dz controller: GPU training kernels against the FP64 CPU
oracle's MLP, and the controller end to end (data from step-doubling runs,
training on the GPU, proposals judged by step doubling)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05988_gb300 import workloads as W
from tests.conftest import rel_l2

pytestmark = pytest.mark.gpu
NIN, NH = 6, 64


@pytest.fixture(scope="module")
def fcn():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1507_05988_gb300 import build
    build.build()
    from paper_1507_05988_gb300 import fcn as m
    return m


def _bf16(p):
    """Round to bfloat16 (the precision the kernels use the weights in)."""
    return torch.tensor(np.asarray(p, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def test_mlp_gradient_matches_the_oracle(fcn):
    rng = np.random.default_rng(2)
    npar = oracle.mlp_param_count(NIN, NH)
    assert npar == fcn.FCN_MLP_NPARAM
    params = (0.3 * rng.standard_normal(npar)).astype(np.float32)
    x = rng.standard_normal((300, NIN)).astype(np.float32)
    y = rng.standard_normal(300).astype(np.float32)
    loss, g = fcn.mlp_loss_grad(params, x, y)
    lref, gref = oracle.mlp_loss_grad(_bf16(params), x.astype(np.float64), y.astype(np.float64),
                                      NIN, NH)
    assert loss == pytest.approx(lref, rel=1e-5)
    assert rel_l2(g, gref) < 1e-5


def test_mlp_training_fits_a_smooth_function(fcn):
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (2048, NIN)).astype(np.float32)
    y = (np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] - x[:, 4] / 3).astype(np.float32)
    wl = W.small(8, 16)
    s = fcn.Solver(wl.physics(), precision=fcn.FCN_FP32_MIXED)
    l0 = s.mlp_train(x, y, epochs=0, seed=1)
    l1 = s.mlp_train(x, y, epochs=60, batch=128, lr=3e-3, seed=1)
    s.close()
    assert l1 < 0.05 * l0 and l1 < 5e-3


def training_set(rec, margin=0.95):
    """Features and labels from logged attempts.  The safe step of the state
    an attempt started from is h (rtol/err)^(1/3) (Strang: O(dz^3) local
    error); the controller proposes exp(f4 - f5/3 + y) L_ref (the law applied
    to the previous accepted attempt) so the label of y is log(safe step) -
    (f4 - f5/3), with a margin, limited to the [0.2, 2] range of the law."""
    from paper_1507_05988_gb300.learned_dz import net_inputs
    safe = rec[:, 7] - rec[:, 8] / 3.0
    base = rec[:, 4] - rec[:, 5] / 3.0
    y = np.clip(safe - base + np.log(margin), np.log(0.2), np.log(2.0))
    return net_inputs(rec[:, :7]).astype(np.float32), y


def _adaptive(fcn, wl, prec, z_end, dz0, rtol, controller, params=None, log=0):
    s = fcn.Solver(wl.physics(), precision=prec)
    if params is not None:
        s.mlp_set(params)
    if log:
        s.mlp_log(log)
    s.set_field(wl.field())
    st = s.propagate(z_end, dz0, rtol=rtol, controller=controller)
    A = s.get_field()
    rec = s.mlp_log_records() if log else None
    s.close()
    return A, st, rec


def test_learned_dz_controller_end_to_end(fcn):
    """The learned controller on the filamentation pulse family (w0 = 2 mm,
    50 fs, 5 P_cr, n2 + n4, 1 % noise) on a 256 x 1024 grid: training data
    from step-doubling runs at noise seeds 1-6, the network (a correction to
    the step-doubling law) trained on the GPU, its margin chosen on seed 7;
    on seed 0 both controllers land on z_end within the tolerance of a
    fine-step FP64 reference, and the learned one needs fewer substeps than
    plain step doubling."""
    from paper_1507_05988_gb300 import learned_dz as LD
    rtol, z_end, dz0 = 1e-4, 0.3, 2e-3

    def pulse(seed):
        return W.config2(seed=seed).with_(nr=256, nt=1024, name=f"fil_256x1024_s{seed}")

    recs = [_adaptive(fcn, pulse(seed), fcn.FCN_FP32_MIXED, z_end, dz0, rtol, 0, log=20000)[2]
            for seed in range(1, 7)]
    x, y = LD.labels(np.concatenate(recs))
    assert len(y) > 200 and np.all(np.isfinite(x)) and np.all(np.isfinite(y))
    params, loss = LD.train(x, y, epochs=200, lr=2e-3)
    assert loss < 0.5 * np.var(y)

    def substeps(m):
        return _adaptive(fcn, pulse(7), fcn.FCN_FP32_MIXED, z_end, dz0, rtol, 1,
                         params=LD.with_margin(params, m))[1]["substeps"]
    margin = min((0.0, 0.05, 0.1, 0.15), key=substeps)
    wl = pulse(0)
    A0, st0, _ = _adaptive(fcn, wl, fcn.FCN_FP32_MIXED, z_end, dz0, rtol, 0)
    A1, st1, _ = _adaptive(fcn, wl, fcn.FCN_FP32_MIXED, z_end, dz0, rtol, 1,
                           params=LD.with_margin(params, margin))
    s = fcn.Solver(wl.physics(), precision=fcn.FCN_FP64)
    s.set_field(wl.field())
    s.step(z_end / 3000, 3000)
    ref = s.get_field()
    s.close()
    for A, st in ((A0, st0), (A1, st1)):
        assert st["z"] == z_end
        assert rel_l2(A, ref) < 30 * rtol
    assert st1["mlp_proposals"] > 0
    gain = 1.0 - st1["substeps"] / st0["substeps"]
    print(f"\nplain step doubling: accepted {st0['accepted']} rejected {st0['rejected']} "
          f"substeps {st0['substeps']}; learned dz (margin {margin}): accepted {st1['accepted']} "
          f"rejected {st1['rejected']} substeps {st1['substeps']} (mlp proposals {st1['mlp_proposals']}); "
          f"substeps saved {100 * gain:.1f} %")
    # the network must gain on the held-out seed: fewer Strang substeps
    # (accepted and rejected attempts, 3 substeps each) at the same rtol
    assert st1["substeps"] < st0["substeps"]
