"""The learned warm start end to end on small chips (32x32x4, s = 8):
data from the library's block CG, training with the library's FNO kernels,
prediction, the residual-based fallback and warm-started solves.  The gain
(or loss) in iterations against the zero start is printed; what is asserted
is what the construction guarantees."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_warm_start_pipeline_on_small_chips(capsys):
    from paper_2510_23221_gb300 import fno, synth
    from paper_2510_23221_gb300 import warmstart as W
    dims = dict(nx=32, ny=32, n_layers=4, s=8)
    tr = [synth.FNO_TRAIN_SEED0 + i for i in range(24)]
    X, Y, t_scale, iters = W.build_dataset(tr, **dims)
    assert X.shape == (24 * 8, 4, 32, 32, W.C_IN) and Y.shape == (24 * 8, 4, 32, 32)
    chip0, _ = synth.warm_start_chip(tr[0], 32, 32, 4, 8)
    shape = W.shape_for(chip0, max_batch=8, layers=2, hidden=32, mx=8, my=8, mz=2)
    net = fno.Fno(shape, W.init_params(shape, 7))
    hist = W.train(net, X, Y, epochs=25, lr=3e-3)
    assert hist[-1] < 0.3 * hist[0], hist
    ws = W.WarmStart(net, t_scale)
    ev = W.evaluate(ws, [synth.FNO_HELDOUT_SEED0 + i for i in range(4)], threshold=1e-2, **dims)
    assert ev["all_converged"]
    for r in ev["rows"]:
        assert r["use_warm"] == (r["pred_relres_max"] <= 1e-2)
        assert r["pred_rel_error"] < 0.5          # the prediction is far closer than the zero start
    with capsys.disabled():
        print("\nwarm start, 32x32x4: zero %.1f, chosen %.1f, always-warm %.1f iterations; "
              "prediction error %.3f, residual %.2f (median)" %
              (ev["zero_iters_mean"], ev["chosen_iters_mean"], ev["always_warm_iters_mean"],
               ev["pred_rel_error_median"], ev["pred_relres_median"]))
