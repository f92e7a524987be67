"""What the trained network gains over the method without it (Sec. 5.1's estimator
against the sensitivity curves alone).

The pairs are measured on the GPU: every configuration-3 victim beside every tuned
co-runner configuration, with both sides' solo features.  The method without the
network predicts a pair's slowdown as 1 + S_v,r(x), the victim's measured sensitivity
curve for the co-runner's resource read at the co-runner's solo intensity.  The
network (trained by the library's own kernels on the training pairs) must beat it by
a wide margin on held-out pairs, both when the held-out pairs are a random fifth and
when they belong to co-runner configurations never seen in training."""
import pytest

import paper_2501_16909_b300 as ifr
from paper_2501_16909_b300 import train_predictor as TP
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def measured():
    need_gpu()
    ctx = ifr.Context(0)
    d = TP.collect(ctx, repeats=1, log=lambda *x: None)
    yield ctx, d
    ctx.close()


@pytest.mark.parametrize("split", ["random", "unseen"])
def test_network_beats_sensitivity_curves_on_held_out_pairs(measured, split):
    ctx, d = measured
    assert len(d["y"]) >= 10000
    ev = TP.evaluate(ctx, d, split, max_epochs=200)
    assert ev["test_pairs"] >= 1000 and ev["train_pairs"] >= 5000, ev
    # the network's error is a fraction of the curves' and small in absolute terms
    assert ev["mlp_mape"] <= 0.5 * ev["baseline_mape"], ev
    assert ev["mlp_mape"] <= 0.25, ev
