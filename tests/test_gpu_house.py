"""Parity and precision at the full size of the house workload (3M Gaussians
in eight rooms, opacity sigmoid(N(0, 2)), 20% tiny floaters at log-scale
N(-6, 0.5); 300 training views at 1280x720; 1024 candidates at 320x240;
bf16 field, f32 colour, f32 compositing; tile 8 for scoring and 16 for the
field), in the launch configuration bench.py times.  The comparisons are
those of test_gpu_fullsize.py: oracle fields only, parity against the oracle
on the same rounded inputs, and the storage error per output against the
float32-input float64 oracle on 8 sampled views, gated by the stated bound."""
import numpy as np
import pytest
import torch

import oracle
from _util import TOL, visibility_check
from test_gpu_fullsize import PRECISION_GATES, _build, _candidate_checks, _field_checks, _report, _spread

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def house():
    gv, c = _build(4)
    sc = c["scene"]
    ctx = gv.Context(0)
    gs = gv.Gaussians.from_numpy(sc)
    ti = _spread(len(c["train"]), 8)
    g_o, _, _, rad = oracle.vf_build([c["train"][i] for i in ti], sc, 3, want_rad=True)
    yield dict(gv=gv, ctx=ctx, c=c, gs=gs, p=gv.Params(vf_degree=3, tile=8), p_vf=gv.Params(vf_degree=3, tile=16),
               ti=ti, g_o=g_o, rad=rad, dtype=torch.bfloat16, sh_dtype=torch.float32,
               name="house 3M (20% floaters), bf16 field, f32 colour")
    ctx.close()


# --------------------------------------------------------------------------- house workload

def test_house_training_view_visibility(house):
    """Floaters (20% of 3M Gaussians at log-scale N(-6, 0.5)) stress the
    footprint culls: the sampled view's visibility against the oracle."""
    ctx, c, gs = house["ctx"], house["c"], house["gs"]
    p = house["ti"][3]
    sumT, cnt = ctx.debug_visibility(gs, [c["train"][p]], params=house["p_vf"])
    _, rc, _, _, b = oracle.visibility_view(c["train"][p], c["scene"], want_bounds=True)
    bad, err, moved = visibility_check(sumT[0].cpu().numpy(), cnt[0].cpu().numpy(), b)
    assert bad == 0 and err <= TOL, (bad, err, moved)
    assert (rc > 0).sum() > 10000


def test_house_field_on_sampled_views(house):
    st = _field_checks(house)
    _report(house["name"], {"gamma_over_P": st})
    assert st["max_abs"] <= PRECISION_GATES["bf16"]["gamma_over_P"], st


def test_house_sampled_candidate_views(house):
    views = _spread(1024, 8)
    out, res = _candidate_checks(house, views)
    _report(house["name"], res)
    for k, st in res.items():
        assert st["max_abs"] <= PRECISION_GATES["bf16"][k], (k, st)
    s = out["score"].cpu().numpy()
    assert out["best"] == int(np.argmax(s)) and len(s) == 1024
