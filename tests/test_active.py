"""Active-mapping driver: the field grows incrementally with the chosen views
and equals a fresh construction over them; each step picks the argmax of the
scores of the density-controlled scene."""
import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


def test_active_mapping_loop():
    import __graft_entry__ as g
    g.build()
    import paper_2605_30342_gb300 as gv
    from paper_2605_30342_gb300.active import ActiveMapper
    c = sg.config(1, n=1500, n_train=2, train_wh=(96, 96))
    sc = c["scene"]
    ctx = gv.Context(0)
    gs = gv.Gaussians.from_numpy(sc)
    vm = torch.as_tensor(np.random.default_rng(3).uniform(-1.5, 1.5, (400, 3)).astype(np.float32)).cuda()
    am = ActiveMapper(ctx, gs, c["train"], degree=2, virtual_means=vm, rho=100.0)
    for step in range(3):
        cands = sg.fibonacci_cameras(8, 2.6 + 0.3 * step, 96, 96)
        rec = am.step(cands)
        s = rec["scores"].cpu().numpy()
        assert rec["best"] == int(np.argmax(s)) and rec["pose"] is cands[rec["best"]]
        assert am.vf.n_train_views == len(am.views) - 1
        assert rec["n_virtual_kept"] > 0
    assert len(am.views) == 5
    fresh = ctx.vf_build(gs, am.views[:4], degree=2)
    assert torch.allclose(fresh.coeffs, am.vf.coeffs, atol=1e-5)
    # the last step's scores equal a direct scoring of the same augmented scene
    dc = ctx.density_control(gs, vm, am.views[:4], rho=100.0)
    gs2, vf2 = am.ctx.augment(gs, am.vf, dc["kept_means"], dc["scale"])
    direct = ctx.score_views(gs2, vf2, sg.fibonacci_cameras(8, 2.6 + 0.3 * 2, 96, 96))
    assert torch.equal(direct["score"], am.history[-1]["scores"])
    ctx.close()
