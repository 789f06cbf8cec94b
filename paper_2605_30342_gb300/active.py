"""Active-mapping driver around the library (Alg. "Active Mapping with GAVIS").

Per planning step: the visibility field is extended with the views taken
since the last step (eq:vis_gamma is a sum over views, so only new views are
rasterized), visibility-field density control runs on all views taken so
far, candidate poses are scored on the augmented scene, the argmax is taken
(eq:i_gain) and the chosen pose joins the training set.  3DGS training and
the simulator are outside this library: the Gaussian scene stays fixed and
"taking an image" only records the pose.  Every computation runs in the CUDA
library through its binding; this module only sequences the calls.
"""
from __future__ import annotations

import torch

from . import Context, Gaussians, Params, VisibilityField


class ActiveMapper:
    def __init__(self, ctx: Context, gs: Gaussians, initial_views, degree: int = 2, dtype=torch.float32,
                 virtual_means: torch.Tensor | None = None, rho: float = 100.0, eta: float = 0.5,
                 eps_v: float = 0.95, params: Params | None = None):
        """virtual_means: caller-drawn uniform centres of the virtual particles
        (device [n, 3]) for density control, or None to skip it."""
        self.ctx, self.gs, self.degree = ctx, gs, int(degree)
        self.params = params or Params(vf_degree=self.degree)
        self.views = list(initial_views)
        self.vf = VisibilityField(torch.zeros((gs.n, (self.degree + 1) ** 2), dtype=dtype, device=gs.means.device),
                                  self.degree, 0, float(self.params.kappa))
        self._built = 0
        self.virtual_means, self.rho, self.eta, self.eps_v = virtual_means, rho, eta, eps_v
        self.history = []

    def _extend_field(self):
        new = self.views[self._built:]
        if new:
            self.ctx.vf_build(self.gs, new, degree=self.degree, params=self.params, out=self.vf,
                              accumulate=self._built > 0)
            self._built = len(self.views)

    def step(self, candidates):
        """One planning step over `candidates` (camera objects of one
        resolution); returns dict(best, pose, scores, n_virtual_kept)."""
        self._extend_field()
        gs, vf, kept = self.gs, self.vf, 0
        if self.virtual_means is not None and len(self.virtual_means):
            dc = self.ctx.density_control(self.gs, self.virtual_means, self.views, rho=self.rho, eta=self.eta,
                                          eps_v=self.eps_v, params=self.params)
            kept = dc["n_keep"]
            gs, vf = self.ctx.augment(self.gs, self.vf, dc["kept_means"], dc["scale"])
        out = self.ctx.score_views(gs, vf, candidates, params=self.params, want_rgb=False)
        best = int(out["best"])
        self.views.append(candidates[best])                   # the pose whose image is taken next
        rec = dict(best=best, pose=candidates[best], scores=out["score"].detach().clone(), n_virtual_kept=kept)
        self.history.append(rec)
        return rec
