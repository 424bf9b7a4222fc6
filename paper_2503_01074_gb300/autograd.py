"""torch.autograd.Function around sonar_render / sonar_render_backward.

theta = (alpha, gain, mu[0..n_mat)) is a device tensor; the forward returns
the normalised polar image N.  The backward turns the scatter-add of the
forward into a gather over the per-ray hit records (saved, or recomputed by
re-casting the rays when `save_hits` is False, bitwise the same records).
"""
from __future__ import annotations

import torch

from .sonar import RenderParams, Sonar


class SonarRenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, sonar: Sonar, scene_id: int, spec, params: RenderParams, seed: int,
                frame: int, save_hits: bool):
        out = sonar.render(scene_id, spec, theta.detach().contiguous(), params, seed, frame,
                           hits=save_hits, fan=False)
        ctx.sonar, ctx.scene_id, ctx.spec, ctx.params = sonar, scene_id, spec, params
        ctx.seed, ctx.frame = seed, frame
        hits = out.get("hits")
        ctx.save_for_backward(theta, out["noised"], *( [hits] if hits is not None else [] ))
        ctx.has_hits = hits is not None
        return out["polar"]

    @staticmethod
    def backward(ctx, grad_polar):
        saved = ctx.saved_tensors
        theta, noised = saved[0], saved[1]
        hits = saved[2] if ctx.has_hits else None
        d = ctx.sonar.backward(ctx.scene_id, ctx.spec, theta.detach().contiguous(), ctx.params, ctx.seed,
                               ctx.frame, grad_polar.contiguous(), noised, hits)
        return d, None, None, None, None, None, None, None


def sonar_render(theta, sonar: Sonar, scene_id: int, spec, params: RenderParams = RenderParams(),
                 seed: int = 0, frame: int = 0, save_hits: bool = True):
    """Differentiable sonar render: returns N (normalised polar image)."""
    return SonarRenderFn.apply(theta, sonar, scene_id, spec, params, seed, frame, save_hits)
