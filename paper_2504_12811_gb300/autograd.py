"""torch.autograd.Function over the C-ABI: forward = aaag_render_frame,
backward = aaag_render_backward (K6 + K7).  Argument marshalling only."""
from __future__ import annotations

import torch

from . import aaag


def _scene_struct(means, log_scales, quats, opacity_logits, sh, vhat_train, sh_degree):
    return aaag.aaag_scene(means.shape[0], sh_degree, 0, means.data_ptr(), log_scales.data_ptr(),
                           quats.data_ptr(), opacity_logits.data_ptr(), sh.data_ptr(), vhat_train.data_ptr())


class RenderFunction(torch.autograd.Function):
    """rgb [3,H,W], alpha [H,W] = render(scene tensors, camera).

    The workspace `ws` holds the frame between forward and backward: use one
    workspace per view that is rendered before the backward pass."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, vhat_train, cam, ws, params):
        tensors = [t.contiguous() for t in (means, log_scales, quats, opacity_logits, sh, vhat_train)]
        for t in tensors:
            if t.dtype != torch.float32 or not t.is_cuda:
                raise TypeError("scene tensors must be float32 CUDA tensors")
        sh_degree = int(round(tensors[4].shape[1] ** 0.5)) - 1
        scene = _scene_struct(*tensors, sh_degree)
        dev = means.device
        rgb = torch.empty(3, cam.height, cam.width, dtype=torch.float32, device=dev)
        alpha = torch.empty(cam.height, cam.width, dtype=torch.float32, device=dev)
        aaag.aaag_render_frame(scene, aaag.make_camera(cam), params if params is not None else aaag.make_params(),
                               ws.handle, rgb.data_ptr(), alpha.data_ptr(), aaag.current_stream())
        ctx.save_for_backward(*tensors, rgb)
        ctx.ws = ws
        ctx.sh_degree = sh_degree
        return rgb, alpha

    @staticmethod
    def backward(ctx, drgb, dalpha):
        means, log_scales, quats, opacity_logits, sh, vhat_train, rgb = ctx.saved_tensors
        scene = _scene_struct(means, log_scales, quats, opacity_logits, sh, vhat_train, ctx.sh_degree)
        out = [torch.empty_like(t) for t in (means, log_scales, quats, opacity_logits, sh)]
        grads = aaag.aaag_grads(*[t.data_ptr() for t in out])
        drgb = drgb.contiguous() if drgb is not None else torch.zeros_like(rgb)
        dalpha = dalpha.contiguous() if dalpha is not None else None
        dalpha_ptr = dalpha.data_ptr() if dalpha is not None else None
        aaag.aaag_render_backward(scene, ctx.ws.handle, rgb.data_ptr(), drgb.data_ptr(), dalpha_ptr, grads,
                                  aaag.current_stream())
        return (*out, None, None, None, None)


def render(means, log_scales, quats, opacity_logits, sh, vhat_train, cam, ws, params=None):
    return RenderFunction.apply(means, log_scales, quats, opacity_logits, sh, vhat_train, cam, ws, params)
