"""Pose refinement as a torch.autograd.Function.

``PoseRefineLoss.apply(delta, ctx)`` returns the depth-band projection loss
of the frames reconstructed with poses ``T(t) T(c) R(w) T(-c) P`` (delta =
(t, w) per frame, about each frame centre c), and its backward gives
dL/d(delta) from the library's adjoint kernel.  The kernel differentiates a
left perturbation of the poses it is given, so the gradient is exact at
delta = 0 -- a refinement step applies its delta to the poses and starts
again from zero (``refine`` below).  All arithmetic runs in the library's
CUDA kernels; torch holds the tensors.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import usvol


@dataclass
class PoseProblem:
    """Frames, poses and target of one refinement (device tensors)."""
    vol: usvol.Volume          # trilinear, used as scratch by each evaluation
    images: torch.Tensor       # [n, H, W] uint8 or float32
    poses: torch.Tensor        # [n, 4, 4] float64
    cal: usvol.Calibration
    band: tuple
    target: torch.Tensor       # [ny, nx] float32
    eps: float = 1e-2

    def __post_init__(self):
        nx, ny, nz = self.vol.grid
        lo, hi = self.band
        dev = self.images.device
        self.proj = torch.empty((ny, nx), dtype=torch.float32, device=dev)
        self.adj = torch.empty((hi - lo, ny, nx, 2), dtype=torch.float32, device=dev)
        self.loss = torch.empty(1, dtype=torch.float64, device=dev)
        self.grad = torch.empty((self.images.shape[0], 6), dtype=torch.float64, device=dev)

    def evaluate(self, poses: torch.Tensor):
        """(loss, grad [n, 6]) at `poses` (delta = 0)."""
        n, H, W = self.images.shape
        dt = usvol.U8 if self.images.dtype == torch.uint8 else usvol.F32
        usvol.pose_loss_grad(self.vol.handle, self.images.data_ptr(), n, H, W, dt,
                             poses.contiguous().data_ptr(), self.cal, self.band[0], self.band[1],
                             self.eps, self.target.data_ptr(), self.proj.data_ptr(),
                             self.adj.data_ptr(), self.loss.data_ptr(), self.grad.data_ptr())
        return self.loss.clone(), self.grad.clone()

    def perturbed(self, delta: torch.Tensor) -> torch.Tensor:
        n, H, W = self.images.shape
        out = torch.empty_like(self.poses)
        usvol.apply_pose_delta(self.poses.data_ptr(), delta.contiguous().data_ptr(), n, H, W,
                               self.cal, out.data_ptr())
        return out


class PoseRefineLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, delta: torch.Tensor, prob: PoseProblem):
        poses = prob.perturbed(delta.detach().to(torch.float64))
        loss, grad = prob.evaluate(poses)
        ctx.save_for_backward(grad)
        return loss.to(delta.dtype).reshape(())

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad.to(g.dtype), None


def refine(prob: PoseProblem, steps: int = 200, step_t: float = 0.2, step_w: float = 0.003,
           decay: float = 0.985, backtrack: int = 6):
    """Descent on every frame's (t, w), re-linearised each step (the kernel's
    gradient is exact at delta = 0).  Each frame moves along its own
    gradient direction by a common length -- step_t mm for the
    translation, step_w rad for the rotation, shrinking by `decay` per
    step -- because the per-frame gradients differ by orders of magnitude
    (frames that cross the band's bright bone against frames that do not).
    The splat is only piecewise linear in the poses, so a step is halved up
    to `backtrack` times until the loss does not increase, else skipped.
    Returns the refined poses and the loss after each step."""
    poses = prob.poses.clone()
    loss, grad = prob.evaluate(poses)
    hist = [float(loss.item())]
    saved = prob.poses
    st, sw = step_t, step_w
    try:
        for _ in range(steps):
            gt, gw = grad[:, :3], grad[:, 3:]
            nt = gt.norm(dim=1, keepdim=True).clamp_min(1e-300)
            nw = gw.norm(dim=1, keepdim=True).clamp_min(1e-300)
            scale = 1.0
            for _ in range(backtrack + 1):
                delta = torch.cat([-scale * st * gt / nt, -scale * sw * gw / nw], 1)
                prob.poses = poses
                cand = prob.perturbed(delta)
                c_loss, c_grad = prob.evaluate(cand)
                if float(c_loss.item()) <= hist[-1]:
                    poses, grad = cand, c_grad
                    break
                scale *= 0.5
            else:
                hist.append(hist[-1])
                st *= decay
                sw *= decay
                continue
            hist.append(float(c_loss.item()))
            st *= decay
            sw *= decay
    finally:
        prob.poses = saved
    return poses, hist
