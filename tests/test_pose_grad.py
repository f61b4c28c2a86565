"""Pose gradients of the depth-band projection loss (trilinear splat):
oracle pins on the CPU (finite differences of the oracle's own loss at a
small step, perturbation algebra); GPU adjoint kernel against the FP64
oracle gradient, the GPU loss, and the autograd wrapper."""
import numpy as np
import pytest

from oracle import pose


def _problem(n=4, **kw):
    from paper_2412_00058_gb300 import synth
    args = dict(n=n, H=48, W=40, grid=(64, 80, 64), spacing=0.3, band=(20, 45), sweep_mm=4.0)
    args.update(kw)
    w = synth.pose_refine(**args)
    _, _, T, _ = pose.forward(w, w.poses, w.band, 1e-2)
    return w, w.meta["noisy_poses"], T


def test_oracle_gradient_matches_finite_differences():
    w, noisy, T = _problem(n=3)
    L, g = pose.analytic_grad(w, noisy, w.band, 1e-2, T)
    fd = pose.fd_grad(w, noisy, w.band, 1e-2, T, 1e-6, frames=[0, 2])
    for f in (0, 2):
        assert np.max(np.abs(fd[f] - g[f])) <= 1e-5 * np.max(np.abs(g[f]))
    assert L > 0


def test_oracle_loss_is_zero_at_the_target_poses_and_gradient_vanishes():
    w, _, T = _problem(n=2)
    L, g = pose.analytic_grad(w, w.poses, w.band, 1e-2, T)
    assert L == 0.0 and np.all(g == 0.0)


def test_pose_delta_algebra():
    w, noisy, _ = _problem(n=2)
    z = pose.apply_pose_delta(noisy, np.zeros((2, 6)), w.calib, w.H, w.W, w.sx, w.sy)
    assert np.allclose(z, noisy, atol=0, rtol=0)
    d = np.zeros((2, 6))
    d[0, :3] = (1.0, -2.0, 0.5)
    t = pose.apply_pose_delta(noisy, d, w.calib, w.H, w.W, w.sx, w.sy)
    assert np.allclose(t[0, :3, 3] - noisy[0, :3, 3], d[0, :3], atol=1e-12)
    d = np.zeros((2, 6))
    d[1, 3:] = (0.01, -0.02, 0.03)
    r = pose.apply_pose_delta(noisy, d, w.calib, w.H, w.W, w.sx, w.sy)
    c0 = pose.frame_centre(noisy[1], w.calib, w.H, w.W, w.sx, w.sy)
    c1 = pose.frame_centre(r[1], w.calib, w.H, w.W, w.sx, w.sy)
    assert np.allclose(c0, c1, atol=1e-12)            # rotation about the frame centre


def _gpu_problem(w, poses, T):
    import torch
    from paper_2412_00058_gb300 import posegrad, usvol
    vol = usvol.Volume(w.grid, w.spacing, w.origin, "trilinear")
    return posegrad.PoseProblem(vol, torch.from_numpy(w.images).cuda(),
                                torch.from_numpy(np.ascontiguousarray(poses)).cuda(),
                                usvol.calibration_of(w), w.band,
                                torch.from_numpy(T.astype(np.float32)).cuda(), 1e-2)


@pytest.mark.gpu
def test_gpu_pose_gradient_matches_fp64_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from helpers import build_library
    build_library()
    w, noisy, T = _problem(n=6)
    prob = _gpu_problem(w, noisy, T)
    loss, grad = prob.evaluate(prob.poses)
    L, g = pose.analytic_grad(w, noisy, w.band, 1e-2, T.astype(np.float32).astype(np.float64))
    assert abs(float(loss.item()) - L) <= 1e-4 * L
    gg = grad.cpu().numpy()
    for f in range(w.n):
        assert np.max(np.abs(gg[f] - g[f])) <= 1e-4 * np.max(np.abs(g[f])), (f, gg[f], g[f])
    # the perturbation kernel against the oracle's
    rng = np.random.default_rng(0)
    d = rng.normal(0, [0.3, 0.3, 0.3, 0.01, 0.01, 0.01], size=(w.n, 6))
    out = prob.perturbed(torch.from_numpy(d).cuda()).cpu().numpy()
    ref = pose.apply_pose_delta(noisy, d, w.calib, w.H, w.W, w.sx, w.sy)
    assert np.allclose(out, ref, rtol=0, atol=1e-10)


@pytest.mark.gpu
def test_gpu_autograd_and_refinement_reduce_the_loss():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from helpers import build_library
    from paper_2412_00058_gb300 import posegrad
    build_library()
    w, noisy, T = _problem(n=6)
    prob = _gpu_problem(w, noisy, T)
    delta = torch.zeros((w.n, 6), dtype=torch.float64, device="cuda", requires_grad=True)
    loss = posegrad.PoseRefineLoss.apply(delta, prob)
    loss.backward()
    _, grad = prob.evaluate(prob.poses)
    assert torch.allclose(delta.grad, grad)
    _, hist = posegrad.refine(prob, steps=6, lr_t=2e-6, lr_w=2e-9)
    assert all(b <= a for a, b in zip(hist, hist[1:]))     # never accepts a worse loss
    assert hist[-1] <= hist[0]
