"""torch.autograd wrappers over the FMM deflection and its adjoint.

``deflect(stars, masses, kappa_s, gamma, rays, ...)`` returns y (m, 2); its
backward runs ``lens_deflect_adjoint`` (the transposed FMM on the same tree)
and returns gradients for the stars (n, 2), masses (n,), kappa_s and gamma
(0-dim tensors).  ``light_curve(y, ...)`` is the Gaussian-source light curve
(a ray sum) with ``lens_light_curve_grad`` as its backward.  Both are thin:
every step runs in liblens.so.
"""
from __future__ import annotations

import torch

from . import lens


# Above this many stars the backward pass rebuilds the tree and expansions
# instead of keeping the forward plan alive between forward and backward
# (between them only the inputs are held).
RECOMPUTE_MIN_STARS = 10_000_000


class LensDeflect(torch.autograd.Function):
    @staticmethod
    def forward(ctx, stars, masses, kappa_s, gamma, rays, p, leaf_size, prec, target_box,
                recompute):
        st = stars.detach().contiguous()
        ms = masses.detach().contiguous()
        args = (float(kappa_s), float(gamma))
        kw = dict(p=p, leaf_size=leaf_size, prec=prec, target_box=target_box)
        plan = lens.LensFMM(st, ms, *args, **kw)
        rays_c = rays.detach().contiguous()
        y = plan.deflect(rays_c)
        if recompute is None:
            recompute = st.shape[0] >= RECOMPUTE_MIN_STARS
        if recompute:
            plan.close()
            plan = None
            ctx.save_for_backward(rays_c, st, ms)
        else:
            ctx.save_for_backward(rays_c)
        ctx.plan = plan
        ctx.rebuild = (args, kw)
        ctx.ks_is_tensor = isinstance(kappa_s, torch.Tensor)
        ctx.g_is_tensor = isinstance(gamma, torch.Tensor)
        return y

    @staticmethod
    def backward(ctx, grad_y):
        saved = ctx.saved_tensors
        rays = saved[0]
        plan = ctx.plan
        if plan is None:
            args, kw = ctx.rebuild
            plan = lens.LensFMM(saved[1], saved[2], *args, **kw)
        gxy, gm, gkg = plan.adjoint(rays, grad_y.contiguous())
        plan.close()
        ctx.plan = None
        gks = gkg[0] if ctx.ks_is_tensor else None
        gg = gkg[1] if ctx.g_is_tensor else None
        return gxy, gm, gks, gg, None, None, None, None, None, None


def deflect(stars, masses, kappa_s, gamma, rays, p=24, leaf_size=16, prec=lens.FP64,
            target_box=None, recompute=None):
    """Differentiable y(rays) = lens equation with FMM deflections.  With
    ``recompute`` (default: N* >= 1e7) the tree and expansions are rebuilt in
    the backward pass instead of being held since the forward pass."""
    return LensDeflect.apply(stars, masses, kappa_s, gamma, rays, p, leaf_size, prec, target_box,
                             recompute)


class LightCurve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, w_ray, samples, sigma, trunc):
        y_c = y.detach().contiguous()
        F = lens.light_curve(y_c, w_ray, samples, sigma, trunc)
        ctx.save_for_backward(y_c, samples, F)
        ctx.args = (w_ray, sigma, trunc)
        return F

    @staticmethod
    def backward(ctx, gF):
        # dL/dy for a general upstream gradient gF: the kernel computes
        # sum_k 2 (F_k - T_k) dF_k/dy; with T = F - gF/2 that is sum_k gF_k dF_k/dy.
        y, samples, F = ctx.saved_tensors
        w_ray, sigma, trunc = ctx.args
        T = F - 0.5 * gF
        gy = lens.light_curve_grad(y, w_ray, samples, sigma, F, T, trunc)
        return gy.reshape(y.shape), None, None, None, None


def light_curve(y, w_ray, samples, sigma, trunc=6.0):
    return LightCurve.apply(y, w_ray, samples, sigma, trunc)
