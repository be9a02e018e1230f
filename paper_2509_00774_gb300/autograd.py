"""Differentiable A_B, A_B^H and prox step, and SPGM unrolled with learnable steps.

The forward of each op is a call into the CUDA library; its backward is the
hand-written adjoint kernel (for A_B), the forward kernel (for A_B^H) or the
prox-step backward kernel.  Complex gradients follow PyTorch's convention for
a real loss L: grad = dL/dRe + j dL/dIm.  For a linear map y = A s this makes
the vector-Jacobian product grad_s = A^H grad_y.

UnrolledSPGM runs a fixed number of SPGM iterations (Sec. IV, Eq. 5 with the
minibatch gradient of Eq. 6),

    s_{i+1} = prox_{eta_i lambda_i}( s_i - (eta_i / B_i) A_{B_i}^H (A_{B_i} s_i - y_{B_i}) ),

with a learnable step eta_i and weight lambda_i per iteration, and checkpoints
each iteration's input so the backward pass recomputes the operator instead of
storing residuals and gradients.
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint as _checkpoint


class _ForwardFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, op, pairs):
        ctx.op = op
        ctx.pairs = pairs
        return op.forward(pairs, s.contiguous())

    @staticmethod
    def backward(ctx, gy):
        return ctx.op.adjoint(ctx.pairs, gy.contiguous()), None, None


class _ResidualFn(torch.autograd.Function):
    """r = A_B s - y_B in one fused launch (the residual of Eq. 4 / Eq. 6); y is data (no gradient)."""

    @staticmethod
    def forward(ctx, s, op, pairs, y):
        ctx.op = op
        ctx.pairs = pairs
        return op.residual(pairs, s.contiguous(), y)

    @staticmethod
    def backward(ctx, gr):
        return ctx.op.adjoint(ctx.pairs, gr.contiguous()), None, None, None


class _AdjointFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, r, op, pairs):
        ctx.op = op
        ctx.pairs = pairs
        return op.adjoint(pairs, r.contiguous())

    @staticmethod
    def backward(ctx, gg):
        return ctx.op.forward(ctx.pairs, gg.contiguous()), None, None


class _ProxStepFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, g, step, alpha, shrink, op):
        s = s.contiguous()
        g = g.contiguous()
        st, al, sh = float(step), float(alpha), float(shrink)
        out = torch.empty_like(s)
        op.prox_step(s, g, st, al, out, sh)
        ctx.save_for_backward(s, g)
        ctx.op, ctx.st, ctx.al, ctx.sh = op, st, al, sh
        ref = step if torch.is_tensor(step) else alpha
        ctx.scalar_meta = (ref.dtype, ref.device) if torch.is_tensor(ref) else (torch.float64, torch.device("cpu"))
        return out

    @staticmethod
    def backward(ctx, go):
        s, g = ctx.saved_tensors
        need_s, need_g, need_step, need_alpha, need_shrink = ctx.needs_input_grad[:5]
        grad_s = torch.empty_like(s) if need_s else None
        grad_g = torch.empty_like(g) if need_g else None
        scalars = torch.empty(3, dtype=torch.float64, device=s.device)
        ctx.op.prox_step_backward(s, g, ctx.st, ctx.al, go.contiguous(), grad_s, grad_g, scalars, ctx.sh)
        dt, dev = ctx.scalar_meta
        sc = scalars.to(device=dev, dtype=dt)
        return (grad_s, grad_g, (sc[0] if need_step else None), (sc[1] if need_alpha else None),
                (sc[2] if need_shrink else None), None)


class _ProxGroupStepFn(torch.autograd.Function):
    """shrink G_{alpha_g}(prox_alpha(s - step g)) over the grid's 2 x 2 x 1 voxel blocks."""

    @staticmethod
    def forward(ctx, s, g, step, alpha, alpha_g, shrink, op):
        s = s.contiguous()
        g = g.contiguous()
        st, al, ag, sh = float(step), float(alpha), float(alpha_g), float(shrink)
        out = torch.empty_like(s)
        op.prox_group_step(s, g, st, al, ag, out, sh)
        ctx.save_for_backward(s, g)
        ctx.op, ctx.st, ctx.al, ctx.ag, ctx.sh = op, st, al, ag, sh
        ref = next((x for x in (step, alpha, alpha_g, shrink) if torch.is_tensor(x)), None)
        ctx.scalar_meta = (ref.dtype, ref.device) if ref is not None else (torch.float64, torch.device("cpu"))
        return out

    @staticmethod
    def backward(ctx, go):
        s, g = ctx.saved_tensors
        need = ctx.needs_input_grad[:6]
        grad_s = torch.empty_like(s) if need[0] else None
        grad_g = torch.empty_like(g) if need[1] else None
        scalars = torch.empty(4, dtype=torch.float64, device=s.device)
        ctx.op.prox_group_step_backward(s, g, ctx.st, ctx.al, ctx.ag, go.contiguous(), grad_s, grad_g, scalars, ctx.sh)
        dt, dev = ctx.scalar_meta
        sc = scalars.to(device=dev, dtype=dt)
        return (grad_s, grad_g, (sc[0] if need[2] else None), (sc[1] if need[3] else None),
                (sc[2] if need[4] else None), (sc[3] if need[5] else None), None)


def forward_op(op, pairs, s):
    """y = A_B s, differentiable in s (op: nfmimo.Context, pairs: int32 device tensor)."""
    return _ForwardFn.apply(s, op, pairs)


def residual_op(op, pairs, s, y):
    """r = A_B s - y_B with y the full measurement vector [P*K] (fused into the forward kernel),
    differentiable in s."""
    return _ResidualFn.apply(s, op, pairs, y)


def adjoint_op(op, pairs, r):
    """g = A_B^H r, differentiable in r."""
    return _AdjointFn.apply(r, op, pairs)


def prox_step(op, s, g, step, alpha, shrink=1.0, alpha_g=None):
    """shrink * prox_alpha(s - step g), differentiable in s, g, step, alpha and shrink (0-dim tensors or floats);
    shrink = 1/(1 + eta lambda w2) gives the prox of the elastic net w1 ||s||_1 + (w2/2) ||s||^2 with
    alpha = eta lambda w1.  With alpha_g (= eta lambda w3) the block shrink of the group term
    w3 sum_b ||s_b||_2 over the grid's 2 x 2 x 1 voxel blocks follows the soft threshold (the prox of the
    sparse-group penalty), differentiable in alpha_g as well."""
    if alpha_g is None:
        return _ProxStepFn.apply(s, g, step, alpha, shrink, op)
    return _ProxGroupStepFn.apply(s, g, step, alpha, alpha_g, shrink, op)


class UnrolledSPGM(torch.nn.Module):
    """n_iter SPGM iterations with learnable per-iteration eta_i and lambda_i (FP64 CPU parameters)."""

    def __init__(self, op, n_iter: int, eta: float, lam: float, checkpoint: bool = True, w1: float = 1.0,
                 w2: float = 0.0, w3: float = 0.0):
        """w1, w2, w3: regulariser w1 ||s||_1 + (w2/2) ||s||^2 + w3 sum_b ||s_b||_2 over the grid's 2 x 2 x 1
        voxel blocks (w2 = w3 = 0: the paper's l1)."""
        super().__init__()
        self.op = op
        self.n_iter = int(n_iter)
        self.eta = torch.nn.Parameter(torch.full((self.n_iter,), float(eta), dtype=torch.float64))
        self.lam = torch.nn.Parameter(torch.full((self.n_iter,), float(lam), dtype=torch.float64))
        self.checkpoint = checkpoint
        self.w1, self.w2, self.w3 = float(w1), float(w2), float(w3)

    def _iteration(self, s, y, pairs, eta, lam):
        B = pairs.numel() * self.op.K
        r = residual_op(self.op, pairs, s, y)       # A_B s - y_B fused in the forward kernel
        g = adjoint_op(self.op, pairs, r)
        shrink = 1.0 / (1.0 + eta * lam * self.w2) if self.w2 != 0.0 else 1.0
        alpha_g = eta * lam * self.w3 if self.w3 != 0.0 else None
        return prox_step(self.op, s, g, eta / B, eta * lam * self.w1, shrink, alpha_g)

    def forward(self, y, batches, s0=None):
        """y: [M] or [n_scenes, M] complex64 device; batches: n_iter int32 pair lists.
        Returns the final iterate(s), [N] or [n_scenes, N]."""
        single = y.dim() == 1
        ys = y.unsqueeze(0) if single else y
        outs = []
        for j in range(ys.shape[0]):
            yj = ys[j].contiguous()
            if s0 is None:
                s = torch.zeros(self.op.N, dtype=torch.complex64, device=y.device)
            else:
                s = (s0 if single else s0[j]).contiguous()
            for i in range(self.n_iter):
                pairs = batches[i % len(batches)]
                if self.checkpoint and torch.is_grad_enabled():
                    s = _checkpoint(self._iteration, s, yj, pairs, self.eta[i], self.lam[i], use_reentrant=False)
                else:
                    s = self._iteration(s, yj, pairs, self.eta[i], self.lam[i])
            outs.append(s)
        return outs[0] if single else torch.stack(outs)
