"""torch.autograd wrappers of the pair network (argument marshalling only).

NNEnergy(cfg, params) -> E per pair, differentiable in cfg and in params, with
a differentiable backward: the gradient with respect to cfg is itself an
autograd function whose backward returns the weight gradient of
sum_b v_b . dE_b/dcfg_b (the second-order product computed by
rb_nn_weight_vjp).  That is exactly what force matching needs: forces and
torques are (linear in) dE/dcfg, and their loss is differentiated in params.
The second derivative with respect to cfg itself is not provided.
"""
from __future__ import annotations

import torch

from . import api


class _Ctx:
    """Binds one MLP and one Trainer (workspace) to a parameter tensor."""

    def __init__(self, width: int, depth: int, max_batch: int):
        self.mlp = api.MLP(width, depth)
        self.trainer = api.Trainer(self.mlp, max_batch)
        self.escale_index = self.mlp.n_params - 2

    def load(self, params: torch.Tensor):
        self.mlp.set_params(params.detach().contiguous().float())


def _eval(ctx: _Ctx, cfg: torch.Tensor):
    out, g = ctx.mlp.pairs(cfg.detach().contiguous(), "fp32", grad=True)
    return out[:, 3].clone(), g


class _InputGrad(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cfg, params, ctx):
        ctx.load(params)
        _, g = _eval(ctx, cfg)
        fctx.save_for_backward(cfg, params)
        fctx.ctx = ctx
        return g

    @staticmethod
    def backward(fctx, gG):
        cfg, params = fctx.saved_tensors
        ctx = fctx.ctx
        ctx.load(params)
        es = params[ctx.escale_index].detach()
        zero = torch.zeros(cfg.shape[0], dtype=torch.float32, device=cfg.device)
        gW = ctx.trainer.weight_vjp(cfg.detach().contiguous(), (gG * es).contiguous().float(), zero)
        return None, gW, None


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cfg, params, ctx):
        ctx.load(params)
        E, _ = _eval(ctx, cfg)
        fctx.save_for_backward(cfg, params)
        fctx.ctx = ctx
        return E

    @staticmethod
    def backward(fctx, gE):
        cfg, params = fctx.saved_tensors
        ctx = fctx.ctx
        G = _InputGrad.apply(cfg, params, ctx)
        g_cfg = gE[:, None] * G
        ctx.load(params)
        es = params[ctx.escale_index].detach()
        u0 = torch.zeros((cfg.shape[0], 8), dtype=torch.float32, device=cfg.device)
        gW = ctx.trainer.weight_vjp(cfg.detach().contiguous(), u0, (gE * es).contiguous().float())
        return g_cfg, gW, None


class NNEnergy:
    """E = NNEnergy(width, depth, max_batch)(cfg, params): cfg (n, 8) CUDA
    float32 (s xyz, 0, q wxyz in the frame of body i), params the flat FP32
    parameter vector.  E[b] is the pair energy; autograd supplies dE/dcfg
    and dE/dparams, and dE/dcfg is differentiable in params."""

    def __init__(self, width: int, depth: int = 3, max_batch: int = 65536):
        self.ctx = _Ctx(width, depth, max_batch)

    def __call__(self, cfg: torch.Tensor, params: torch.Tensor) -> torch.Tensor:
        return _Energy.apply(cfg, params, self.ctx)
