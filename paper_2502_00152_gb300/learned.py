"""Learned initial guess for CG: a gauge-covariant parallel-transport network.

Each layer is out_b = sum_a sum_h w[b,a,h] T_h in_a with T_h the identity and the
eight one-hop fat-link transports of the Dirac operator (hisq_net_layer); the
forward, adjoint and weight-gradient passes and the Adam step are the library's
CUDA kernels, wrapped here in a torch.autograd.Function.  The network is linear:
the map it approximates, eta -> M^-1 eta, is linear, so nonlinear activations
would only cost accuracy.  Channels 3 -> 16 -> 16 -> 16 -> 3: three right-hand
sides (colour-vector fields) in, three guesses out.

The guess enters the solve through hisq_solve_params.guess: CG starts from it
(its residual deflated when deflation is on) and still runs to the same FP64
true residual, so the plain solve remains both the fallback and the arbiter.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hisq as H

CHANNELS = (3, 16, 16, 16, 3)


class PTLayer(torch.autograd.Function):
    """One parallel-transport layer: forward, adjoint and weight gradient are
    hand-written kernels (hisq_net_layer, hisq_net_wgrad)."""

    @staticmethod
    def forward(fctx, x, w, hctx, bf16):
        x = x.contiguous()
        out = torch.empty((w.shape[0],) + tuple(x.shape[1:]), dtype=torch.complex64, device=x.device)
        H.hisq_net_layer(hctx, w.detach().contiguous(), x, out, w_bf16=bf16, adjoint=False)
        fctx.save_for_backward(x, w)
        fctx.hctx = hctx
        fctx.bf16 = bf16
        return out

    @staticmethod
    def backward(fctx, gout):
        x, w = fctx.saved_tensors
        gout = gout.contiguous()
        gin = torch.empty_like(x)
        H.hisq_net_layer(fctx.hctx, w.detach().contiguous(), gout, gin, w_bf16=fctx.bf16, adjoint=True)
        gw = torch.empty_like(w)
        H.hisq_net_wgrad(fctx.hctx, x, gout, gw)
        return gin, gw, None, None


class GuessNet:
    """The network's weights (complex64, FP32 master copies) and its training."""

    def __init__(self, hctx, channels=CHANNELS, seed: int = 0, bf16: bool = True, device="cuda"):
        self.hctx = hctx
        self.bf16 = bf16
        gen = torch.Generator().manual_seed(seed)
        self.weights = []
        for cin, cout in zip(channels[:-1], channels[1:]):
            scale = 1.0 / np.sqrt(9 * cin)
            w = (torch.randn(cout, cin, 9, 2, generator=gen) * scale).to(device)
            self.weights.append(torch.view_as_complex(w.contiguous()).requires_grad_(True))
        self.m1 = [torch.zeros_like(torch.view_as_real(w.detach())) for w in self.weights]
        self.m2 = [torch.zeros_like(m) for m in self.m1]
        self.step = 0

    def __call__(self, x):
        for w in self.weights:
            x = PTLayer.apply(x, w, self.hctx, self.bf16)
        return x

    def train_step(self, x, target, mask, lr: float = 1e-3) -> float:
        """One Adam step on the relative squared error over the masked sites."""
        out = self(x)
        diff = (out - target) * mask
        loss = (diff.abs() ** 2).sum() / ((target * mask).abs() ** 2).sum()
        for w in self.weights:
            w.grad = None
        loss.backward()
        self.step += 1
        with torch.no_grad():
            for w, m1, m2 in zip(self.weights, self.m1, self.m2):
                wr = torch.view_as_real(w)
                gr = torch.view_as_real(w.grad).contiguous()
                H.hisq_net_adam(self.hctx, wr, gr, m1, m2, lr, self.step)
        return float(loss.detach())

    def state(self):
        return [w.detach().cpu().numpy() for w in self.weights]
