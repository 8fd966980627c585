"""Learned low-rank DtN correction with a residual gate (not in the paper).

For boxes of one order p, side h and wavenumber kappa, an MLP predicts from
the sampled coefficient b the factors of T - T0 ~ s U V^T, where T0 is the
DtN map for b = 1.  Serving forms T_hat = T0 + s U V^T, checks each box with
the probe-residual gate and recomputes the rejected boxes with the exact
batched leaf reduction.  Training data are exact DtN maps from the same
library.  Every numerical step runs in the library's kernels; this module
only sequences C-ABI calls (torch supplies device memory and box gathers).
"""
from __future__ import annotations

import numpy as np

from . import (HPS_FP32_IR, LeafKind, hps_dtn_gate, hps_leaf_build_dtn, hps_leaf_sizes, hps_lowrank_dtn,
               hps_mlp_adam_step, hps_mlp_create, hps_mlp_destroy, hps_mlp_forward, hps_mlp_grad,
               hps_mlp_grad_target, hps_mlp_target)


class LearnedDtN:
    def __init__(self, ctx, p: int, h, kappa: float, hidden=(512, 512), rank: int = 32, seed: int = 0,
                 device: int = 0, prec: int = HPS_FP32_IR):
        import torch
        self.ctx, self.p, self.rank, self.prec = ctx, p, rank, prec
        self.h = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,)).copy()
        self.kappa = float(kappa)
        self.kind = LeafKind(p, self.h, kappa)
        self.n, self.m = hps_leaf_sizes(p)
        self.dev = torch.device("cuda", device)
        self.net = hps_mlp_create(device, p ** 3, hidden[0], hidden[1], self.m, rank, seed)
        ones = torch.ones(1, p ** 3, dtype=torch.float64, device=self.dev)
        self.T0 = self.exact(ones)[0].contiguous()
        self.scale = 1.0

    def close(self):
        if self.net:
            hps_mlp_destroy(self.net)
            self.net = None

    # ---------------------------------------------------------------- exact path

    def exact(self, b):
        """Exact DtN maps T [nbox][m][m] of boxes b [nbox][p^3] (device)."""
        import torch
        nbox = b.shape[0]
        T = torch.empty(nbox, self.m, self.m, dtype=torch.float64, device=self.dev)
        st = torch.zeros(nbox, dtype=torch.int32, device=self.dev)
        hps_leaf_build_dtn(self.ctx, self.kind, nbox, b.contiguous(), T, None, self.prec, st)
        return T

    def targets(self, b, chunk: int = 2048):
        """Exact DtN maps of every box (device), computed in chunks."""
        import torch
        out = torch.empty(b.shape[0], self.m, self.m, dtype=torch.float64, device=self.dev)
        for i in range(0, b.shape[0], chunk):
            out[i:i + chunk] = self.exact(b[i:i + chunk])
        return out

    # ---------------------------------------------------------------- training

    def fit(self, b, T, epochs: int = 20, batch: int = 128, lr: float = 1e-3, seed: int = 0, log=None):
        """Adam on mean (U V^T - (T - T0)/s)^2; s is fixed from the data at the
        start (root-mean-square of T - T0, measured by the loss kernel on a
        first batch while U V^T is still near zero).  The FP32 targets
        (T - T0)/s are formed once for the whole set."""
        import torch
        N = b.shape[0]
        first = min(N, batch)
        self.scale = 1.0
        l0 = hps_mlp_grad(self.net, first, b[:first].contiguous(), T[:first].contiguous(), self.T0, 1.0)
        self.scale = float(np.sqrt(max(l0, 1e-300)))
        D = torch.empty(T.shape, dtype=torch.float32, device=self.dev)
        hps_mlp_target(N, self.m, T.contiguous(), self.T0, self.scale, D)
        rng = np.random.default_rng(seed)
        steps = max(1, epochs * ((N + batch - 1) // batch))
        losses, step = [], 0
        for ep in range(epochs):
            order = torch.from_numpy(rng.permutation(N)).to(self.dev)
            for i in range(0, N, batch):
                idx = order[i:i + batch]
                bb = b.index_select(0, idx).contiguous()
                dd = D.index_select(0, idx).contiguous()
                want = (i == 0)
                loss = hps_mlp_grad_target(self.net, idx.numel(), bb, dd, want_loss=want)
                cur = lr * 0.5 * (1.0 + np.cos(np.pi * step / steps))
                hps_mlp_adam_step(self.net, cur)
                step += 1
                if want:
                    losses.append(loss)
                    if log:
                        log(ep, loss)
        return losses

    # ---------------------------------------------------------------- serving

    def predict(self, b):
        """T_hat = T0 + s U V^T for boxes b (device)."""
        import torch
        nbox = b.shape[0]
        U = torch.empty(nbox, self.m, self.rank, dtype=torch.float64, device=self.dev)
        V = torch.empty_like(U)
        hps_mlp_forward(self.net, nbox, b.contiguous(), U, V)
        T = torch.empty(nbox, self.m, self.m, dtype=torch.float64, device=self.dev)
        hps_lowrank_dtn(nbox, self.m, self.rank, self.T0, self.scale, U, V, T)
        return T

    def gate(self, b, T_hat, tol: float, nprobe: int = 4, seed: int = 12345, iters: int = 16):
        """(accept [nbox] int32, err [nbox] float64) on the device."""
        import torch
        nbox = b.shape[0]
        acc = torch.zeros(nbox, dtype=torch.int32, device=self.dev)
        err = torch.zeros(nbox, dtype=torch.float64, device=self.dev)
        hps_dtn_gate(self.ctx, self.kind, nbox, b.contiguous(), T_hat.contiguous(), nprobe, seed, iters, tol, acc,
                     err)
        return acc, err

    def serve(self, b, tol: float, **gate_kw):
        """DtN maps for boxes b: the prediction where the gate accepts it, the
        exact reduction elsewhere.  Returns (T, accept, err)."""
        T = self.predict(b)
        acc, err = self.gate(b, T, tol, **gate_kw)
        rej = (acc == 0).nonzero().flatten()
        if rej.numel():
            T.index_copy_(0, rej, self.exact(b.index_select(0, rej)))
        return T, acc, err
