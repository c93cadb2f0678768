"""Per-operator materialising GPU baseline (comparison only, not the product).

Restates the evaluation model the paper measures (TensorGP in TensorFlow eager
mode, Sec. 3.1 and 4.2): every node of every tree is one eager tensor
operation over the whole domain, each intermediate tensor is materialised in
device memory, protected operators are compositions of library calls
(Sec. 3.2), and there is no subtree caching.  Here the library is PyTorch
eager on the same GPU.  The fused evaluator is measured against this.
"""
from __future__ import annotations

import math

import torch

from . import inputs as I


class PerOpEvaluator:
    def __init__(self, grid: I.Grid, device="cuda"):
        f = torch.float32
        W, H = grid.W, grid.H
        sx = (torch.tensor(grid.xhi, dtype=f) - grid.xlo) / (W - 1) if W > 1 else torch.tensor(0.0)
        sy = (torch.tensor(grid.yhi, dtype=f) - grid.ylo) / (H - 1) if H > 1 else torch.tensor(0.0)
        cols = torch.arange(W, dtype=f, device=device)
        rows = torch.arange(H, dtype=f, device=device)
        xs = grid.xlo + cols * sx.to(device)
        ys = grid.ylo + rows * sy.to(device)
        self.X = xs.repeat(H)
        self.Y = ys.repeat_interleave(W)
        x4 = (self.X * self.X) * (self.X * self.X)
        y4 = (self.Y * self.Y) * (self.Y * self.Y)
        self.target = x4 / (1 + x4) + y4 / (1 + y4)
        self.device = device
        self.launches = 0

    def _eval(self, t):
        op, v, kids = t
        if op == I.X:
            return self.X
        if op == I.Y:
            return self.Y
        if op == I.CONST:
            self.launches += 1
            return torch.full_like(self.X, float(v))
        a = self._eval(kids[0])
        b = self._eval(kids[1]) if len(kids) > 1 else None
        if op == I.ADD:
            self.launches += 1
            return a + b
        if op == I.SUB:
            self.launches += 1
            return a - b
        if op == I.MUL:
            self.launches += 1
            return a * b
        if op == I.DIV:   # protected: 0 where the denominator is 0
            self.launches += 3
            return torch.where(b == 0, torch.zeros_like(a), a / b)
        if op == I.SIN:
            self.launches += 2
            return torch.sin(a * math.pi)
        if op == I.COS:
            self.launches += 2
            return torch.cos(a * math.pi)
        if op == I.NEG:
            self.launches += 1
            return -a
        if op == I.ABS:
            self.launches += 1
            return torch.abs(a)
        if op == I.MIN:
            self.launches += 1
            return torch.fmin(a, b)
        if op == I.MAX:
            self.launches += 1
            return torch.fmax(a, b)
        raise ValueError(op)

    def fitness(self, trees):
        """RMSE of each tree against the Pagie target; returns a device tensor."""
        out = []
        for t in trees:
            f = self._eval(t)
            d = f - self.target
            out.append(torch.sqrt(torch.mean(d * d)))
            self.launches += 4
        return torch.stack(out)
