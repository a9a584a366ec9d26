"""Learned support-4 gridding kernel (pattern 4): training loop, fields,
checkpoints.

The network (3 -> H GELU -> H GELU -> 16 outputs) gives a correction to the
support-4 Kaiser-Bessel taps.  It is trained on the GPU by the library's own
kernels: ``rick_mlp_forward`` bakes the correction table on the lattice,
``rick_learn_field_grad`` images a point-source field (sources at continuous
positions) with Kaiser-Bessel taps plus that correction and measures it
against the direct Fourier inversion at probe pixels spread over the
taper-gated field, ``rick_mlp_backward`` carries the table gradient into
the network and ``rick_adam_step`` updates it.  This module only orders those
calls, draws the seeded fields, and saves/resumes the state (parameters, Adam
moments, step).

Start: the output layer is zero, so the untrained kernel is exactly the
support-4 Kaiser-Bessel -- the method without the learned part.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass

import numpy as np

from . import rick


def init_params(hidden: int, seed: int, zero_output: bool = True) -> np.ndarray:
    """He-scaled normal hidden weights, zero biases and (by default) a zero
    output layer, packed W1, b1, W2, b2, W3, b3."""
    g = np.random.Generator(np.random.Philox(key=[seed, 0x4D4C50]))
    H = hidden
    W1 = g.normal(0, math.sqrt(2.0 / 3.0), (H, 3))
    W2 = g.normal(0, math.sqrt(2.0 / H), (H, H))
    W3 = g.normal(0, math.sqrt(1.0 / H), (16, H))
    if zero_output:
        W3[:] = 0.0
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), W3.ravel(),
                           np.zeros(16)]).astype(np.float32)


def training_field(seed: int, N: int, margin: int = 4, n_range=(1, 50),
                   flux=(0.01, 1.0), inner: float | None = None) -> np.ndarray:
    """A point-source field: 1-50 sources at continuous positions anywhere in
    the image (margin pixels from the edge; positions in pixels, rounded to
    float32, which the library takes), fluxes log-uniform.  With inner, the
    sources lie in the central square of half-width inner * N instead (the
    square the probes are taken in).  [ns, 3] (p, q, A)."""
    g = np.random.Generator(np.random.Philox(key=[seed, 0x46494C44]))
    ns = int(g.integers(n_range[0], n_range[1] + 1))
    lo, hi = margin, N - margin
    if inner is not None:
        lo, hi = N // 2 - int(inner * N) + margin, N // 2 + int(inner * N) - margin
    pq = lo + g.random((ns, 2)) * (hi - lo)
    pq = pq.astype(np.float32).astype(np.float64)
    a = np.exp(math.log(flux[0]) + g.random(ns) * (math.log(flux[1]) - math.log(flux[0])))
    return np.concatenate([pq, a[:, None]], axis=1)


def field_probes(seed: int, N: int, src: np.ndarray, count: int = 64, inner: float = 0.4) -> np.ndarray:
    """The pixels a field is judged at, all inside the central square of
    half-width inner * N (for the support-4 Kaiser-Bessel taper, inner = 0.4
    keeps the taper gain C(p) C(q) / C(N/2)^2 above about 1e-2, so that no
    probe's error is amplified more than ~100 times by the taper division):
    the pixel nearest each of the field's brightest sources inside it (at
    most count // 4), the corners and edge midpoints of the square, and
    seeded pixels in it for the rest.  [count, 2] int32 (p, q)."""
    g = np.random.Generator(np.random.Philox(key=[seed, 0x50524F42]))
    h = N // 2
    e = int(inner * N)
    lo, hi = h - e, h + e - 1
    inside = (np.abs(src[:, 0] - h) <= e - 1) & (np.abs(src[:, 1] - h) <= e - 1)
    cand = np.nonzero(inside)[0]
    order = cand[np.argsort(-src[cand, 2])][: count // 4]
    near = np.clip(np.rint(src[order, :2]), lo, hi).astype(np.int64)
    fixed = np.array([(lo, lo), (hi, lo), (lo, hi), (hi, hi), (h, lo), (h, hi), (lo, h), (hi, h)],
                     dtype=np.int64)
    rest = g.integers(lo, hi + 1, size=(count - len(near) - len(fixed), 2))
    return np.concatenate([near, fixed, rest]).astype(np.int32)


def heldout_losses(learn: rick.Learn, table, n: int, seed0: int, loss, per_field: bool = False,
                   inner: float | None = None):
    """Loss of n held-out fields imaged with `table` (mean and median, or the
    losses themselves)."""
    out = []
    for s in range(n):
        src = training_field(seed0 + s, learn.cfg.N, inner=inner)
        learn.field_grad(table, src, field_probes(seed0 + s, learn.cfg.N, src), None, loss)
        out.append(float(loss.item()))
    if per_field:
        return np.array(out)
    return float(np.mean(out)), float(np.median(out))


@dataclass
class TrainState:
    step: int = 0
    seed: int = 0
    losses: list | None = None


class LearnedKernel:
    def __init__(self, n_wplanes: int, hidden: int = 64, lattice: int = 32, seed: int = 0,
                 zero_output: bool = True):
        import torch
        self.Nw, self.H, self.L = n_wplanes, hidden, lattice
        self.n_params = rick.mlp_param_count(hidden)
        self.params = torch.from_numpy(init_params(hidden, seed, zero_output)).cuda()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        npts = n_wplanes * (lattice + 1) ** 2
        self.lattice_in = torch.empty((npts, 3), dtype=torch.float32, device="cuda")
        rick.mlp_lattice_inputs(n_wplanes, lattice, self.lattice_in)
        self.table = torch.empty((npts, 16), dtype=torch.float32, device="cuda")
        self.table_grad = torch.empty_like(self.table)
        self.work = torch.empty((npts, 6 * hidden), dtype=torch.float32, device="cuda")
        self.scratch = torch.empty((npts, 16), dtype=torch.float32, device="cuda")
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.state = TrainState(seed=seed, losses=[])
        self.adam_t = 0

    def bake(self):
        """Evaluate the network on the lattice: the correction table the gridder reads."""
        rick.mlp_forward(self.params, self.H, self.lattice_in, self.table)
        return self.table

    def _update(self, lr):
        self.grad.zero_()
        rick.mlp_backward(self.params, self.H, self.lattice_in, self.table_grad, self.grad,
                          self.work, self.scratch)
        self.adam_t += 1
        rick.adam_step(self.params, self.grad, self.m, self.v, lr, self.adam_t)

    def train(self, learn: rick.Learn, updates: int, lr: float = 1e-5, batch: int = 8,
              N: int | None = None, log_every: int = 0, field_seed0: int = 1_000_000,
              lr_final: float | None = None, inner: float | None = None):
        """``updates`` Adam steps, each on the mean gradient of ``batch`` fields
        (field seeds field_seed0 + 0, 1, 2, ... in order, so a resumed run
        sees the same sequence; ``inner`` as for training_field).  The
        learning rate decays on a cosine from lr to lr_final (default lr / 10)."""
        N = N or learn.cfg.N
        lr_final = lr / 10 if lr_final is None else lr_final
        last = []
        for u in range(updates):
            self.bake()
            total = 0.0
            for b in range(batch):
                seed = field_seed0 + self.state.step
                src = training_field(seed, N, inner=inner)
                learn.field_grad(self.table, src, field_probes(seed, N, src), self.table_grad,
                                 self.loss, accumulate=b > 0, grad_scale=1.0 / batch)
                self.state.step += 1
                if log_every:
                    total += float(self.loss.item())
            c = 0.5 * (1 + math.cos(math.pi * u / max(1, updates)))
            self._update(lr_final + (lr - lr_final) * c)
            if log_every and (u + 1) % log_every == 0:
                last.append(total / batch)
                self.state.losses.append(("field", self.state.step, total / batch))
        return last

    def heldout_loss(self, learn: rick.Learn, n: int = 32, seed0: int = 9_000_000,
                     inner: float | None = None):
        """Mean and median loss over n held-out fields (seeds never trained on)."""
        self.bake()
        return heldout_losses(learn, self.table, n, seed0, self.loss, inner=inner)

    def losses(self, learn: rick.Learn, n: int = 32, seed0: int = 9_000_000,
               inner: float | None = None) -> np.ndarray:
        """The loss of each of n held-out fields (seeds never trained on)."""
        self.bake()
        return heldout_losses(learn, self.table, n, seed0, self.loss, per_field=True, inner=inner)

    # ---- checkpoint / resume ------------------------------------------------
    def save(self, path: str):
        np.savez(path, params=self.params.cpu().numpy(), m=self.m.cpu().numpy(),
                 v=self.v.cpu().numpy())
        with open(path + ".json", "w") as f:
            json.dump({"step": self.state.step, "adam_t": self.adam_t, "seed": self.state.seed, "H": self.H,
                       "L": self.L, "Nw": self.Nw}, f)

    @classmethod
    def load(cls, path: str) -> "LearnedKernel":
        import torch
        with open(path + ".json") as f:
            meta = json.load(f)
        k = cls(meta["Nw"], meta["H"], meta["L"], meta["seed"])
        z = np.load(path if path.endswith(".npz") else path + ".npz")
        k.params.copy_(torch.from_numpy(z["params"]))
        k.m.copy_(torch.from_numpy(z["m"]))
        k.v.copy_(torch.from_numpy(z["v"]))
        k.state.step = meta["step"]
        k.adam_t = meta["adam_t"]
        return k
