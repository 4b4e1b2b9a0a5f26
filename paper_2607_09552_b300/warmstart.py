"""Learned warm start of the steady UGKWP-LTS iteration.

A coordinate MLP (Fourier features of stretched coordinates plus the case conditions Kn, Ma, T_w; 4 hidden
SiLU layers of 256; outputs log rho, u / U_inf, v / U_inf, log T) is trained on converged fields that the
method itself produces and then sets the field a new case starts from (`Solver.warm_start`). The local time
steps stay those of the freestream start and the iteration is unchanged, so the converged state is the
method's own; the freestream start remains the fallback. The paper has no such network; it shortens the
transient of the steady iteration (Sec. III C, Sec. IV B) only.

Everything numeric runs in the library's kernels through its C ABI (features, forward, backward, Adam,
field averaging, training pairs, warm start); this module only sequences the calls, draws the minibatch
order (seeded, on the host) and moves the index arrays to the device. One network per geometry family
(cylinder O-meshes, flat plates), because the inputs (x, y, Kn, Ma, T_w) carry no geometry descriptor.
"""
from __future__ import annotations

import math

import numpy as np

from . import ugkwp
from . import workloads as wl

N_FEATURES, WIDTH, DEPTH = 64, 256, 4

_RANGES = dict(kn_lo=0.005, kn_hi=0.2, ma_lo=5.0, ma_hi=15.0, tw_lo=1.0, tw_hi=5.0)
FAMILY_MAPS = {
    # cylinder of diameter 1 at the origin: stretching on the radius 0.5, outer boundary up to 20 D
    "cylinder": dict(cx=0.0, cy=0.0, ell=0.5, ext=20.0, **_RANGES),
    # plate leading edge at the origin, wall on y = 0: stretching on 0.05 L, domain up to about 2 L
    "plate": dict(cx=0.0, cy=0.0, ell=0.05, ext=2.0, **_RANGES),
}


def family(case) -> str:
    m = case.mesh
    # an unstructured plate mesh carries the plate length L in its info, a cylinder mesh the radius
    plate = m.kind == wl.MESH_PLATE or (m.kind == wl.MESH_UNSTRUCTURED and "L" in m.info)
    return "plate" if plate else "cylinder"


def averaged_field(solver, n_steps: int, every: int = 1):
    """Time average of the conservative field over the next n_steps (sampled every `every` steps) as a
    float64 CUDA tensor (4 C), summed on the device."""
    import torch
    acc = torch.zeros(4 * solver.C, dtype=torch.float64, device="cuda")
    n = 0
    for k in range(n_steps):
        solver.step(1)
        if k % every == 0:
            solver.field_accumulate(acc, reset=(n == 0))
            n += 1
    return acc, 1.0 / n


class TrainingSet:
    """Feature and target rows of several converged fields, concatenated on the device."""

    def __init__(self):
        self.feats, self.targs, self.sizes = [], [], []

    def add(self, solver, fmap: dict, W=None, scale: float = 1.0):
        f, t = solver.dataset(fmap, W, scale, N_FEATURES)
        self.feats.append(f)
        self.targs.append(t)
        self.sizes.append(solver.C)

    def tensors(self):
        import torch
        return torch.cat(self.feats).contiguous(), torch.cat(self.targs).contiguous()


def train(mlp, feats, targs, steps: int = 3000, batch: int = 8192, lr: float = 2e-3, lr_final: float = 5e-5,
          seed: int = 0, log_every: int = 0):
    """Adam on minibatches drawn without replacement (a new seeded permutation each epoch), learning rate
    decayed along a cosine from lr to lr_final. Returns [(step, loss), ...] sampled every log_every steps
    plus the last step."""
    import torch
    n = feats.shape[0]
    batch = min(batch, n)
    rng = np.random.default_rng(seed)
    per_epoch = max(1, n // batch)
    hist = []
    perm = None
    for k in range(steps):
        e = k % per_epoch
        if e == 0:
            perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).to("cuda", non_blocking=False)
        rows = perm[e * batch:(e + 1) * batch]
        want = (log_every and k % log_every == 0) or k == steps - 1
        loss = mlp.loss_grad(feats, targs, rows, want_loss=bool(want))
        a = 0.5 * (1.0 + math.cos(math.pi * k / max(steps - 1, 1)))
        mlp.adam(lr_final + (lr - lr_final) * a)
        if want:
            hist.append((k, loss))
    return hist


def new_network(seed: int = 0):
    return ugkwp.Mlp(N_FEATURES, WIDTH, DEPTH, 4, params=wl.mlp_init(seed, N_FEATURES, WIDTH, DEPTH))
