"""ORACLE (test infrastructure only): plain float64 numpy definition of the learned warm start's network.

Only tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import this module.

What it defines (the warm start maps a cell centroid and the case conditions (x, y, Kn, Ma, T_w) to an
initial macroscopic field (rho, u, v, T); the method itself, Sec. III C and Sec. IV B, is unchanged by it:
only the field the steady iteration starts from changes):
- `coord_map`, `features`: stretched coordinates x^ = asinh((x - c)/l) / asinh(X/l) in [-1, 1], eight
  octaves of Fourier features sin/cos(2^k pi x^), sin/cos(2^k pi y^) (k = 0..7), the raw x^, y^, and the
  conditions log10 Kn, Ma, T_w mapped linearly to [-1, 1]; 37 values zero-padded to 64.
- `forward`, `loss_and_grad`: an MLP of `depth` hidden SiLU layers of `width` units and a linear output
  layer; mean squared error over the points and the 4 outputs; the analytic backward pass. Weights are used
  as rounded to bfloat16 (round to nearest even) when `bf16=True`, the gradient being the one with respect
  to those effective weights (applied to the float32 master weights).
- `adam`: Adam with bias correction (Kingma & Ba, 2015).
- `targets_from_W`, `field_from_outputs`: (log rho, u/U_inf, v/U_inf, log T) from conservative variables and
  back, with R = 1/2 and a monatomic gas (rho E = rho (|U|^2/2 + 3RT/2)).

Parameter vector layout (shared with the CUDA library's interface, not its code): every layer's weight
matrix [out][in] row-major in layer order, then every layer's bias in layer order.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 64
N_OCTAVES = 8
N_OUT = 4
R_GAS = 0.5


def layer_shapes(n_features: int, width: int, depth: int, n_out: int = N_OUT):
    ins = [n_features] + [width] * depth
    outs = [width] * depth + [n_out]
    return list(zip(ins, outs))


def n_params(n_features: int, width: int, depth: int, n_out: int = N_OUT) -> int:
    return sum(i * o + o for i, o in layer_shapes(n_features, width, depth, n_out))


def unpack(p: np.ndarray, n_features: int, width: int, depth: int, n_out: int = N_OUT):
    """Views (W_l [out][in], b_l [out]) of the flat parameter vector."""
    shapes = layer_shapes(n_features, width, depth, n_out)
    Ws, bs, off = [], [], 0
    for i, o in shapes:
        Ws.append(p[off:off + i * o].reshape(o, i))
        off += i * o
    for i, o in shapes:
        bs.append(p[off:off + o])
        off += o
    return Ws, bs


def bf16_round(a: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 (round to nearest, ties to even) -> float64. Finite inputs only."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def coord_map(x, c, ell, ext):
    return np.arcsinh((np.asarray(x, dtype=np.float64) - c) / ell) / np.arcsinh(ext / ell)


def norm_cond(v, lo, hi):
    return 2.0 * (v - lo) / (hi - lo) - 1.0


def features(x, y, Kn, Ma, Tw, fmap: dict) -> np.ndarray:
    """Feature rows [n][64] for points (x, y) of one case with conditions (Kn, Ma, T_w)."""
    xh = coord_map(x, fmap["cx"], fmap["ell"], fmap["ext"])
    yh = coord_map(y, fmap["cy"], fmap["ell"], fmap["ext"])
    n = xh.shape[0]
    f = np.zeros((n, N_FEATURES))
    for k in range(N_OCTAVES):
        f[:, k] = np.sin(2.0 ** k * np.pi * xh)
        f[:, N_OCTAVES + k] = np.cos(2.0 ** k * np.pi * xh)
        f[:, 2 * N_OCTAVES + k] = np.sin(2.0 ** k * np.pi * yh)
        f[:, 3 * N_OCTAVES + k] = np.cos(2.0 ** k * np.pi * yh)
    f[:, 32] = xh
    f[:, 33] = yh
    f[:, 34] = norm_cond(np.log10(Kn), np.log10(fmap["kn_lo"]), np.log10(fmap["kn_hi"]))
    f[:, 35] = norm_cond(Ma, fmap["ma_lo"], fmap["ma_hi"])
    f[:, 36] = norm_cond(Tw, fmap["tw_lo"], fmap["tw_hi"])
    return f


def forward(p, X, n_features, width, depth, bf16=True, cache=False):
    Ws, bs = unpack(np.asarray(p, dtype=np.float64), n_features, width, depth)
    if bf16:
        Ws = [bf16_round(W) for W in Ws]
    a = np.asarray(X, dtype=np.float64)
    acts, pres = [a], []
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W.T + b
        pres.append(z)
        a = silu(z) if l < depth else z
        acts.append(a)
    if cache:
        return a, (Ws, acts, pres)
    return a


def loss_and_grad(p, X, T, n_features, width, depth, bf16=True):
    """Mean squared error over n points x 4 outputs and its gradient (flat, same layout as p)."""
    Y, (Ws, acts, pres) = forward(p, X, n_features, width, depth, bf16=bf16, cache=True)
    n = Y.shape[0]
    E = Y - np.asarray(T, dtype=np.float64)
    loss = float(np.sum(E * E) / (N_OUT * n))
    dY = 2.0 * E / (N_OUT * n)
    gW, gb = [None] * (depth + 1), [None] * (depth + 1)
    for l in range(depth, -1, -1):
        dZ = dY * silu_grad(pres[l]) if l < depth else dY
        gW[l] = dZ.T @ acts[l]
        gb[l] = dZ.sum(axis=0)
        dY = dZ @ Ws[l]
    g = np.concatenate([w.ravel() for w in gW] + list(gb))
    return loss, g


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def targets_from_W(W: np.ndarray, U_inf: float) -> np.ndarray:
    """W [n][4] conservative (rho, rho u, rho v, rho E) -> (log rho, u/U_inf, v/U_inf, log T)."""
    rho = W[:, 0]
    u, v = W[:, 1] / rho, W[:, 2] / rho
    e = W[:, 3] / rho - 0.5 * (u * u + v * v)
    T = e / (1.5 * R_GAS)
    return np.stack([np.log(rho), u / U_inf, v / U_inf, np.log(T)], axis=1)


def field_from_outputs(Y: np.ndarray, U_inf: float, T_min: float, T_cap: float, U_cap: float,
                       rho_lo: float = 1e-6, rho_hi: float = 1e6) -> np.ndarray:
    """Network outputs -> primitive field [n][4] = (rho, u, v, T), clipped to the realizable range
    (rho in [rho_lo, rho_hi], T in [T_min, T_cap], speed at most U_cap)."""
    rho = np.clip(np.exp(np.clip(Y[:, 0], -700.0, 700.0)), rho_lo, rho_hi)
    u, v = Y[:, 1] * U_inf, Y[:, 2] * U_inf
    sp = np.sqrt(u * u + v * v)
    s = np.where(sp > U_cap, U_cap / np.where(sp > 0, sp, 1.0), 1.0)
    T = np.clip(np.exp(np.clip(Y[:, 3], -700.0, 700.0)), T_min, T_cap)
    return np.stack([rho, u * s, v * s, T], axis=1)
