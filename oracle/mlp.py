"""CPU reference of the learned start network -- TEST INFRASTRUCTURE.

The learned initial subspace maps an instance's potential scalars, its search
interval and a layer's z position to the coefficients of the start block Y on
a separable sine basis of that layer.  This module holds the plain numpy
float64 restatement the GPU kernels are checked against: a 4-layer MLP
(width 512, SiLU after the first three layers), its weighted mean-squared
loss, the exact backward pass, and the sine-basis expansion / projection.

``bf16=True`` rounds the inputs of every matrix product to bfloat16 (round to
nearest even), the points where the GPU kernels store bfloat16 operands, and
keeps float64 accumulation.
"""

from __future__ import annotations

import math

import numpy as np


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Nearest-even rounding of float32 values to bfloat16 (kept as float64)."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(sizes, seed: int):
    """W_k (out x in) ~ N(0, 1/in), b_k = 0."""
    rng = np.random.default_rng(seed)
    params = []
    for fin, fout in zip(sizes[:-1], sizes[1:]):
        params.append((rng.standard_normal((fout, fin)) / math.sqrt(fin), np.zeros(fout)))
    return params


def forward(params, x, bf16: bool = False):
    """x: (B, in).  Returns the output and the cache of pre-activations and
    layer inputs for the backward pass."""
    rnd = round_bf16 if bf16 else (lambda a: a)
    h = x
    cache = []
    for k, (W, b) in enumerate(params):
        hin = rnd(h)
        z = hin @ rnd(W).T + b
        cache.append((hin, z))
        h = silu(z) if k < len(params) - 1 else z
    return h, cache


def loss(out, target, weights):
    """L = sum_{b,o} w_o (out - target)^2 / (2 B)."""
    B = out.shape[0]
    return float(np.sum(weights[None, :] * (out - target) ** 2) / (2.0 * B))


def backward(params, cache, out, target, weights, bf16: bool = False):
    """Exact gradients of `loss` with respect to every (W_k, b_k)."""
    rnd = round_bf16 if bf16 else (lambda a: a)
    B = out.shape[0]
    g = weights[None, :] * (out - target) / B          # dL/d(out)
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        W, _ = params[k]
        hin, z = cache[k]
        if k < len(params) - 1:
            g = g * silu_grad(z)                       # through the activation
        gW = rnd(g).T @ hin
        gb = g.sum(axis=0)
        grads[k] = (gW, gb)
        if k > 0:
            g = rnd(g) @ rnd(W)                        # dL/d(input of layer k)
    return grads


def sine_basis(m: int, modes: int) -> np.ndarray:
    """Orthonormal discrete sine vectors s_p(i) = sqrt(2/(m+1)) sin(p pi (i+1)/(m+1)),
    p = 1..modes, as an (m, modes) array."""
    i = np.arange(1, m + 1)[:, None]
    p = np.arange(1, modes + 1)[None, :]
    return math.sqrt(2.0 / (m + 1)) * np.sin(p * math.pi * i / (m + 1))


def expand(coef: np.ndarray, nx: int, ny: int, nz: int, px: int, py: int) -> np.ndarray:
    """Y[l*n + ix + nx*iy, c] = sum_{p<px, q<py} coef[l, c, q*px + p] s_p(ix) s_q(iy)
    for coef of shape (nz, M0, px*py); returns Y as (N, M0)."""
    Sx, Sy = sine_basis(nx, px), sine_basis(ny, py)
    C = coef.reshape(nz, coef.shape[1], py, px)
    Y = np.einsum("lcqp,xp,yq->lyxc", C, Sx, Sy)
    return Y.reshape(nz * ny * nx, coef.shape[1])


def project(X: np.ndarray, nx: int, ny: int, nz: int, px: int, py: int) -> np.ndarray:
    """Adjoint of `expand`: coef[l, c, q*px + p] = sum_{ix,iy} X[l*n + ix + nx*iy, c] s_p(ix) s_q(iy)."""
    Sx, Sy = sine_basis(nx, px), sine_basis(ny, py)
    Xl = X.reshape(nz, ny, nx, X.shape[1])
    C = np.einsum("lyxc,xp,yq->lcqp", Xl, Sx, Sy)
    return C.reshape(nz, X.shape[1], px * py)
