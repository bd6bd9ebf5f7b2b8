"""FP64 oracle of the learned proximal denoiser: a residual CNN of 3x3
convolutions that replaces the TV prox inside the FISTA loop (plug-and-play
use of a learned prior; the paper's learned prior is the patch dictionary of
Sec. 3.2, the network is its convolutional counterpart).

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg use this module; the library never does.

Network (channel widths C = [1, 32, 32, 32, 32, 32, 32, 32, 1], 8 layers):
    a_0 = z
    a_l = ReLU(conv3x3(a_{l-1}; W_l) + b_l),  l = 1 .. 7
    r   = conv3x3(a_7; W_8) + b_8
    out = z + r
conv3x3 is cross-correlation with zero padding ("same" size):
    conv(a; W)[o, i, j] = sum_{c, u, v} W[o, c, u, v] a[c, i + u - 1, j + v - 1].
Stored precision (the network's definition): weights and the hidden
activations a_1 .. a_7 are bfloat16 (round to nearest even), z, the biases,
r and out are float32 values; sums are exact here (FP64).

Parameters are one flat float vector: for l = 1 .. 8, W_l [C_l][C_{l-1}][3][3]
row-major, then b_l [C_l].

Training: loss = mean over pixels of (out - target)^2; its gradient is
computed by the chain rule in FP64 with the bf16 rounding of activations
treated as the identity (the straight-through reading), and Adam (Kingma &
Ba 2015) updates the float32 master parameters.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (1, 32, 32, 32, 32, 32, 32, 32, 1)
N_LAYERS = len(CHANNELS) - 1


def param_shapes(channels=CHANNELS):
    out = []
    for l in range(1, len(channels)):
        out.append(((channels[l], channels[l - 1], 3, 3), (channels[l],)))
    return out


def n_params(channels=CHANNELS):
    return sum(int(np.prod(w)) + int(np.prod(b)) for w, b in param_shapes(channels))


def unpack(params, channels=CHANNELS):
    """Flat vector -> list of (W_l, b_l) views."""
    params = np.asarray(params)
    out, k = [], 0
    for ws, bs in param_shapes(channels):
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((params[k:k + nw].reshape(ws), params[k + nw:k + nw + nb].reshape(bs)))
        k += nw + nb
    assert k == params.size
    return out


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), returned
    as float64: keep the top 16 bits of the float32 pattern after adding
    0x7FFF plus the lowest kept bit (finite inputs)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def f32_round(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def conv3x3(a, W, b=None):
    """a [C_in][H][W], W [C_out][C_in][3][3] -> [C_out][H][W], zero padding."""
    cin, h, w = a.shape
    pad = np.zeros((cin, h + 2, w + 2))
    pad[:, 1:-1, 1:-1] = a
    out = np.zeros((W.shape[0], h, w))
    for u in range(3):
        for v in range(3):
            out += np.einsum("oc,chw->ohw", W[:, :, u, v], pad[:, u:u + h, v:v + w])
    if b is not None:
        out += b[:, None, None]
    return out


def forward(params, z, rounding=True, channels=CHANNELS):
    """z [H][W] -> (out [H][W], activations [a_0 .. a_7], pre-activations).
    With rounding the weights and hidden activations take their bf16 values
    and z, r, out their float32 values."""
    layers = unpack(np.asarray(params, dtype=np.float64), channels)
    rw = bf16_round if rounding else (lambda t: np.asarray(t, dtype=np.float64))
    rf = f32_round if rounding else (lambda t: np.asarray(t, dtype=np.float64))
    z = rf(z)
    acts, pres = [z[None]], []
    a = z[None]
    for l, (W, b) in enumerate(layers):
        s = conv3x3(a, rw(W), rf(b))
        pres.append(s)
        if l < len(layers) - 1:
            a = rw(np.maximum(s, 0.0))
            acts.append(a)
    r = rf(s[0])
    out = rf(z + r)
    return out, acts, pres


def loss_and_grad(params, z, target, rounding=True, channels=CHANNELS):
    """Mean squared error of one image and its gradient with respect to the
    flat parameter vector (FP64, chain rule; rounding treated as identity)."""
    layers = unpack(np.asarray(params, dtype=np.float64), channels)
    rw = bf16_round if rounding else (lambda t: np.asarray(t, dtype=np.float64))
    out, acts, pres = forward(params, z, rounding, channels)
    npx = out.size
    loss = float(np.mean((out - target) ** 2))
    d = (2.0 / npx) * (out - target)[None]          # d loss / d pre-activation of the last layer
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a = acts[l]
        cin, h, w = a.shape
        pad = np.zeros((cin, h + 2, w + 2))
        pad[:, 1:-1, 1:-1] = a
        gW = np.empty(W.shape)
        for u in range(3):
            for v in range(3):
                gW[:, :, u, v] = np.einsum("ohw,chw->oc", d, pad[:, u:u + h, v:v + w])
        gb = d.sum(axis=(1, 2))
        grads[l] = (gW, gb)
        if l > 0:
            # d loss / d a_l = correlation of d with the flipped, transposed kernel
            Wt = rw(W)[:, :, ::-1, ::-1].transpose(1, 0, 2, 3)
            da = conv3x3(d, Wt)
            d = da * (pres[l - 1] > 0.0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb.ravel()]) for gW, gb in grads])
    return loss, flat


def adam_step(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of float64 copies;
    step counts from 1.  Returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v



def pnp_fista(geo, sino, params, L, n_iter, use_fista=True, x0=None):
    """FISTA/ISTA with the network as the prox (plug-and-play): the steps of
    the oracle's FISTA on Eq. 3 (gradient step of length 1/L on
    1/2 ||sino - P x||^2, prox, momentum of Beck-Teboulle) with
    x_k = forward(params, z_k) in place of the TV prox.  ``geo`` is an
    oracle Geometry.  Returns (x, data term 1/2 ||sino - P x_k||^2 per
    iteration)."""
    sino = np.asarray(sino, dtype=np.float64)
    x = np.zeros((geo.ny, geo.nx)) if x0 is None else np.array(x0, dtype=np.float64)
    y, xprev, t = x.copy(), x.copy(), 1.0
    energy = []
    for _ in range(n_iter):
        z = y - geo.PT(geo.P(y) - sino) / L
        x, _, _ = forward(params, z, rounding=True)
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t)) if use_fista else 1.0
        w = (t - 1.0) / tn if use_fista else 0.0
        y = x + w * (x - xprev)
        xprev, t = x.copy(), tn
        energy.append(0.5 * np.sum((sino - geo.P(x)) ** 2))
    return x, np.array(energy)
