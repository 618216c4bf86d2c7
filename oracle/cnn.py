"""Learned denoiser for Step 4 of Algorithm 1: a residual 3x3 CNN (FP64 reference).

Section 4.3 treats the denoiser as a black box and the paper notes that the
framework extends to deep-learning denoisers (Section 1, citing the DnCNN
line of work).  This module is the FP64 reference of the network the CUDA
library trains and runs:

* f: 17 convolution layers, 3x3 kernels, zero ("same") padding, channels
  1 -> 64 -> ... -> 64 -> 1, a bias per output channel, ReLU after layers
  1..16 and none after layer 17;
* residual form (DnCNN): the network predicts the noise, D(r) = r - f(r);
* scale normalisation: for the GAMP input r with effective noise variance
  tau_r, D_tau(r) = r - sigma f(r / sigma), sigma = sqrt(tau_r), so one
  network serves every iteration (f sees unit-variance noise).

Layout: images [B][H][W]; hidden activations [B][H][W][C] (channels last);
weights ``w[l]`` of shape [3][3][C_in][C_out] (tap (dy, dx) = (ky - 1, kx - 1)
reads input pixel (y + dy, x + dx)), biases ``b[l]`` of shape [C_out].

``bf16=True`` rounds every hidden activation (after ReLU) to bfloat16
(round-to-nearest-even), which is exactly where the GPU stores them in
bfloat16; gradients treat the rounding as the identity.
"""
from __future__ import annotations

import numpy as np

LAYERS = 17
CHANNELS = 64


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    out = u.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


def init_params(seed: int, layers: int = LAYERS, channels: int = CHANNELS, bf16: bool = True):
    """He-initialised weights (std sqrt(2 / (9 C_in))), last layer scaled by 0.1, zero biases."""
    rng = np.random.default_rng(seed)
    ws, bs = [], []
    for l in range(layers):
        cin = 1 if l == 0 else channels
        cout = 1 if l == layers - 1 else channels
        w = rng.standard_normal((3, 3, cin, cout)) * np.sqrt(2.0 / (9 * cin))
        if l == layers - 1:
            w *= 0.1
        ws.append(bf16_round(w) if bf16 else w)
        bs.append(np.zeros(cout))
    return ws, bs


def _shift(a, dy, dx):
    """out[..., y, x, :] = a[..., y + dy, x + dx, :] with zeros outside."""
    out = np.zeros_like(a)
    H, W = a.shape[1], a.shape[2]
    ys, yd = (slice(dy, H), slice(0, H - dy)) if dy >= 0 else (slice(0, H + dy), slice(-dy, H))
    xs, xd = (slice(dx, W), slice(0, W - dx)) if dx >= 0 else (slice(0, W + dx), slice(-dx, W))
    out[:, yd, xd, :] = a[:, ys, xs, :]
    return out


def conv3x3(a: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Same-padded 3x3 convolution, a [B][H][W][Cin], w [3][3][Cin][Cout]."""
    out = np.broadcast_to(b, a.shape[:3] + (w.shape[3],)).copy()
    for ky in range(3):
        for kx in range(3):
            out += _shift(a, ky - 1, kx - 1) @ w[ky, kx]
    return out


def conv3x3_input_grad(g: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv3x3 with respect to its input."""
    gin = np.zeros(g.shape[:3] + (w.shape[2],))
    for ky in range(3):
        for kx in range(3):
            gin += _shift(g @ w[ky, kx].T, -(ky - 1), -(kx - 1))
    return gin


def conv3x3_weight_grad(a: np.ndarray, g: np.ndarray):
    """Gradients of conv3x3 with respect to w and b."""
    gw = np.zeros((3, 3, a.shape[3], g.shape[3]))
    for ky in range(3):
        for kx in range(3):
            sa = _shift(a, ky - 1, kx - 1)
            gw[ky, kx] = sa.reshape(-1, a.shape[3]).T @ g.reshape(-1, g.shape[3])
    return gw, g.reshape(-1, g.shape[3]).sum(axis=0)


def net_forward(x: np.ndarray, ws, bs, bf16: bool = False):
    """f(x) for images x [B][H][W]; returns (f [B][H][W], cache for the backward pass)."""
    a = np.asarray(x, dtype=np.float64)[..., None]
    acts = [a]
    L = len(ws)
    for l in range(L):
        z = conv3x3(a, ws[l], bs[l])
        if l < L - 1:
            a = np.maximum(z, 0.0)
            if bf16:
                a = bf16_round(a)
        else:
            a = z
        acts.append(a)
    return a[..., 0], acts


def net_backward(gout: np.ndarray, ws, acts):
    """Gradients of sum(gout * f) w.r.t. every weight and bias (ReLU masks from the cache)."""
    L = len(ws)
    g = np.asarray(gout, dtype=np.float64)[..., None]
    gws, gbs = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        gws[l], gbs[l] = conv3x3_weight_grad(acts[l], g)
        if l > 0:
            g = conv3x3_input_grad(g, ws[l]) * (acts[l] > 0)
    return gws, gbs


def net_jvp(x: np.ndarray, t: np.ndarray, ws, bs, bf16: bool = False):
    """Forward-mode derivative of f: returns (f(x), J_f(x) t) for images [B][H][W].

    f is piecewise linear (ReLU), so J_f(x) t is the same chain of
    convolutions without biases, each hidden output masked where the
    primal pre-activation is not positive (ReLU'(z) = [z > 0]).  With
    ``bf16`` the primal activations and the tangent's hidden activations are
    both rounded to bfloat16 after the ReLU / mask."""
    a = np.asarray(x, dtype=np.float64)[..., None]
    u = np.asarray(t, dtype=np.float64)[..., None]
    L = len(ws)
    for l in range(L):
        z = conv3x3(a, ws[l], bs[l])
        zt = conv3x3(u, ws[l], np.zeros_like(bs[l]))
        if l < L - 1:
            on = z > 0
            a = np.where(on, z, 0.0)
            u = np.where(on, zt, 0.0)
            if bf16:
                a = bf16_round(a)
                u = bf16_round(u)
        else:
            a, u = z, zt
    return a[..., 0], u[..., 0]


def denoise_jvp(r: np.ndarray, b: np.ndarray, sigma: float, ws, bs, bf16: bool = False):
    """(D_sigma(r), J_D(r) b) for one image: D = r - sigma f(r / sigma) gives
    J_D b = b - sigma J_f(r / sigma) (b / sigma)."""
    r = np.asarray(r, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    f, tf = net_jvp((r / sigma)[None], (b / sigma)[None], ws, bs, bf16)
    return r - sigma * f[0], b - sigma * tf[0]


class Denoiser:
    """D_sigma of one GAMP iteration as a callable with its exact directional
    derivative ``jvp(r, b) = J_D(r) b`` (used for the epsilon -> 0 limit of
    Eq. MC_SURE)."""

    def __init__(self, sigma: float, ws, bs, bf16: bool = True):
        self.sigma, self.ws, self.bs, self.bf16 = sigma, ws, bs, bf16

    def __call__(self, r):
        return denoise(r, self.sigma, self.ws, self.bs, self.bf16)

    def jvp(self, r, b):
        return denoise_jvp(r, b, self.sigma, self.ws, self.bs, self.bf16)[1]


def denoise(r: np.ndarray, sigma: float, ws, bs, bf16: bool = False) -> np.ndarray:
    """D_sigma(r) = r - sigma f(r / sigma) for one image or a batch [B][H][W]."""
    r = np.asarray(r, dtype=np.float64)
    batch = r[None] if r.ndim == 2 else r
    f, _ = net_forward(batch / sigma, ws, bs, bf16)
    out = batch - sigma * f
    return out[0] if r.ndim == 2 else out


def loss_and_grads(r, x_true, sigma, ws, bs, bf16: bool = False):
    """Training loss mean(((D(r) - x_true) / sigma)^2) over a batch, and its gradients.

    Dividing each patch's error by its noise level weighs all noise levels
    alike (for sigma = 1 it is the plain mean squared error)."""
    r = np.asarray(r, dtype=np.float64)
    sg = np.asarray(sigma, dtype=np.float64)[:, None, None]
    f, acts = net_forward(r / sg, ws, bs, bf16)
    d = r - sg * f
    e = (d - x_true) / sg
    loss = float(np.mean(e * e))
    gout = -2.0 * e / e.size
    gws, gbs = net_backward(gout, ws, acts)
    return loss, gws, gbs
