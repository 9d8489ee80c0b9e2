"""FP64 oracle of the MLP constitutive surrogate (test infrastructure only).

The paper notes that a surrogate constitutive model can replace the explicit material
function and that its Jacobian is extracted the same way (Section III-B).  The surrogate
read here: inputs x = [E_voigt / in_scale (6), one-hot phase (2)], three hidden layers of
64 SiLU units, a linear output of 6 normalised second Piola-Kirchhoff components,
de-normalised per phase as S_c = y_c * out_scale[p, c] + out_shift[p, c].  Its tangent
dS/dE is the network's input-Jacobian (forward chain rule through the layers).
Training minimises the mean squared error over the batch and the 6 outputs with Adam.

Layers are [(W [out, in], b [out])] * 4.  silu(z) = z * sigmoid(z).
"""
from __future__ import annotations

import numpy as np


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_prime(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(layers, x, keep=False):
    """y = W4 silu(W3 silu(W2 silu(W1 x + b1) + b2) + b3) + b4 for a batch x [n, 8]."""
    a = np.asarray(x, dtype=np.float64)
    zs, acts = [], [a]
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        if li < len(layers) - 1:
            zs.append(z)
            a = silu(z)
            acts.append(a)
        else:
            a = z
    return (a, zs, acts) if keep else a


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def gradients(layers, x, t):
    """Loss = mean((y - t)^2) over all n*6 entries; returns (loss, [(dW, db)] per layer)
    by reverse-mode differentiation."""
    y, zs, acts = forward(layers, x, keep=True)
    n = y.shape[0]
    d = 2.0 * (y - t) / (n * y.shape[1])  # dLoss/dy
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        grads[li] = (d.T @ acts[li], d.sum(axis=0))
        if li > 0:
            d = (d @ W) * silu_prime(zs[li - 1])
    return mse(y, t), grads


def input_jacobian(layers, x, n_in=6):
    """dy/dx[:, :n_in] per sample: W4 diag(silu'(z3)) W3 diag(silu'(z2)) W2 diag(silu'(z1))
    W1[:, :n_in].  Returns [n, 6, n_in]."""
    _, zs, _ = forward(layers, x, keep=True)
    W1 = layers[0][0][:, :n_in]
    Jm = silu_prime(zs[0])[:, :, None] * W1[None, :, :]
    for li in (1, 2):
        W = layers[li][0]
        Jm = silu_prime(zs[li])[:, :, None] * np.einsum("oh,nhi->noi", W, Jm)
    return np.einsum("oh,nhi->noi", layers[3][0], Jm)


class Adam:
    """Adam with bias correction: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    w -= lr * mhat / (sqrt(vhat) + eps)."""

    def __init__(self, layers, b1=0.9, b2=0.999, eps=1e-8):
        self.b1, self.b2, self.eps, self.t = b1, b2, eps, 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in layers]

    def step(self, layers, grads, lr):
        self.t += 1
        c1, c2 = 1.0 - self.b1 ** self.t, 1.0 - self.b2 ** self.t
        out = []
        for li, ((W, b), (gW, gb)) in enumerate(zip(layers, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[li][j] + (1 - self.b1) * g
                v = self.b2 * self.v[li][j] + (1 - self.b2) * g * g
                self.m[li] = self.m[li][:j] + (m,) + self.m[li][j + 1:]
                self.v[li] = self.v[li][:j] + (v,) + self.v[li][j + 1:]
                new.append(p - lr * (m / c1) / (np.sqrt(v / c2) + self.eps))
            out.append(tuple(new))
        return out


def surrogate_inputs(E6, phase, in_scale):
    E6 = np.asarray(E6, dtype=np.float64)
    x = np.zeros((E6.shape[0], 8))
    x[:, :6] = E6 / in_scale
    x[np.arange(len(phase)), 6 + np.asarray(phase)] = 1.0
    return x


def surrogate_stress(layers, E6, phase, in_scale, out_scale, out_shift):
    """S (Voigt, tensor shear) and dS/dE (6x6 w.r.t. the tensor components of E)."""
    phase = np.asarray(phase)
    x = surrogate_inputs(E6, phase, in_scale)
    y = forward(layers, x)
    sc, sh = np.asarray(out_scale)[phase], np.asarray(out_shift)[phase]
    S = y * sc + sh
    D = input_jacobian(layers, x) * sc[:, :, None] / in_scale
    return S, D
