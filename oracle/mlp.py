"""FP64 reference of the learned-guess network (three linear layers, SiLU).

TEST INFRASTRUCTURE ONLY.  Written from the definitions
    z1 = x W1 + b1, h1 = silu(z1), z2 = h1 W2 + b2, h2 = silu(z2), y = h2 W3 + b3,
    loss = sum(mask (y - t)^2) / sum(mask),  silu(z) = z / (1 + exp(-z)),
with the gradient by the chain rule; pinned by central finite differences in
tests/test_oracle_pins.py.  Parameters are one flat vector laid out
W1 [nin x w], b1, W2 [w x w], b2, W3 [w x nout], b3.
"""
import numpy as np


def unpack(p, nin, w, nout):
    sizes = [nin * w, w, w * w, w, w * nout, nout]
    shapes = [(nin, w), (w,), (w, w), (w,), (w, nout), (nout,)]
    out, o = [], 0
    for n, s in zip(sizes, shapes):
        out.append(np.asarray(p[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def nparams(nin, w, nout):
    return nin * w + w + w * w + w + w * nout + nout


def forward(p, x, nin, w, nout):
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, w, nout)
    z1 = x @ W1 + b1
    h1 = z1 / (1 + np.exp(-z1))
    z2 = h1 @ W2 + b2
    h2 = z2 / (1 + np.exp(-z2))
    return h2 @ W3 + b3, (z1, h1, z2, h2)


def loss(p, x, t, mask, nin, w, nout):
    y, _ = forward(p, x, nin, w, nout)
    return float(np.sum(mask * (y - t) ** 2) / max(np.sum(mask), 1.0))


def grad(p, x, t, mask, nin, w, nout):
    W1, b1, W2, b2, W3, b3 = unpack(p, nin, w, nout)
    y, (z1, h1, z2, h2) = forward(p, x, nin, w, nout)
    dy = 2 * mask * (y - t) / max(np.sum(mask), 1.0)
    s2 = 1 / (1 + np.exp(-z2))
    s1 = 1 / (1 + np.exp(-z1))
    gW3, gb3 = h2.T @ dy, dy.sum(0)
    dz2 = (dy @ W3.T) * s2 * (1 + z2 * (1 - s2))
    gW2, gb2 = h1.T @ dz2, dz2.sum(0)
    dz1 = (dz2 @ W2.T) * s1 * (1 + z1 * (1 - s1))
    gW1, gb1 = x.T @ dz1, dz1.sum(0)
    return np.concatenate([a.ravel() for a in (gW1, gb1, gW2, gb2, gW3, gb3)])
