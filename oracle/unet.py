"""Oracle, part 3: the periodic 3-D convolutional U-Net of the learned warm start, FP64 on the CPU.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, links or calls this module; only
``tests/`` and ``__graft_entry__.smoke()`` do.  It shares no code with the CUDA kernels.

The paper has no learned component: the warm start is an addition to its method.  A network maps
the conductivity field of a cell to a guess of the fluctuation fields of the unit macroscopic
gradients, and that guess is the initial iterate of the PCG of Sec. 4.1, which still runs to the
same tolerance (the stopping rule of Sec. 6 normalised by the right-hand side, so the guess cannot
loosen it).  This module is the plain definition of that network and of its gradient:

* fields are channel-first arrays ``(C, D, H, W)`` per sample (z, y, x axes), periodic in space;
* conv3: ``y[o, v] = b[o] + sum_t sum_i W[t, o, i] x[i, v + off(t)]`` over the 27 offsets
  ``off(t) = (dz, dy, dx)`` in {-1, 0, 1}^3 with ``t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1)``;
* ReLU after every 3x3x3 convolution; 2x2x2 mean pooling down; nearest-neighbour upsampling and
  channel concatenation (skip first) up; a 1x1x1 linear head to one channel per load;
* loss = mean over samples, loads and voxels of the squared difference to the target, or a
  discrete H^1 seminorm of that difference (``field_loss``);
* gradients by the chain rule, one adjoint per operation (``*_T`` functions);
* Adam (Kingma and Ba, 2015) with bias correction.

Parameters live in a flat FP64 vector in the order of ``layer_specs`` (per 3x3x3 layer the
weight ``W[27, Cout, Cin]`` then the bias ``b[Cout]``; last the head ``Wo[L, C0]``, ``bo[L]``).
Pinned by tests/test_oracle_pins_unet.py: the convolution against the circular convolution
theorem (numpy FFT), every adjoint against ``<A x, y> = <x, A^T y>``, the whole gradient against
central finite differences, and the first Adam step against its closed form.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def layer_specs(widths=(16, 32, 64, 128), in_ch: int = 1, n_loads: int = 3):
    """(name, Cin, Cout) of every 3x3x3 layer in forward order, then ('head', C0, n_loads)."""
    w = list(widths)
    L = len(w)
    specs = [("e0a", in_ch, w[0]), ("e0", w[0], w[0])]
    for l in range(1, L):
        specs += [(f"e{l}a", w[l - 1], w[l]), (f"e{l}", w[l], w[l])]
    for l in range(L - 2, -1, -1):
        specs += [(f"d{l}a", w[l] + w[l + 1], w[l]), (f"d{l}", w[l], w[l])]
    specs.append(("head", w[0], n_loads))
    return specs


def n_params(specs) -> int:
    n = 0
    for name, ci, co in specs:
        n += (co * ci + co) if name == "head" else (27 * co * ci + co)
    return n


def unpack(theta, specs):
    """Views of the flat parameter vector: {name: (W, b)}."""
    out, k = {}, 0
    for name, ci, co in specs:
        nw = co * ci if name == "head" else 27 * co * ci
        W = theta[k:k + nw].reshape((co, ci) if name == "head" else (27, co, ci))
        k += nw
        b = theta[k:k + co]
        k += co
        out[name] = (W, b)
    return out


def init_params(specs, seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, from numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, ci, co in specs:
        fan_in = ci if name == "head" else 27 * ci
        nw = co * ci if name == "head" else 27 * co * ci
        std = np.sqrt(1.0 / fan_in) if name == "head" else np.sqrt(2.0 / fan_in)
        parts.append(rng.standard_normal(nw) * std)
        parts.append(np.zeros(co))
    return np.concatenate(parts)


# ----------------------------------------------------------------------------------------------
# operations and their adjoints (one sample, channel-first)
# ----------------------------------------------------------------------------------------------
def shift(x, off):
    """xs[:, v] = x[:, v + off] with periodic wrap."""
    dz, dy, dx = off
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(1, 2, 3))


def conv3(x, W, b):
    C = x.shape[0]
    y = np.zeros((W.shape[1],) + x.shape[1:])
    for t, off in enumerate(OFFSETS):
        y += np.einsum("oi,izyx->ozyx", W[t], shift(x, off))
    assert W.shape[2] == C
    return y + b[:, None, None, None]


def conv3_T(x, W, g):
    """Adjoints of conv3 at input x for the output gradient g: (dx, dW, db)."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for t, off in enumerate(OFFSETS):
        xs = shift(x, off)
        dW[t] = np.einsum("ozyx,izyx->oi", g, xs)
        back = np.einsum("oi,ozyx->izyx", W[t], g)
        dx += shift(back, tuple(-o for o in off))
    return dx, dW, g.sum(axis=(1, 2, 3))


def relu(x):
    return np.maximum(x, 0.0)


def pool(x):
    C, D, H, W = x.shape
    return x.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def pool_T(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_T(g):
    C, D, H, W = g.shape
    return g.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


def head(x, Wo, bo):
    return np.einsum("lc,czyx->lzyx", Wo, x) + bo[:, None, None, None]


# ----------------------------------------------------------------------------------------------
# network
# ----------------------------------------------------------------------------------------------
def forward(theta, specs, x, act_round=None):
    """Forward pass of one sample x (Cin, D, H, W); returns (output, cache).

    ``act_round`` (optional) is applied to every stored activation, e.g. a rounding to the storage
    precision of another implementation; the mathematics is unchanged when it is None.
    """
    P = unpack(theta, specs)
    q = act_round if act_round is not None else (lambda a: a)
    L = sum(1 for s in specs if s[0].startswith("e") and not s[0].endswith("a"))
    cache = {"x": x}
    h = x
    for l in range(L):
        if l > 0:
            h = q(pool(cache[f"e{l - 1}"]))
            cache[f"p{l}"] = h
        a = q(relu(conv3(h, *P[f"e{l}a"])))
        cache[f"e{l}a"] = a
        cache[f"e{l}"] = q(relu(conv3(a, *P[f"e{l}"])))
    below = cache[f"e{L - 1}"]
    for l in range(L - 2, -1, -1):
        c = np.concatenate([cache[f"e{l}"], up(below)], axis=0)
        cache[f"c{l}"] = c
        a = q(relu(conv3(c, *P[f"d{l}a"])))
        cache[f"d{l}a"] = a
        below = q(relu(conv3(a, *P[f"d{l}"])))
        cache[f"d{l}"] = below
    out = head(below, *P["head"])
    return out, cache


def field_loss(r, count, kind="mse", l2_weight=0.0):
    """Loss of one sample's residual r = output - target (n_loads, D, H, W) and its gradient.

    mse: sum r^2 / count.  h1: (sum over the three axes of the squared forward differences of r,
    periodic, + l2_weight sum r^2) / count -- a discrete H^1 seminorm, the energy of the Laplacian.
    count = number of target values of the whole batch."""
    if kind == "mse":
        return float((r * r).sum()) / count, 2.0 * r / count
    loss, g = l2_weight * float((r * r).sum()), 2.0 * l2_weight * r
    for ax in (1, 2, 3):
        d = np.roll(r, -1, axis=ax) - r
        loss += float((d * d).sum())
        g = g + 2.0 * (2.0 * r - np.roll(r, -1, axis=ax) - np.roll(r, 1, axis=ax))
    return loss / count, g / count


def loss_and_grad(theta, specs, xs, targets, act_round=None, loss_kind="mse", l2_weight=0.0):
    """Loss (field_loss, summed over the batch) and its gradient with respect to theta.

    xs: (B, Cin, D, H, W); targets: (B, n_loads, D, H, W).  Returns (loss, grad, outputs).
    """
    P = unpack(theta, specs)
    grad = np.zeros_like(theta)
    G = unpack(grad, specs)
    L = sum(1 for s in specs if s[0].startswith("e") and not s[0].endswith("a"))
    count = targets.size
    loss = 0.0
    outs = []
    for x, t in zip(xs, targets):
        out, c = forward(theta, specs, x, act_round)
        outs.append(out)
        li, g_out = field_loss(out - t, count, loss_kind, l2_weight)
        loss += li
        Wo, bo = P["head"]
        top = c["d0"] if L > 1 else c["e0"]
        G["head"][0][...] += np.einsum("lzyx,czyx->lc", g_out, top)
        G["head"][1][...] += g_out.sum(axis=(1, 2, 3))
        g = np.einsum("lc,lzyx->czyx", Wo, g_out)

        def through(name, inp, g_post, post):
            """ReLU adjoint at the stored output, then conv3 adjoints; accumulates dW, db."""
            g_pre = g_post * (post > 0)
            dx, dW, db = conv3_T(inp, P[name][0], g_pre)
            G[name][0][...] += dW
            G[name][1][...] += db
            return dx

        skip_grad = {}
        for l in range(0, L - 1):
            g = through(f"d{l}", c[f"d{l}a"], g, c[f"d{l}"])
            g = through(f"d{l}a", c[f"c{l}"], g, c[f"d{l}a"])
            Cs = c[f"e{l}"].shape[0]
            skip_grad[l] = g[:Cs]
            g = up_T(g[Cs:])
        # g is now the gradient at e_{L-1}
        for l in range(L - 1, -1, -1):
            if l < L - 1:
                g = skip_grad[l] + g
            g = through(f"e{l}", c[f"e{l}a"], g, c[f"e{l}"])
            inp = c[f"p{l}"] if l > 0 else c["x"]
            g = through(f"e{l}a", inp, g, c[f"e{l}a"])
            if l > 0:
                g = pool_T(g)
    return loss, grad, np.stack(outs)


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (in place on theta, m, v); step counts from 1."""
    m *= beta1
    m += (1.0 - beta1) * grad
    v *= beta2
    v += (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    theta -= lr * mh / (np.sqrt(vh) + eps)
    return theta
