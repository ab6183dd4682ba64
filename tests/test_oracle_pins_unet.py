"""Pins of the warm-start network oracle (oracle/unet.py) against facts fixed by the mathematics:
the circular convolution theorem, adjoint identities, central finite differences of the whole
loss and the closed form of the first Adam step."""
import numpy as np
import pytest

from oracle import unet as U


def _rng(seed=0):
    return np.random.default_rng(seed)


def test_conv3_equals_circular_convolution_by_fft():
    rng = _rng(1)
    Cin, Cout, D, H, W = 3, 4, 4, 6, 5
    x = rng.standard_normal((Cin, D, H, W))
    Wt = rng.standard_normal((27, Cout, Cin))
    b = rng.standard_normal(Cout)
    y = U.conv3(x, Wt, b)
    # y_o(v) = sum_i sum_t W[t,o,i] x_i(v + off_t)  <=>  Y_o(k) = sum_i X_i(k) sum_t W[t,o,i] e^{+2 pi i k.off_t / n}
    X = np.fft.fftn(x, axes=(1, 2, 3))
    kz, ky, kx = np.meshgrid(*[np.fft.fftfreq(n) for n in (D, H, W)], indexing="ij")
    Y = np.zeros((Cout, D, H, W), dtype=complex)
    for t, (dz, dy, dx) in enumerate(U.OFFSETS):
        ph = np.exp(2j * np.pi * (kz * dz + ky * dy + kx * dx))
        Y += np.einsum("oi,izyx->ozyx", Wt[t], X) * ph
    y_fft = np.fft.ifftn(Y, axes=(1, 2, 3)).real + b[:, None, None, None]
    assert np.abs(y - y_fft).max() < 1e-12 * np.abs(y).max()


def test_tap_order_single_impulse():
    # a unit weight on tap t picks x at v + off(t): impulse at the origin lands at -off(t)
    for t, off in enumerate(U.OFFSETS):
        x = np.zeros((1, 4, 4, 4))
        x[0, 0, 0, 0] = 1.0
        Wt = np.zeros((27, 1, 1))
        Wt[t] = 1.0
        y = U.conv3(x, Wt, np.zeros(1))
        idx = tuple((-o) % 4 for o in off)
        assert y[0][idx] == 1.0 and y.sum() == 1.0


def test_adjoints():
    rng = _rng(2)
    x = rng.standard_normal((3, 4, 6, 8))
    Wt = rng.standard_normal((27, 5, 3))
    g = rng.standard_normal((5, 4, 6, 8))
    y = U.conv3(x, Wt, np.zeros(5))
    dx, dW, db = U.conv3_T(x, Wt, g)
    lhs = float((y * g).sum())
    assert abs(lhs - float((x * dx).sum())) < 1e-11 * abs(lhs)       # linear in x
    assert abs(lhs - float((Wt * dW).sum())) < 1e-11 * abs(lhs)      # linear in W
    assert np.allclose(db, g.sum(axis=(1, 2, 3)))
    p = rng.standard_normal((3, 2, 3, 4))
    assert abs(float((U.pool(x) * p).sum()) - float((x * U.pool_T(p)).sum())) < 1e-12
    q = rng.standard_normal((3, 8, 12, 16))
    assert abs(float((U.up(x) * q).sum()) - float((x * U.up_T(q)).sum())) < 1e-11


@pytest.mark.parametrize("widths,n,kind", [((2, 3), 4, "mse"), ((2, 2, 3), 8, "mse"), ((2, 3), 4, "h1")])
def test_gradient_matches_central_differences(widths, n, kind):
    rng = _rng(3)
    specs = U.layer_specs(widths, in_ch=1, n_loads=2)
    theta = U.init_params(specs, seed=5) + 0.05 * rng.standard_normal(U.n_params(specs))
    xs = rng.standard_normal((2, 1, n, n, n))
    ts = rng.standard_normal((2, 2, n, n, n))
    f = lambda th: U.loss_and_grad(th, specs, xs, ts, loss_kind=kind, l2_weight=0.1)
    loss, grad, _ = f(theta)
    h = 1e-6
    idx = rng.choice(theta.size, size=40, replace=False)
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (f(tp)[0] - f(tm)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1e-3, abs(fd)), (i, fd, grad[i])


def test_forward_shapes_and_param_count():
    specs = U.layer_specs((16, 32, 64, 128), in_ch=1, n_loads=3)
    # 3x3x3 layers: 27 Cin Cout + Cout each; head C0 * loads + loads
    manual = (27 * 16 + 16) + (27 * 256 + 16) + (27 * 16 * 32 + 32) + (27 * 32 * 32 + 32) \
        + (27 * 32 * 64 + 64) + (27 * 64 * 64 + 64) + (27 * 64 * 128 + 128) + (27 * 128 * 128 + 128) \
        + (27 * 192 * 64 + 64) + (27 * 64 * 64 + 64) + (27 * 96 * 32 + 32) + (27 * 32 * 32 + 32) \
        + (27 * 48 * 16 + 16) + (27 * 16 * 16 + 16) + (16 * 3 + 3)
    assert U.n_params(specs) == manual
    theta = U.init_params(U.layer_specs((2, 2, 2, 2), 1, 3), seed=0)
    out, _ = U.forward(theta, U.layer_specs((2, 2, 2, 2), 1, 3), np.ones((1, 8, 8, 8)))
    assert out.shape == (3, 8, 8, 8)


def test_translation_equivariance():
    # periodic convolutions, pooling and nearest upsampling commute with shifts by the coarsest stride
    rng = _rng(4)
    specs = U.layer_specs((2, 3, 4), 1, 2)
    theta = U.init_params(specs, seed=1)
    x = rng.standard_normal((1, 8, 8, 8))
    out, _ = U.forward(theta, specs, x)
    xs = np.roll(x, shift=(4, 0, 4), axis=(1, 2, 3))
    outs, _ = U.forward(theta, specs, xs)
    assert np.abs(np.roll(out, shift=(4, 0, 4), axis=(1, 2, 3)) - outs).max() < 1e-12


def test_first_adam_step_closed_form():
    rng = _rng(6)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    new = U.adam_step(th.copy(), g, m, v, step=1, lr=1e-2)
    # m_hat = g, v_hat = g^2 after bias correction
    assert np.allclose(new, th - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_h1_loss_of_a_single_mode():
    # r = cos(2 pi x / n) on one load: each forward difference squared sums to n^3 (2 - 2 cos(2 pi / n)) / 2
    n = 8
    x = np.arange(n)
    r = np.broadcast_to(np.cos(2 * np.pi * x / n), (1, n, n, n)).copy()
    loss, g = U.field_loss(r, count=1, kind="h1", l2_weight=0.0)
    assert abs(loss - n ** 3 * (2 - 2 * np.cos(2 * np.pi / n)) / 2) < 1e-10
    # the gradient is 2 (-Laplacian) r = 2 (2 - 2 cos(2 pi / n)) r for this eigenmode
    assert np.abs(g - 2 * (2 - 2 * np.cos(2 * np.pi / n)) * r).max() < 1e-12
