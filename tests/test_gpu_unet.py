"""Warm-start network on the GPU against the FP64 oracle (oracle/unet.py): the tcgen05 convolution and
weight-gradient kernels element by element, the whole network's loss and gradient, one Adam step,
and what a trained network gains as a PCG initial guess."""
import numpy as np
import pytest

from oracle import unet as U

pytestmark = pytest.mark.gpu


def _bf16_round(a):
    """Round-to-nearest-even to bfloat16, returned as float64 (the values the GPU stores)."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _to_bf16_tensor(a, torch):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).cuda()


CONV_CASES = [
    # (B, D, H, W, Cin, Cout)
    (2, 4, 16, 8, 16, 16),
    (1, 8, 8, 8, 48, 32),      # H < 16: tile rows wrap
    (1, 3, 20, 12, 32, 64),    # ragged tiles in y and x
    (1, 2, 2, 2, 192, 64),     # tiny grid, deep K
    (2, 4, 8, 16, 64, 128),    # two N tiles
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_conv3_forward_matches_oracle(case):
    import torch
    from paper_2203_02962_gb300 import fehom
    B, D, H, W, Cin, Cout = case
    rng = np.random.default_rng(sum(case))
    x = _bf16_round(rng.standard_normal((B, D, H, W, Cin)))
    w = _bf16_round(rng.standard_normal((27, Cout, Cin)) / np.sqrt(27 * Cin))
    bias = rng.standard_normal(Cout).astype(np.float32)
    for relu in (False, True):
        y = fehom.conv3_bf16(_to_bf16_tensor(x, torch), _to_bf16_tensor(w, torch),
                             torch.tensor(bias).cuda(), relu=relu).cpu().numpy().astype(np.float64)
        for b in range(B):
            ref = U.conv3(np.moveaxis(x[b], -1, 0), w, bias.astype(np.float64))
            if relu:
                ref = U.relu(ref)
            ref = np.moveaxis(ref, 0, -1)
            # FP32 accumulation of 27 Cin exact BF16 products
            bound = 1e-5 * (np.abs(np.moveaxis(x[b], -1, 0)).max() * np.abs(w).sum(axis=(0, 2)).max() + 1.0)
            assert np.abs(y[b] - ref).max() <= bound, (case, relu, np.abs(y[b] - ref).max(), bound)


@pytest.mark.parametrize("case", [c for c in CONV_CASES if c[5] <= 128])
def test_conv3_weight_gradient_matches_oracle(case):
    import torch
    from paper_2203_02962_gb300 import fehom
    B, D, H, W, Cin, Cout = case
    rng = np.random.default_rng(7 + sum(case))
    x = _bf16_round(rng.standard_normal((B, D, H, W, Cin)))
    dy = _bf16_round(rng.standard_normal((B, D, H, W, Cout)))
    dw = fehom.conv3_wgrad_bf16(_to_bf16_tensor(x, torch), _to_bf16_tensor(dy, torch)).cpu().numpy()
    ref = np.zeros((27, Cout, Cin))
    for b in range(B):
        ref += U.conv3_T(np.moveaxis(x[b], -1, 0), np.zeros((27, Cout, Cin)), np.moveaxis(dy[b], -1, 0))[1]
    scale = np.sqrt(B * D * H * W) * 4.0
    assert np.abs(dw - ref).max() <= 2e-5 * scale, (case, np.abs(dw - ref).max())


def _net_case(n=16, widths=(16, 32, 64, 128), B=2, seed=0):
    rng = np.random.default_rng(seed)
    specs = U.layer_specs(widths, 1, 3)
    theta = U.init_params(specs, seed=seed)
    # nonzero biases so that every bias gradient path is exercised
    P = U.unpack(theta, specs)
    for name, (Wt, b) in P.items():
        b[...] = 0.05 * rng.standard_normal(b.shape)
    theta = theta.astype(np.float32).astype(np.float64)
    ids = (rng.random((B, n, n, n)) < 0.3).astype(np.uint8)
    feat = np.stack([[0.0, rng.uniform(0.3, 1.0)] for _ in range(B)]).astype(np.float32)
    target = rng.standard_normal((B, 3, n, n, n)) * 0.02
    return specs, theta, ids, feat, target


def _gpu_rounded_theta(specs, theta):
    """The weights the kernels multiply: BF16 for the tensor-core layers, FP32 for the first layer and head."""
    th = theta.copy()
    P = U.unpack(th, specs)
    for name, (Wt, b) in P.items():
        if name not in ("e0a", "head"):
            Wt[...] = _bf16_round(Wt)
    return th


@pytest.mark.parametrize("kind", ["mse", "h1"])
def test_unet_loss_and_gradient_match_oracle(kind):
    import torch
    from paper_2203_02962_gb300 import fehom
    n, widths, B = 16, (16, 32, 64, 128), 2
    specs, theta, ids, feat, target = _net_case(n, widths, B)
    out_scale = 0.05
    net = fehom.UNet(n, widths, n_phases=2, n_out=3, max_batch=B)
    net.set_loss(kind, l2_weight=0.1)
    assert net.n_params == U.n_params(specs)
    net.set_params(theta)
    ids_t = torch.tensor(ids.reshape(B, -1)).cuda()
    feat_t = torch.tensor(feat).cuda()
    tgt_t = torch.tensor(target.reshape(B, 3, -1)).cuda()
    loss, g = net.loss_grad(ids_t, feat_t, tgt_t, out_scale)
    xs = feat[np.arange(B)[:, None, None, None], ids].astype(np.float64)[:, None]
    ref_loss, ref_g, _ = U.loss_and_grad(_gpu_rounded_theta(specs, theta), specs, xs, target / out_scale,
                                         act_round=_bf16_round, loss_kind=kind, l2_weight=0.1)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss, (loss, ref_loss)
    G, RG = U.unpack(g.astype(np.float64), specs), U.unpack(ref_g, specs)
    for name in G:
        err = np.linalg.norm(G[name][0] - RG[name][0]) / np.linalg.norm(RG[name][0])
        assert err < 3e-2, (name, err)
    # BF16 storage of activations and gradients; the H1 output gradient (a discrete Laplacian of the
    # residual) amplifies the rounding of the stored fields, hence the looser bound for it
    assert np.linalg.norm(g - ref_g) <= (1e-2 if kind == "mse" else 2e-2) * np.linalg.norm(ref_g)
    # predictions = out_scale * network output
    x0 = net.predict(ids_t, feat_t, out_scale).cpu().numpy()
    out, _ = U.forward(_gpu_rounded_theta(specs, theta), specs, xs[0], act_round=_bf16_round)
    assert np.abs(x0[0].reshape(out.shape) - out_scale * out).max() <= 1e-2 * out_scale * np.abs(out).max()
    net.close()


def test_unet_adam_step_matches_oracle():
    import torch
    from paper_2203_02962_gb300 import fehom
    n, widths, B = 8, (16, 32), 2
    specs, theta, ids, feat, target = _net_case(n, widths, B, seed=3)
    net = fehom.UNet(n, widths, n_phases=2, n_out=3, max_batch=B)
    net.set_params(theta)
    ids_t = torch.tensor(ids.reshape(B, -1)).cuda()
    feat_t = torch.tensor(feat).cuda()
    tgt_t = torch.tensor(target.reshape(B, 3, -1)).cuda()
    _, g = net.loss_grad(ids_t, feat_t, tgt_t, 0.05)
    net.train_step(ids_t, feat_t, tgt_t, 0.05, lr=1e-3)
    new = net.get_params().astype(np.float64)
    ref = U.adam_step(theta.copy(), g.astype(np.float64), np.zeros_like(theta), np.zeros_like(theta), 1, 1e-3)
    assert np.abs(new - ref).max() <= 1e-6
    net.close()


def test_trained_network_reduces_the_initial_energy_error():
    """A network trained briefly on solver-generated 32^3 samples: the training loss falls, and its
    Galerkin-scaled guess is closer to the solution in the energy norm than the zero guess.  PCG
    from the guess still converges to the same tolerance; its iteration count is reported by the
    experiment, not asserted (from a guess whose error is spread over the whole spectrum PCG can need
    more iterations than from zero, whose residual b excites few modes)."""
    from paper_2203_02962_gb300 import warmstart
    res = warmstart.experiment(n=32, n_train=64, n_test=8, steps=400, batch=8, seed=0, widths=(16, 32, 64, 128))
    assert res["train_loss_last"] < 0.5 * res["train_loss_first"], res
    assert res["warm"]["energy_error_rel_mean"] < 0.9, res
    assert res["warm"]["all_converged"] and res["cold"]["all_converged"]
