"""Pins of the surrogate-MLP oracle: finite differences of its FP64 losses,
PyTorch's FP64 autograd of the same network, the BF16 rounding helper,
Adam's first step in closed form and torch.optim.Adam."""
import numpy as np

from oracle import mlp

mlp_in_pad, mlp_in_feat = mlp.IN_PAD, mlp.IN_FEAT


def random_params(seed, scale=0.08):
    g = np.random.default_rng(seed)
    lay = mlp.param_layout()
    p = g.normal(0, scale, lay["total"])
    # padded input columns of W_0 carry no signal
    W0 = p[lay["W"][0]:lay["W"][0] + 256 * mlp_in_pad].reshape(256, mlp_in_pad)
    W0[:, mlp_in_feat:] = 0.0
    return p


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 1e-30, 3.0e38])
    r = mlp.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                       # tie -> even
    assert r[2] == 1.0 + 2 ** -7             # above the tie -> up
    assert r[3] == -2.5
    assert abs(r[4] - 1e-30) / 1e-30 < 2 ** -8
    g = np.random.default_rng(0).normal(0, 3, 1000)
    assert np.max(np.abs(mlp.bf16(g) - g) / np.abs(g)) <= 2 ** -8


def test_trunk_gradient_finite_differences():
    g = np.random.default_rng(1)
    p = random_params(2)
    q = np.concatenate([g.normal(0, 0.05, (3, 21)), g.uniform(0, 10, (3, 1)),
                        g.uniform(-2, 2, (3, 1))], axis=1)
    t = g.normal(0, 1, (3, 1536))
    L, Le, grad = mlp.loss_and_grads(p, q, t, emulate=False)
    lay = mlp.param_layout()
    picks = []
    for l in range(mlp.NLAYER):
        picks += list(g.integers(lay["W"][l], lay["b"][l], 3))
        picks += list(g.integers(lay["b"][l], lay["b"][l] + mlp.layer_out(l), 2))
    # skip padded (dead) input columns of W_0
    picks = [i for i in picks if not (i < lay["b"][0] and (i - lay["W"][0]) % mlp_in_pad >= mlp_in_feat)]
    h = 1e-6
    for i in picks:
        d = np.zeros_like(p)
        d[i] = h
        lp = mlp.loss_and_grads(p + d, q, t, emulate=False)[0]
        lm = mlp.loss_and_grads(p - d, q, t, emulate=False)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-5 * max(1e-3, abs(fd)), i


def test_error_head_gradient_finite_differences():
    g = np.random.default_rng(3)
    p = random_params(4)
    q = np.concatenate([g.normal(0, 0.05, (4, 21)), g.uniform(0, 10, (4, 1)),
                        g.uniform(-2, 2, (4, 1))], axis=1)
    t = g.normal(0, 1, (4, 1536))
    _, Le, grad = mlp.loss_and_grads(p, q, t, emulate=False)
    lay = mlp.param_layout()
    h = 1e-6
    for i in list(g.integers(lay["We"], lay["We"] + 256, 6)) + [lay["be"]]:
        d = np.zeros_like(p)
        d[i] = h
        fd = (mlp.loss_and_grads(p + d, q, t, emulate=False)[1]
              - mlp.loss_and_grads(p - d, q, t, emulate=False)[1]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3])
    p, m, v = mlp.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, lr=0.01, step=1)
    # m_hat = g, v_hat = g^2 -> p = -lr sign(g) (up to eps)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)


def test_gradients_equal_torch_autograd():
    """The oracle's hand-written backward (FP64, no BF16 emulation) equals
    PyTorch's autograd of the same network in FP64: trunk parameters from
    the relative-L2 loss, the error head from its regression loss (the head
    reads the last hidden layer and the relative error as constants)."""
    import torch
    g = np.random.default_rng(11)
    p = random_params(12)
    q = np.concatenate([g.normal(0, 0.05, (5, 21)), g.uniform(0, 10, (5, 1)),
                        g.uniform(-2, 2, (5, 1))], axis=1)
    t = g.normal(0, 1, (5, 1536))
    L, Le, grad = mlp.loss_and_grads(p, q, t, emulate=False)
    pt = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    lay = mlp.param_layout()
    x = torch.tensor(mlp.normalize(q), dtype=torch.float64)
    h = x
    for l in range(mlp.NLAYER):
        W = pt[lay["W"][l]:lay["W"][l] + mlp.layer_out(l) * mlp.layer_in(l)].view(
            mlp.layer_out(l), mlp.layer_in(l))
        b = pt[lay["b"][l]:lay["b"][l] + mlp.layer_out(l)]
        z = h @ W.T + b
        if l < mlp.NLAYER - 1:
            h = torch.nn.functional.silu(z)
        else:
            out = z
    tt = torch.tensor(t, dtype=torch.float64)
    d = out - tt
    n2 = (tt * tt).sum(dim=1)
    e2 = (d * d).sum(dim=1)
    L_t = (e2 / n2).mean()
    rel = torch.sqrt(e2 / n2).detach()
    we = pt[lay["We"]:lay["We"] + mlp.HID]
    e = h.detach() @ we + pt[lay["be"]]
    Le_t = ((e - torch.log10(torch.clamp(rel, min=1e-7))) ** 2).mean()
    (L_t + Le_t).backward()
    gt = pt.grad.numpy()
    assert abs(L_t.item() - L) <= 1e-12 * abs(L) and abs(Le_t.item() - Le) <= 1e-12 * abs(Le)
    live = np.ones_like(p, dtype=bool)
    W0 = live[lay["W"][0]:lay["W"][0] + 256 * mlp_in_pad].reshape(256, mlp_in_pad)
    W0[:, mlp_in_feat:] = False            # padded input columns: zero input, zero gradient
    scale = np.max(np.abs(gt))
    assert np.max(np.abs(grad[live] - gt[live])) <= 1e-10 * scale
    assert np.all(grad[~live] == 0.0) and np.all(gt[~live] == 0.0)


def test_adam_equals_torch_adam():
    """Three Adam steps of the oracle against torch.optim.Adam (FP64, the
    same hyperparameters and gradient sequence)."""
    import torch
    g = np.random.default_rng(5)
    p0 = g.normal(0, 1, 7)
    grads = [g.normal(0, s, 7) for s in (1.0, 0.1, 3.0)]
    p, m, v = p0.copy(), np.zeros(7), np.zeros(7)
    pt = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    for k, gk in enumerate(grads, start=1):
        p, m, v = mlp.adam(p, m, v, gk, lr=3e-3, step=k)
        opt.zero_grad()
        pt.grad = torch.tensor(gk, dtype=torch.float64)
        opt.step()
    assert np.allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)
