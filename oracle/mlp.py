"""Surrogate MLP oracle (FP64, test infrastructure only).

The network is the one the library trains: x = (c_1..c_21 / 0.05,
depth / 5 - 1, z / 2, Fourier features of the last two; see ``normalize``)
padded to 120 inputs -> 4 hidden layers of 256 with SiLU -> 1536 outputs (complex I_0, I_1, I_2 at 256 radii), plus an error head
256 -> 1 on the last hidden layer that regresses log10 of the relative L2
error of the output.  Losses (per batch of B samples):

    L   = (1/B) sum_b |out_b - t_b|^2 / |t_b|^2
    L_e = (1/B) sum_b (e_b - log10(max(rel_err_b, 1e-7)))^2   (head only)

``emulate=True`` rounds to BF16 exactly where the GPU kernels store BF16
(inputs, weight copies, pre-activations, activations, output and hidden
gradients), so GPU results can be compared element by element; with
``emulate=False`` everything stays in FP64 (the finite-difference pins use
that form).  The surrogate is not part of the paper, so its agreement with
the paper is "parity unpinned"; finite differences and PyTorch's FP64
autograd pin the gradients, torch.optim.Adam the update.
"""
import numpy as np

IN, HID, OUT, NLAYER = 23, 256, 1536, 5
NFREQ = 24
IN_FEAT = IN + 4 * NFREQ      # 119 network inputs
IN_PAD = 120


def layer_in(l):
    return IN_PAD if l == 0 else HID


def layer_out(l):
    return OUT if l == NLAYER - 1 else HID


def param_layout():
    """Offsets of the packed parameter vector (same packing as the library)."""
    o, W, b = 0, [], []
    for l in range(NLAYER):
        W.append(o)
        o += layer_out(l) * layer_in(l)
        b.append(o)
        o += layer_out(l)
    We = o
    o += HID
    be = o
    o += 1
    return dict(W=W, b=b, We=We, be=be, total=o)


def unpack(p):
    L = param_layout()
    Ws = [p[L["W"][l]:L["W"][l] + layer_out(l) * layer_in(l)].reshape(layer_out(l), layer_in(l))
          for l in range(NLAYER)]
    bs = [p[L["b"][l]:L["b"][l] + layer_out(l)] for l in range(NLAYER)]
    return Ws, bs, p[L["We"]:L["We"] + HID], p[L["be"]]


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def normalize(query):
    """Network input: c / 0.05, d = depth / 5 - 1, u = z / 2, then for
    k < NFREQ (sin, cos)(2 pi f_k u) and (sin, cos)(2 pi g_k d) with the
    geometric ladders f_k = 0.5 * 16^(k/(NFREQ-1)), g_k = 0.5 * 40^(k/(NFREQ-1))
    (Fourier-feature encoding of the two oscillatory coordinates)."""
    q = np.asarray(query, dtype=np.float64)
    x = np.zeros((q.shape[0], IN_PAD))
    x[:, :21] = q[:, :21] / 0.05
    d = q[:, 21] / 5.0 - 1.0
    u = q[:, 22] / 2.0
    x[:, 21] = d
    x[:, 22] = u
    for k in range(NFREQ):
        f = 0.5 * 16.0 ** (k / (NFREQ - 1))
        gk = 0.5 * 40.0 ** (k / (NFREQ - 1))
        c = IN + 4 * k
        x[:, c] = np.sin(2 * np.pi * f * u)
        x[:, c + 1] = np.cos(2 * np.pi * f * u)
        x[:, c + 2] = np.sin(2 * np.pi * gk * d)
        x[:, c + 3] = np.cos(2 * np.pi * gk * d)
    return x


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(p, query, emulate=True):
    r = bf16 if emulate else (lambda a: np.asarray(a, dtype=np.float64))
    Ws, bs, we, be = unpack(np.asarray(p, dtype=np.float64))
    x = r(normalize(query))
    acts, zs = [x], []
    for l in range(NLAYER - 1):
        z = r(acts[-1] @ r(Ws[l]).T + bs[l])
        zs.append(z)
        acts.append(r(z * sigmoid(z)))
    out = acts[-1] @ r(Ws[-1]).T + bs[-1]
    e = acts[-1] @ we + be
    return dict(acts=acts, zs=zs, out=out, err=e)


def loss_and_grads(p, query, target, emulate=True):
    """Returns (L, L_e, packed gradient)."""
    r = bf16 if emulate else (lambda a: np.asarray(a, dtype=np.float64))
    p = np.asarray(p, dtype=np.float64)
    Ws, bs, we, be = unpack(p)
    f = forward(p, query, emulate)
    t = np.asarray(target, dtype=np.float64)
    B = t.shape[0]
    d = f["out"] - t
    n2 = np.maximum(np.sum(t * t, axis=1), 1e-30)
    e2 = np.sum(d * d, axis=1)
    L = float(np.sum(e2 / n2) / B)
    rel = np.sqrt(e2 / n2)
    g = r(2.0 / B * d / n2[:, None])
    lay = param_layout()
    grads = np.zeros(lay["total"])
    acts, zs = f["acts"], f["zs"]
    for l in range(NLAYER - 1, -1, -1):
        dW = g.T @ acts[l]
        grads[lay["W"][l]:lay["W"][l] + dW.size] = dW.ravel()
        grads[lay["b"][l]:lay["b"][l] + layer_out(l)] = g.sum(axis=0)
        if l == 0:
            break
        dy = g @ r(Ws[l])
        z = zs[l - 1]
        s = sigmoid(z)
        g = r(dy * s * (1.0 + z * (1.0 - s)))
    res = f["err"] - np.log10(np.maximum(rel, 1e-7))
    Le = float(np.sum(res * res) / B)
    grads[lay["We"]:lay["We"] + HID] = 2.0 / B * (res @ acts[-1])
    grads[lay["be"]] = 2.0 / B * np.sum(res)
    return L, Le, grads


def adam(p, m, v, g, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
