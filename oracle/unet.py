"""Float64 reference of the learned warm start / preconditioner network.

The paper has no learned component; this network is the one the GPU path
trains and runs: a 4-level U-Net on NHWC images (batch, height, width,
channels), written layer by layer with the backward pass derived by hand:

  encoder l = 0..3:  e_l = relu(conv3(relu(conv3(in_l, A_l)), B_l)),
                     in_0 = the input, in_l = avgpool2(e_{l-1})
  decoder l = 2..0:  d_l = relu(conv3(relu(conv3(cat(up2(d_{l+1}), e_l), C_l)), D_l)),
                     d_3 = e_3
  output:            y = conv1(d_0, O)

conv3: 3x3 convolution with zero padding and bias, weights [3, 3, Cin, Cout]
(cross-correlation: out[y, x] = sum_{dy,dx} in[y+dy-1, x+dx-1] W[dy, dx]);
avgpool2: mean over 2x2 blocks; up2: nearest-neighbour upsampling; cat:
channel concatenation (upsampled first).  Parameter layout and order are
given by `param_shapes`.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def conv3_fwd(x, W, b):
    B, H, Wd, Ci = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    out = np.zeros((B, H, Wd, W.shape[3])) + b
    for dy in range(3):
        for dx in range(3):
            out += xp[:, dy:dy + H, dx:dx + Wd, :] @ W[dy, dx]
    return out


def conv3_bwd(x, W, g):
    """Gradients of sum(g * conv3_fwd(x, W, b)) w.r.t. x, W, b."""
    B, H, Wd, Ci = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, Ci))
    xp[:, 1:-1, 1:-1, :] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, dy:dy + H, dx:dx + Wd, :]
            gW[dy, dx] = np.einsum("bhwi,bhwo->io", patch, g)
            gxp[:, dy:dy + H, dx:dx + Wd, :] += g @ W[dy, dx].T
    return gxp[:, 1:-1, 1:-1, :], gW, g.sum(axis=(0, 1, 2))


def conv1_fwd(x, W, b):
    return x @ W + b


def conv1_bwd(x, W, g):
    return g @ W.T, np.einsum("bhwi,bhwo->io", x, g), g.sum(axis=(0, 1, 2))


def pool_fwd(x):
    B, H, Wd, C = x.shape
    return x.reshape(B, H // 2, 2, Wd // 2, 2, C).mean(axis=(2, 4))


def pool_bwd(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def up_fwd(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(g):
    B, H, Wd, C = g.shape
    return g.reshape(B, H // 2, 2, Wd // 2, 2, C).sum(axis=(2, 4))


def param_shapes(cin: int = 3, ch=(16, 32, 48, 64)):
    """[(name, shape)] in storage order."""
    shapes = []
    prev = cin
    for l, c in enumerate(ch):
        shapes += [(f"A{l}", (3, 3, prev, c)), (f"a{l}", (c,)), (f"B{l}", (3, 3, c, c)), (f"b{l}", (c,))]
        prev = c
    for l in (2, 1, 0):
        cc = ch[l + 1] + ch[l]
        shapes += [(f"C{l}", (3, 3, cc, ch[l])), (f"c{l}", (ch[l],)), (f"D{l}", (3, 3, ch[l], ch[l])),
                   (f"d{l}", (ch[l],))]
    shapes += [("O", (ch[0], 1)), ("o", (1,))]
    return shapes


def init_params(rng, cin: int = 3, ch=(16, 32, 48, 64)):
    """He-normal weights, zero biases."""
    P = {}
    for name, shp in param_shapes(cin, ch):
        if len(shp) == 1:
            P[name] = np.zeros(shp)
        else:
            fan_in = int(np.prod(shp[:-1]))
            P[name] = rng.standard_normal(shp) * np.sqrt(2.0 / fan_in)
    return P


def forward(P, x, ch=(16, 32, 48, 64), rnd=None):
    """Returns (y, cache).  rnd, if given, is applied to the input and to
    every stored activation (after each conv + relu and each pooling), to
    evaluate the network at the storage precision of an implementation."""
    r = rnd if rnd is not None else (lambda a: a)
    cache = {}
    h = r(x)
    enc = []
    for l in range(4):
        if l > 0:
            h = r(pool_fwd(enc[-1]))
        cache[f"in{l}"] = h
        z1 = conv3_fwd(h, P[f"A{l}"], P[f"a{l}"])
        a1 = r(np.maximum(z1, 0.0))
        z2 = conv3_fwd(a1, P[f"B{l}"], P[f"b{l}"])
        e = r(np.maximum(z2, 0.0))
        cache[f"ez1{l}"], cache[f"ea1{l}"], cache[f"ez2{l}"] = z1, a1, z2
        enc.append(e)
    d = enc[3]
    for l in (2, 1, 0):
        u = up_fwd(d)
        cat = np.concatenate([u, enc[l]], axis=3)
        z1 = conv3_fwd(cat, P[f"C{l}"], P[f"c{l}"])
        a1 = r(np.maximum(z1, 0.0))
        z2 = conv3_fwd(a1, P[f"D{l}"], P[f"d{l}"])
        d = r(np.maximum(z2, 0.0))
        cache[f"cat{l}"], cache[f"dz1{l}"], cache[f"da1{l}"], cache[f"dz2{l}"] = cat, z1, a1, z2
    cache["enc"] = enc
    cache["d0"] = d
    y = conv1_fwd(d, P["O"], P["o"])
    return y, cache


def backward(P, cache, gy, ch=(16, 32, 48, 64)):
    """Gradients of sum(gy * y) w.r.t. the parameters (dict) and the input."""
    G = {}
    gd, G["O"], G["o"] = conv1_bwd(cache["d0"], P["O"], gy)
    enc = cache["enc"]
    genc = [np.zeros_like(e) for e in enc]
    # decoders in reverse order of the forward pass: d_0, d_1, d_2
    for l in (0, 1, 2):
        g2 = gd * (cache[f"dz2{l}"] > 0)
        ga1, G[f"D{l}"], G[f"d{l}"] = conv3_bwd(cache[f"da1{l}"], P[f"D{l}"], g2)
        g1 = ga1 * (cache[f"dz1{l}"] > 0)
        gcat, G[f"C{l}"], G[f"c{l}"] = conv3_bwd(cache[f"cat{l}"], P[f"C{l}"], g1)
        cu = ch[l + 1]
        genc[l] += gcat[..., cu:]
        gd = up_bwd(gcat[..., :cu])          # gradient of d_{l+1}
    genc[3] += gd                            # d_3 = e_3
    gx = None
    for l in (3, 2, 1, 0):
        g2 = genc[l] * (cache[f"ez2{l}"] > 0)
        ga1, G[f"B{l}"], G[f"b{l}"] = conv3_bwd(cache[f"ea1{l}"], P[f"B{l}"], g2)
        g1 = ga1 * (cache[f"ez1{l}"] > 0)
        gin, G[f"A{l}"], G[f"a{l}"] = conv3_bwd(cache[f"in{l}"], P[f"A{l}"], g1)
        if l > 0:
            genc[l - 1] += pool_bwd(gin)
        else:
            gx = gin
    return G, gx


def mse_loss(y, t):
    """mean((y - t)^2) and its gradient w.r.t. y."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def features(v, rho, ct, hz):
    """Network input of a 2D field (rows z, columns x) and the output scale:
    ch0 = v/rms(v), ch1 = log(rho/mean rho), ch2 = log(1/(c~ rho hz^2))/10;
    s = rms(v) / (mean c~ + pi^2 mean(1/rho)).  Returns ([1, H, W, 3], s)."""
    v = np.asarray(v, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    ct = np.asarray(ct, dtype=np.float64)
    rms = np.sqrt(np.mean(v * v))
    x = np.stack([v / rms, np.log(rho / rho.mean()), np.log(1.0 / (ct * rho * hz * hz)) / 10.0], axis=-1)
    s = rms / (ct.mean() + np.pi ** 2 * np.mean(1.0 / rho))
    return x[None], s


def flat_params(P, cin=3, ch=(16, 32, 48, 64)):
    return np.concatenate([P[n].ravel() for n, _ in param_shapes(cin, ch)])


def unflat_params(a, cin=3, ch=(16, 32, 48, 64)):
    P, o = {}, 0
    for n, shp in param_shapes(cin, ch):
        k = int(np.prod(shp))
        P[n] = np.asarray(a[o:o + k], dtype=np.float64).reshape(shp)
        o += k
    return P
