"""FP64 CPU oracle of the warm-start network for the anelastic projection:
a three-level 3D U-Net.  Test infrastructure only: the CUDA library never
imports it.

Architecture (channels 16 / 32 / 64, 3x3x3 convolutions with zero padding,
ReLU after every convolution but the last):

    x (2: rhs / s, alpha)
    e1 = conv(conv(x; 2->16); 16->16)                     full resolution
    e2 = conv(conv(pool(e1); 16->32); 32->32)             1/2
    bt = conv(conv(pool(e2); 32->64); 64->64)             1/4
    d2 = conv(conv([up(bt), e2]; 96->32); 32->32)         1/2
    d1 = conv(conv([up(d2), e1]; 48->16); 16->16)         full
    y  = conv1x1(d1; 16->1)                               (no ReLU)

pool = 2x2x2 average, up = 2x nearest, [a, b] = channel concatenation.
Parameters are one flat vector: per layer, weights [cout][cin][k][k][k] then
biases [cout], layers in the order above.  Loss: half the masked mean square
error, 0.5 sum(mask (y - t)^2) / sum(mask).  The backward pass is written out
layer by layer from the chain rule; tests check it against central finite
differences.  Arrays are (channels, nz, ny, nx).
"""
import numpy as np

# (cin, cout, kernel size)
LAYERS = [(2, 16, 3), (16, 16, 3), (16, 32, 3), (32, 32, 3), (32, 64, 3), (64, 64, 3),
          (96, 32, 3), (32, 32, 3), (48, 16, 3), (16, 16, 3), (16, 1, 1)]


def num_params():
    return sum(co * ci * k ** 3 + co for ci, co, k in LAYERS)


def unpack(p):
    """List of (W, b) views of the flat parameter vector."""
    out, o = [], 0
    for ci, co, k in LAYERS:
        n = co * ci * k ** 3
        W = p[o:o + n].reshape(co, ci, k, k, k)
        o += n
        b = p[o:o + co]
        o += co
        out.append((W, b))
    assert o == p.size
    return out


def init_params(seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co, k in LAYERS:
        parts.append(rng.standard_normal(co * ci * k ** 3) * np.sqrt(2.0 / (ci * k ** 3)))
        parts.append(np.zeros(co))
    return np.concatenate(parts)


# ---- layers ---------------------------------------------------------------

def conv(x, W, b):
    """y[o, v] = b[o] + sum_{i, a} W[o, i, a] x[i, v + a - r] (zero outside)."""
    k = W.shape[2]
    r = k // 2
    C, D, H, Wd = x.shape
    xp = np.zeros((C, D + 2 * r, H + 2 * r, Wd + 2 * r))
    xp[:, r:r + D, r:r + H, r:r + Wd] = x
    y = np.zeros((W.shape[0], D, H, Wd)) + b[:, None, None, None]
    for a in range(k):
        for bb in range(k):
            for c in range(k):
                y += np.einsum("oi,idhw->odhw", W[:, :, a, bb, c], xp[:, a:a + D, bb:bb + H, c:c + Wd])
    return y


def conv_backward(x, W, dy):
    """Gradients (dx, dW, db) of conv for the output gradient dy."""
    k = W.shape[2]
    r = k // 2
    C, D, H, Wd = x.shape
    xp = np.zeros((C, D + 2 * r, H + 2 * r, Wd + 2 * r))
    xp[:, r:r + D, r:r + H, r:r + Wd] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for a in range(k):
        for bb in range(k):
            for c in range(k):
                sl = (slice(None), slice(a, a + D), slice(bb, bb + H), slice(c, c + Wd))
                dxp[sl] += np.einsum("oi,odhw->idhw", W[:, :, a, bb, c], dy)
                dW[:, :, a, bb, c] = np.einsum("odhw,idhw->oi", dy, xp[sl])
    return dxp[:, r:r + D, r:r + H, r:r + Wd], dW, dy.sum(axis=(1, 2, 3))


def pool(x):
    C, D, H, W = x.shape
    return x.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def pool_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up_backward(dy):
    C, D, H, W = dy.shape
    return dy.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


def relu(x):
    return np.maximum(x, 0.0)


# ---- network ----------------------------------------------------------------

def forward(p, x):
    """Output (1, nz, ny, nx) and the activations the backward pass needs."""
    P = unpack(p)
    a = {}
    a["x"] = x
    a["e1a"] = relu(conv(x, *P[0]))
    a["e1"] = relu(conv(a["e1a"], *P[1]))
    a["p1"] = pool(a["e1"])
    a["e2a"] = relu(conv(a["p1"], *P[2]))
    a["e2"] = relu(conv(a["e2a"], *P[3]))
    a["p2"] = pool(a["e2"])
    a["ba"] = relu(conv(a["p2"], *P[4]))
    a["bt"] = relu(conv(a["ba"], *P[5]))
    a["c2"] = np.concatenate([up(a["bt"]), a["e2"]])
    a["d2a"] = relu(conv(a["c2"], *P[6]))
    a["d2"] = relu(conv(a["d2a"], *P[7]))
    a["c1"] = np.concatenate([up(a["d2"]), a["e1"]])
    a["d1a"] = relu(conv(a["c1"], *P[8]))
    a["d1"] = relu(conv(a["d1a"], *P[9]))
    y = conv(a["d1"], *P[10])
    return y, a


def loss(y, t, mask):
    n = mask.sum()
    e = (y - t) * mask
    return 0.5 * float(np.sum(e * e)) / n, e / n


def backward(p, a, dy):
    """Flat parameter gradient and the input gradient for the output
    gradient dy."""
    P = unpack(p)
    g = [None] * len(LAYERS)

    def step(name_in, layer, d_out, post):
        # post: the layer's ReLU output (None for the linear head)
        if post is not None:
            d_out = d_out * (post > 0)
        dx, dW, db = conv_backward(a[name_in], P[layer][0], d_out)
        g[layer] = (dW, db)
        return dx

    d = step("d1", 10, dy, None)
    d = step("d1a", 9, d, a["d1"])
    dc1 = step("c1", 8, d, a["d1a"])
    n_up1 = a["d2"].shape[0]
    d = up_backward(dc1[:n_up1])
    de1 = dc1[n_up1:]
    d = step("d2a", 7, d, a["d2"])
    dc2 = step("c2", 6, d, a["d2a"])
    n_up2 = a["bt"].shape[0]
    d = up_backward(dc2[:n_up2])
    de2 = dc2[n_up2:]
    d = step("ba", 5, d, a["bt"])
    d = step("p2", 4, d, a["ba"])
    de2 = de2 + pool_backward(d)
    d = step("e2a", 3, de2, a["e2"])
    d = step("p1", 2, d, a["e2a"])
    de1 = de1 + pool_backward(d)
    d = step("e1a", 1, de1, a["e1"])
    dx = step("x", 0, d, a["e1a"])
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in g])
    return flat, dx


def adam(p, m, v, grad, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t = 1, 2, ...): returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
