"""FP64 reference of the linewidth surrogate network (no counterpart in the paper's equations;
used to check the GPU training kernels).

Network: x_in = (log(max(x, 1e-12)) - mu_x) / sd_x, hidden layers h = silu(h W + b),
output y_hat = h W + b; loss = mean((y_hat - (log(gamma) - mu_y) / sd_y)^2).  The parameter
vector of one member is laid out layer by layer as W [in][out] (row-major) then b [out].
"""
import numpy as np


def layer_shapes(n_in, width, depth):
    shapes = []
    for l in range(depth + 1):
        i = n_in if l == 0 else width
        o = 1 if l == depth else width
        shapes.append((i, o))
    return shapes


def unpack(params, n_in, width, depth):
    out, off = [], 0
    for i, o in layer_shapes(n_in, width, depth):
        W = params[off:off + i * o].reshape(i, o)
        off += i * o
        b = params[off:off + o]
        off += o
        out.append((W, b))
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def loss_and_grad(params, norm, X, y, n_in, width, depth):
    """Loss and gradient (same layout as params) of one member, in float64."""
    params = np.asarray(params, dtype=np.float64)
    mu_x, sd_x = norm[:n_in], norm[n_in:2 * n_in]
    mu_y, sd_y = norm[2 * n_in], norm[2 * n_in + 1]
    h = (np.log(np.maximum(X, 1e-12)) - mu_x) / sd_x
    t = (np.log(y) - mu_y) / sd_y
    layers = unpack(params, n_in, width, depth)
    acts, pres = [h], []
    for l, (W, b) in enumerate(layers):
        z = acts[-1] @ W + b
        pres.append(z)
        acts.append(silu(z) if l < depth else z)
    yhat = acts[-1][:, 0]
    r = yhat - t
    loss = float(np.mean(r * r))
    d = (2.0 * r / X.shape[0])[:, None]
    grads = [None] * (depth + 1)
    for l in range(depth, -1, -1):
        if l < depth:
            d = d * silu_grad(pres[l])
        W, _ = layers[l]
        grads[l] = (acts[l].T @ d, d.sum(axis=0))
        d = d @ W.T
    g = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, g


def predict(params, norm, X, n_in, width, depth):
    mu_x, sd_x = norm[:n_in], norm[n_in:2 * n_in]
    mu_y, sd_y = norm[2 * n_in], norm[2 * n_in + 1]
    h = (np.log(np.maximum(X, 1e-12)) - mu_x) / sd_x
    for l, (W, b) in enumerate(unpack(np.asarray(params, np.float64), n_in, width, depth)):
        h = h @ W + b
        if l < depth:
            h = silu(h)
    return h[:, 0] * sd_y + mu_y
