"""FP64 restatement of the learned-ratio network and its features (TEST INFRASTRUCTURE).

Only tests may import this module.  The network is written from its
definition: xn = (x - mean) / std; z1 = xn W1 + b1; h = GELU(z1) with
GELU(z) = z * Phi(z) (Phi the standard normal CDF, via erf); y = h W2 + b2;
loss = mean over samples and outputs of (y - t)^2.  Backward follows the
chain rule term by term.  The features are per subspace the two smallest
half-subspace centroid distances and log(1 + size of the cell of the two
nearest centroids), taken from the query oracle's own distance tables.
"""
import math

import numpy as np
from scipy.special import erf

from . import suco_oracle as so


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(x, mean, std, W1, b1, W2, b2):
    x = np.asarray(x, np.float64)
    xn = (x - mean) / std
    z1 = xn @ W1 + b1
    h = gelu(z1)
    y = h @ W2 + b2
    return dict(xn=xn, z1=z1, h=h, y=y)


def loss_and_grads(x, t, mean, std, W1, b1, W2, b2):
    f = forward(x, mean, std, W1, b1, W2, b2)
    B = x.shape[0]
    e = f["y"] - t
    loss = float(np.sum(e * e) / (2.0 * B))
    dy = 2.0 * e / (2.0 * B)
    dW2 = f["h"].T @ dy
    db2 = dy.sum(axis=0)
    dh = dy @ W2.T
    dz1 = dh * gelu_grad(f["z1"])
    dW1 = f["xn"].T @ dz1
    db1 = dz1.sum(axis=0)
    return loss, dict(W1=dW1, b1=db1, W2=dW2, b2=db2, dy=dy, dz1=dz1), f


def features(X, index, q):
    """3*Ns features of one query, from the oracle's FP32 ranking distances."""
    Ns, sk = index["Ns"], index["sqrtK"]
    o = so.query(X, index, q, 1, 1, 1, rank_precision=1, debug=True)
    dt = o["dtab"]  # [Ns][2][sk]
    out = np.empty(3 * Ns, np.float64)
    for i in range(Ns):
        a1 = int(np.argmin(dt[i, 0]))
        a2 = int(np.argmin(dt[i, 1]))
        out[2 * i] = dt[i, 0, a1]
        out[2 * i + 1] = dt[i, 1, a2]
        co = index["cell_off"][i]
        cell = a1 * sk + a2
        out[2 * Ns + i] = math.log1p(float(co[cell + 1] - co[cell]))
    return out


def adamw(p, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    upd = (m / (1 - beta1 ** step)) / (np.sqrt(v / (1 - beta2 ** step)) + eps)
    p = p - lr * (upd + wd * p)
    return p, m, v
