"""FP64 reference of the filter-strength predictor (test infrastructure only).

The paper (Section 3.2) finds each element's entropy-filter strength by an
iterative root-find.  The learned part predicts that strength as the
root-find's starting guess.  Network (reading; the paper has no network):
inputs x (4 element features) normalised by training-set mean and standard
deviation, h1 = SiLU(W1 x + b1) (32), h2 = SiLU(W2 h1 + b2) (32),
o = W3 h2 + b3, predicted strength z0 = softplus(o).  Loss over a batch:
mean of (log z0 - log z*)^2 against the root-find's zeta*.

Parameter vector layout (float, 1257 entries):
W1[32][4], b1[32], W2[32][32], b2[32], W3[32], b3, mean[4], std[4].
The last 8 entries are the input normalisation (not trained).

Pins (tests/test_oracle_mlp.py): backward against central finite
differences of the forward pass in FP64.
"""
import numpy as np

H = 32
NIN = 4
SIZES = [("W1", (H, NIN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
         ("W3", (H,)), ("b3", (1,)), ("mean", (NIN,)), ("std", (NIN,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)
NTRAIN = NPARAM - 2 * NIN


def unpack(theta):
    out, i = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[i:i + n], np.float64).reshape(shape)
        i += n
    return out


def init(seed=0, mean=None, std=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    theta = np.zeros(NPARAM)
    p = {}
    p["W1"] = rng.normal(0, 1 / np.sqrt(NIN), (H, NIN))
    p["W2"] = rng.normal(0, 1 / np.sqrt(H), (H, H))
    p["W3"] = rng.normal(0, 1 / np.sqrt(H), (H,))
    i = 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        if name in p:
            theta[i:i + n] = p[name].ravel()
        elif name == "mean":
            theta[i:i + n] = 0.0 if mean is None else mean
        elif name == "std":
            theta[i:i + n] = 1.0 if std is None else std
        i += n
    return theta


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def softplus(x):
    return np.logaddexp(0.0, x)


def forward(theta, x):
    """Predicted strength z0 for inputs x (n, 4); returns (z0, cache)."""
    p = unpack(theta)
    xn = (x - p["mean"]) / p["std"]
    a1 = xn @ p["W1"].T + p["b1"]
    h1 = silu(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(a2)
    o = h2 @ p["W3"] + p["b3"][0]
    return softplus(o), (xn, a1, h1, a2, h2, o, p)


def loss_and_grad(theta, x, zstar):
    """Mean squared log error and its gradient w.r.t. every parameter
    (normalisation entries get zero gradient)."""
    z0, (xn, a1, h1, a2, h2, o, p) = forward(theta, x)
    n = len(x)
    r = np.log(z0) - np.log(zstar)
    loss = np.mean(r * r)
    dz0 = 2.0 * r / n / z0
    do = dz0 / (1.0 + np.exp(-o))          # d softplus / d o = sigmoid(o)
    g = {}
    g["W3"] = h2.T @ do
    g["b3"] = np.array([do.sum()])
    dh2 = np.outer(do, p["W3"])
    da2 = dh2 * dsilu(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * dsilu(a1)
    g["W1"] = da1.T @ xn
    g["b1"] = da1.sum(axis=0)
    g["mean"] = np.zeros(NIN)
    g["std"] = np.zeros(NIN)
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES])
    return loss, flat
