"""FP64 reference of the learned-preconditioner network (test infrastructure).

A two-hidden-layer perceptron 16 -> 64 -> 64 -> 4 with tanh activations, inputs
standardised by (mu, sd) and outputs scaled by os, trained on the mean squared error of
the standardised outputs.  Packed parameters (float): W1[64][16] b1[64] W2[64][64] b2[64]
W3[4][64] b3[4] (5508 trained) then mu[16] sd[16] os[4].  Plain numpy, written from the
definition of the network and of back-propagation; shares no code with the CUDA kernels.
Pinned in tests/test_learned_oracle.py against central finite differences.
"""
import numpy as np

F, H, O = 16, 64, 4
NTRAIN = H * F + H + H * H + H + O * H + O
NW = NTRAIN + 2 * F + O


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in (("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (O, H)), ("b3", (O,)),
                        ("mu", (F,)), ("sd", (F,)), ("os", (O,))):
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def forward(w, X):
    """Scaled outputs [n, 4] (the dimensionless corrections)."""
    p = unpack(w)
    xs = (np.asarray(X, np.float64) - p["mu"]) / p["sd"]
    h1 = np.tanh(xs @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    return (h2 @ p["W3"].T + p["b3"]) * p["os"]


def loss_and_grad(w, X, Yt):
    """Mean squared error of the standardised outputs and its gradient w.r.t. the
    5508 trained parameters (back-propagation)."""
    p = unpack(w)
    n = X.shape[0]
    xs = (np.asarray(X, np.float64) - p["mu"]) / p["sd"]
    h1 = np.tanh(xs @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    y = h2 @ p["W3"].T + p["b3"]
    e = y - np.asarray(Yt, np.float64) / p["os"]
    loss = np.mean(e * e)
    dy = 2.0 * e / (n * O)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    d2 = (dy @ p["W3"]) * (1 - h2 * h2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ p["W2"]) * (1 - h1 * h1)
    gW1 = d1.T @ xs
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g
