"""Plain FP64 restatement of the learned screen's network -- TEST INFRASTRUCTURE.

A 4 -> 64 -> 64 -> 1 multilayer perceptron with tanh hidden layers, written out
with numpy for checking the CUDA training and inference kernels.  The parameter
vector uses the library's documented layout: W1[64][4], b1[64], W2[64][64],
b2[64], W3[64], b3, x_mean[4], x_std[4], y_mean, y_std.
"""
import numpy as np

H, IN = 64, 4
NP = H * IN + H + H * H + H + H + 1
NALL = NP + 10


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]; o += 1
    xm, xs, ym, ys = p[o:o + 4], p[o + 4:o + 8], p[o + 8], p[o + 9]
    return W1, b1, W2, b2, W3, b3, xm, xs, ym, ys


def forward(p, x):
    """Predicted log10 term norms for rows x [n, 4]."""
    W1, b1, W2, b2, W3, b3, xm, xs, ym, ys = unpack(p)
    z = (np.asarray(x, np.float64) - xm) / xs
    h1 = np.tanh(z @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return (h2 @ W3 + b3) * ys + ym


def loss_and_grad(p, x, y):
    """L = mean((o - (y - y_mean)/y_std)^2) and dL/dp for the 4545 trainable entries."""
    W1, b1, W2, b2, W3, b3, xm, xs, ym, ys = unpack(p)
    n = len(y)
    z = (np.asarray(x, np.float64) - xm) / xs
    h1 = np.tanh(z @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    o = h2 @ W3 + b3
    t = (np.asarray(y, np.float64) - ym) / ys
    e = o - t
    L = float(np.mean(e * e))
    do = 2.0 * e / n
    gW3 = h2.T @ do
    gb3 = do.sum()
    d2 = np.outer(do, W3) * (1.0 - h2 * h2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    gW1 = d1.T @ z
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return L, g
