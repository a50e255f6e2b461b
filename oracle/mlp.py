"""The learned short-range factor: a 1-16-16-1 SiLU network (oracle side).

Test infrastructure only.  Float64 forward, backward and Adam, written from
the definitions:

* input z0 = 2 r / rcut - 1 (r unsoftened, in [0, rcut));
* a1 = W1 z0 + b1, h1 = silu(a1);   a2 = W2 h1 + b2, h2 = silu(a2);
  y = W3 . h2 + b3;  the network's factor is g_hat(r) = y;
* silu(a) = a sigma(a) = a / (1 + exp(-a));
* loss over a batch: mean of ((g_hat - g) / g)^2 with g the exact factor of
  Eq. (split);
* Adam (Kingma & Ba 2015): m = b1 m + (1-b1) grad, v = b2 v + (1-b2) grad^2,
  theta -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Flat parameter layout (321 values): W1[16], b1[16], W2[16][16] (row k holds
the weights into unit k), b2[16], W3[16], b3.

Random numbers: training samples and minibatch indices come from splitmix64
(G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used as a counter-based generator: the k-th value
of stream s is splitmix64's output function applied to s + (k+1) * gamma.
"""
from __future__ import annotations

import math

import numpy as np

NH = 16
NPARAM = NH + NH + NH * NH + NH + NH + 1     # 321
GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def offsets():
    o = {}
    i = 0
    for name, size in (("W1", NH), ("b1", NH), ("W2", NH * NH), ("b2", NH), ("W3", NH), ("b3", 1)):
        o[name] = (i, i + size)
        i += size
    return o


OFF = offsets()


def unpack(theta):
    theta = np.asarray(theta, np.float64)
    W1 = theta[slice(*OFF["W1"])]
    b1 = theta[slice(*OFF["b1"])]
    W2 = theta[slice(*OFF["W2"])].reshape(NH, NH)
    b2 = theta[slice(*OFF["b2"])]
    W3 = theta[slice(*OFF["W3"])]
    b3 = theta[OFF["b3"][0]]
    return W1, b1, W2, b2, W3, b3


def sigmoid(a):
    return 1.0 / (1.0 + np.exp(-a))


def silu(a):
    return a * sigmoid(a)


def silu_grad(a):
    s = sigmoid(a)
    return s * (1.0 + a * (1.0 - s))


def forward(theta, z0):
    """g_hat for inputs z0 (any shape); also returns the cached activations."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    z0 = np.asarray(z0, np.float64).reshape(-1)
    a1 = z0[:, None] * W1[None, :] + b1[None, :]
    h1 = silu(a1)
    a2 = h1 @ W2.T + b2[None, :]
    h2 = silu(a2)
    y = h2 @ W3 + b3
    return y, (z0, a1, h1, a2, h2)


def g_hat(theta, r, rcut):
    return forward(theta, 2.0 * np.asarray(r, np.float64) / rcut - 1.0)[0]


def loss_and_grad(theta, z0, target):
    """Mean relative squared error and its gradient (chain rule, by hand)."""
    y, (z0, a1, h1, a2, h2) = forward(theta, z0)
    target = np.asarray(target, np.float64).reshape(-1)
    n = y.size
    rel = (y - target) / target
    loss = float(np.mean(rel * rel))
    dy = 2.0 * rel / target / n                       # d loss / d y
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    dh2 = dy[:, None] * W3[None, :]
    da2 = dh2 * silu_grad(a2)
    gW2 = da2.T @ h1                                   # [k, j]
    gb2 = da2.sum(0)
    dh1 = da2 @ W2
    da1 = dh1 * silu_grad(a1)
    gW1 = (da1 * z0[:, None]).sum(0)
    gb1 = da1.sum(0)
    g = np.concatenate([gW1, gb1, gW2.reshape(-1), gb2, gW3, [gb3]])
    return loss, g


class Adam:
    def __init__(self, n, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.b1, self.b2, self.eps = b1, b2, eps

    def step(self, theta, grad, lr):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - lr * mh / (np.sqrt(vh) + self.eps)


# ------------------------------------------------------------ random streams
def splitmix64(stream, k):
    """k-th (0-based) value of the counter-based splitmix64 stream ``stream``."""
    k = np.asarray(k, np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(stream) + (k + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform24(stream, k):
    """Uniform floats in [0, 1) with 24 random bits (exact in float32)."""
    return (splitmix64(stream, k) >> np.uint64(40)).astype(np.float64) * 2.0 ** -24


def init_params(seed):
    """Seeded initial parameters: U(-1/sqrt(fan_in), 1/sqrt(fan_in)), drawn
    from stream ``seed`` in the flat parameter order."""
    u = uniform24(seed, np.arange(NPARAM))
    fan = np.empty(NPARAM)
    for name, f in (("W1", 1), ("b1", 1), ("W2", NH), ("b2", NH), ("W3", NH), ("b3", NH)):
        fan[slice(*OFF[name])] = f
    return ((2.0 * u - 1.0) / np.sqrt(fan)).astype(np.float32).astype(np.float64)


def lr_at(step, steps, lr0, lr_min):
    """Cosine decay from lr0 to lr_min over ``steps`` steps."""
    return lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * step / max(steps, 1)))


def train(rcut_over_rs, n_samples, batch, steps, lr0, lr_min, seed, theta0=None, targets_fn=None):
    """Replica of the GPU training loop (float64): samples, batches, Adam.

    Samples: x_k = uniform24(seed + 1, k), z0 = 2 x_k - 1, r = x_k rcut, target
    = the exact factor at r (``targets_fn(x)`` if given, else Eq. (split));
    step s uses samples splitmix64(seed + 2, s*batch + k) mod n_samples.
    """
    from scipy.special import erfc
    x = uniform24(seed + 1, np.arange(n_samples))
    if targets_fn is None:
        s = x * rcut_over_rs          # r / R_s
        tgt = erfc(s / 2.0) + s / np.sqrt(np.pi) * np.exp(-s * s / 4.0)
    else:
        tgt = targets_fn(x)
    z0 = 2.0 * x - 1.0
    theta = init_params(seed) if theta0 is None else np.asarray(theta0, np.float64)
    opt = Adam(NPARAM)
    losses = []
    for st in range(steps):
        idx = (splitmix64(seed + 2, np.arange(batch) + np.uint64(st * batch)) % np.uint64(n_samples)).astype(np.int64)
        loss, g = loss_and_grad(theta, z0[idx], tgt[idx])
        theta = opt.step(theta, g, lr_at(st, steps, lr0, lr_min))
        losses.append(loss)
    return theta, losses
