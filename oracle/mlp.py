"""Oracle of the learned warm start (test infrastructure: used by tests/ only).

The warm start maps a parameter vector mu to reduced coefficients y(mu) in R^n,
so that x_0 = W y(mu) starts the RB solvers (Alg. 2, Alg. 3) inside span(W)
instead of at 0.  The network: features of mu (log of the diffusion
coefficients, the load parameters as they are), standardised with the mean
and standard deviation of the training features; two hidden layers of width
128 with GELU; a linear output layer predicting standardised coefficients.

Precision contract shared with the CUDA kernels: weights are used as BF16
values (the FP32 master weights rounded to nearest, ties to even), biases and
activations stay FP32 there and FP64 here.  The gradient treats the rounding
as the identity (the master weights are what Adam updates).

Every function restates its definition; nothing here calls or imports the
CUDA library.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np
from scipy.special import erf

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def bf16_round(a) -> np.ndarray:
    """Round to BF16 (8 significant bits, binary32 exponent range), nearest with
    ties to even, via the binary32 value; returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    """GELU(z) = z Phi(z) with the standard normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2."""
    return 0.5 * z * (1.0 + erf(z / SQRT2))


def gelu_grad(z):
    """d/dz z Phi(z) = Phi(z) + z phi(z), phi the standard normal density."""
    return 0.5 * (1.0 + erf(z / SQRT2)) + z * INV_SQRT_2PI * np.exp(-0.5 * z * z)


def features(mu, P: int) -> np.ndarray:
    """log mu_i for the P diffusion coefficients, mu_i for the load parameters."""
    mu = np.atleast_2d(np.asarray(mu, dtype=np.float64))
    F = mu.copy()
    F[:, :P] = np.log(mu[:, :P])
    return F


def standardisation(F: np.ndarray, T: np.ndarray):
    """Per-column mean and standard deviation (population, floored at 1e-12) of
    the training features F [S][I] and targets T [S][O]."""
    fm, tm = F.mean(axis=0), T.mean(axis=0)
    fs = np.maximum(F.std(axis=0), 1e-12)
    ts = np.maximum(T.std(axis=0), 1e-12)
    return fm, fs, tm, ts


@dataclasses.dataclass
class Net:
    W: List[np.ndarray]          # master weights, W_l [out][in]
    b: List[np.ndarray]
    in_mean: np.ndarray
    in_scale: np.ndarray
    out_mean: np.ndarray
    out_scale: np.ndarray


def from_init(params, F: np.ndarray, T: np.ndarray) -> Net:
    """A network with initial (W_l, b_l) and the standardisation of (F, T)."""
    fm, fs, tm, ts = standardisation(F, T)
    return Net([np.array(W, dtype=np.float64) for W, _ in params], [np.array(b, dtype=np.float64) for _, b in params],
               fm, fs, tm, ts)


def forward(net: Net, X: np.ndarray, rounding: bool = True):
    """Layer values for standardised inputs X [S][I]: [(z_l, a_l)], output a_L = z_L."""
    acts = []
    a = X
    L = len(net.W)
    for l in range(L):
        Wl = bf16_round(net.W[l]) if rounding else net.W[l]
        z = a @ Wl.T + net.b[l]
        a = gelu(z) if l < L - 1 else z
        acts.append((z, a))
    return acts


def predict(net: Net, mu, P: int) -> np.ndarray:
    """y(mu) = out_mean + out_scale * network((features(mu) - in_mean) / in_scale)."""
    X = (features(mu, P) - net.in_mean) / net.in_scale
    return net.out_mean + net.out_scale * forward(net, X)[-1][1]


def loss_and_grads(net: Net, X: np.ndarray, Ts: np.ndarray, rounding: bool = True):
    """Mean squared error L = sum (y - t)^2 / (S O) over standardised targets Ts [S][O]
    and its gradient with respect to every W_l and b_l (back-propagation)."""
    acts = forward(net, X, rounding)
    S, O = Ts.shape
    Y = acts[-1][1]
    L = float(np.sum((Y - Ts) ** 2) / (S * O))
    dA = 2.0 * (Y - Ts) / (S * O)
    gW, gb = [None] * len(net.W), [None] * len(net.W)
    for l in range(len(net.W) - 1, -1, -1):
        z, _ = acts[l]
        dZ = dA if l == len(net.W) - 1 else dA * gelu_grad(z)
        prev = X if l == 0 else acts[l - 1][1]
        gW[l] = dZ.T @ prev
        gb[l] = dZ.sum(axis=0)
        Wl = bf16_round(net.W[l]) if rounding else net.W[l]
        dA = dZ @ Wl
    return L, gW, gb


@dataclasses.dataclass
class Adam:
    """Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""
    lr: float = 3e-3
    b1: float = 0.9
    b2: float = 0.999
    eps: float = 1e-8
    t: int = 0
    m: list = dataclasses.field(default_factory=list)
    v: list = dataclasses.field(default_factory=list)

    def step(self, params: List[np.ndarray], grads: List[np.ndarray]) -> None:
        if not self.m:
            self.m = [np.zeros_like(p) for p in params]
            self.v = [np.zeros_like(p) for p in params]
        self.t += 1
        c1, c2 = 1.0 - self.b1 ** self.t, 1.0 - self.b2 ** self.t
        for p, g, m, v in zip(params, grads, self.m, self.v):
            m *= self.b1
            m += (1.0 - self.b1) * g
            v *= self.b2
            v += (1.0 - self.b2) * g * g
            p -= self.lr * (m / c1) / (np.sqrt(v / c2) + self.eps)


def train(net: Net, F: np.ndarray, T: np.ndarray, steps: int, lr: float = 3e-3) -> List[float]:
    """Full-batch Adam on the standardised pairs; returns the loss before each step."""
    X = (F - net.in_mean) / net.in_scale
    Ts = (T - net.out_mean) / net.out_scale
    opt = Adam(lr=lr)
    hist = []
    for _ in range(steps):
        L, gW, gb = loss_and_grads(net, X, Ts)
        hist.append(L)
        params = [p for pair in zip(net.W, net.b) for p in pair]
        grads = [g for pair in zip(gW, gb) for g in pair]
        opt.step(params, grads)
    return hist
