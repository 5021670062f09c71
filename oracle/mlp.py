"""Surrogate network of the control-variate level, plain FP64 (test
infrastructure only; see the oracle package docstring).

The surrogate S(xi) maps the KL coefficients of a sample to its level-0
outflux; it enters the estimator as one more level below the coarsest grid:
  E[Q_L] = E[S] + E[Q_0 - S] + sum_{l>=1} E[Q_l - Q_(l-1)],
which stays unbiased for any S (the same telescoping as Eq. 2); a good S only
lowers V[Q_0 - S].

Network: x (M inputs) -> three hidden layers of 256 with GELU
gelu(z) = z (1 + erf(z / sqrt 2)) / 2 -> one output; the target is the
standardised outflux (Q - mu) / sd and S(xi) = mu + sd * output.

`forward` / `backward` take a `rounding` switch: with rounding=True they
round to BF16 (round to nearest even) exactly where the tensor-core kernels
hold BF16 operands - the weights, the input, each hidden activation and each
back-propagated pre-activation gradient - and otherwise compute in FP64;
with rounding=False the network is the plain FP64 function whose gradients
the finite-difference test checks.
"""
import numpy as np

HIDDEN = 256
LAYERS = 4


def bf16(x):
    """Round FP64 -> FP32 -> BF16 (nearest even on the FP32 bit pattern), back to FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(f)
    out = (r.astype(np.uint32)).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def gelu(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def init_params(M, rng_uniform):
    """Weights W_l [out][in] and biases, U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from
    the given uniform(0,1) draws (a callable n -> array)."""
    dims = [M, HIDDEN, HIDDEN, HIDDEN, 1]
    params = []
    for l in range(LAYERS):
        fan_in, fan_out = dims[l], dims[l + 1]
        a = 1.0 / np.sqrt(fan_in)
        W = (2.0 * rng_uniform(fan_out * fan_in) - 1.0) * a
        b = (2.0 * rng_uniform(fan_out) - 1.0) * a
        params.append((W.reshape(fan_out, fan_in), b))
    return params


def forward(params, X, rounding=True):
    """Returns (output [B], cache).  X [B][M] standardised inputs."""
    r = bf16 if rounding else (lambda v: v)
    H = r(X)
    cache = []
    for l, (W, b) in enumerate(params):
        Z = H @ r(W).T + b                      # FP32 accumulation on the GPU
        cache.append((H, Z))
        if l < LAYERS - 1:
            H = r(gelu(Z))
        else:
            H = Z
    return H[:, 0], cache


def backward(params, cache, dout, rounding=True):
    """Gradients of sum_b dout[b] * output[b]; returns [(dW, db)] per layer."""
    r = bf16 if rounding else (lambda v: v)
    grads = [None] * LAYERS
    dZ = dout[:, None]                          # output layer: dZ = dout
    for l in range(LAYERS - 1, -1, -1):
        W, b = params[l]
        H, Z = cache[l]
        if l < LAYERS - 1:
            dZ = r(dZ)                          # the GEMM operand is BF16
        grads[l] = (dZ.T @ H, dZ.sum(axis=0))
        if l > 0:
            dH = dZ @ r(W)
            Zp = cache[l - 1][1]
            dZ = dH * gelu_grad(Zp)
    return grads


def mse_loss_and_grad(params, X, t, rounding=True):
    """L = mean_b (out_b - t_b)^2; returns (L, grads)."""
    out, cache = forward(params, X, rounding)
    diff = out - t
    L = float(np.mean(diff * diff))
    grads = backward(params, cache, 2.0 * diff / len(t), rounding)
    return L, grads


class Adam:
    """Kingma & Ba (2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
    p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.t = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params, grads, lr=None):
        lr = self.lr if lr is None else lr
        self.t += 1
        out = []
        for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[l][j] + (1 - self.b1) * g
                v = self.b2 * self.v[l][j] + (1 - self.b2) * g * g
                self.m[l] = (m, self.m[l][1]) if j == 0 else (self.m[l][0], m)
                self.v[l] = (v, self.v[l][1]) if j == 0 else (self.v[l][0], v)
                mh = m / (1 - self.b1 ** self.t)
                vh = v / (1 - self.b2 ** self.t)
                new.append(p - lr * mh / (np.sqrt(vh) + self.eps))
            out.append((new[0], new[1]))
        return out
