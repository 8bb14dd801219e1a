"""FP64 numpy reference of the learned halo network's forward and backward passes.

TEST INFRASTRUCTURE ONLY (the oracle of the library's training kernels).  The network maps 65
features to 20 outputs through two hidden layers of 64 with the tanh form of GELU; the loss is the
mean squared error over all outputs of the batch.  Parameter layout: W1[64][65], b1[64],
W2[64][64], b2[64], W3[20][64], b3[20].
"""
import numpy as np

NIN, NH, NOUT = 65, 64, 20
K0, K1 = 0.7978845608028654, 0.044715
NPARAM = NH * NIN + NH + NH * NH + NH + NOUT * NH + NOUT


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    out = []
    for shape in ((NH, NIN), (NH,), (NH, NH), (NH,), (NOUT, NH), (NOUT,)):
        n = int(np.prod(shape))
        out.append(p[i:i + n].reshape(shape))
        i += n
    return out


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(K0 * (z + K1 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * K0 * (1.0 + 3.0 * K1 * z * z)


def forward(p, X):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    return h2 @ W3.T + b3, (z1, h1, z2, h2)


def loss_and_grad(p, X, T):
    """Mean squared error over all n x 20 outputs and its gradient (flat, in parameter order)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    Y, (z1, h1, z2, h2) = forward(p, X)
    n = X.shape[0]
    D = Y - T
    loss = float(np.mean(D * D))
    dY = 2.0 * D / (n * NOUT)
    gW3 = dY.T @ h2
    gb3 = dY.sum(axis=0)
    dz2 = (dY @ W3) * gelu_grad(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def init_params(seed=0):
    """Seeded initial parameters (uniform +-1/sqrt(fan_in), zero biases), FP32."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, shape in ((NIN, (NH, NIN)), (None, (NH,)), (NH, (NH, NH)), (None, (NH,)), (NH, (NOUT, NH)), (None, (NOUT,))):
        if fan_in is None:
            parts.append(np.zeros(shape))
        else:
            parts.append(rng.uniform(-1.0, 1.0, size=shape) / np.sqrt(fan_in))
    return np.concatenate([q.ravel() for q in parts]).astype(np.float32)
