"""Float64 reference of the lens-surrogate MLP (4 -> 128 -> 128 -> 128 -> 2, tanh).

TEST INFRASTRUCTURE ONLY (tests may import it; the library never does).  A
textbook dense network with its hand-written backward pass, in numpy float64.
`round_bf16=True` rounds to bfloat16 exactly where the tensor-core kernels
store bf16 values (the two hidden weight matrices, the three hidden
activations and the back-propagated dZ of layers 3 and 2), so that the CUDA
gradient can be compared closely; the arithmetic stays float64.

Parameter vector layout: W1[128][4], b1[128], W2[128][128], b2[128],
W3[128][128], b3[128], W4[2][128], b4[2].
Loss: mean over the batch of the squared error summed over both outputs.
"""
import numpy as np

H = 128
SIZES = [("W1", (H, 4)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)), ("b3", (H,)),
         ("W4", (2, H)), ("b4", (2,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SIZES])


def bf16(x):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def forward_backward(p, X, Y, round_bf16=False):
    """Loss and gradient (packed like p) on the batch X [n][4], Y [n][2]."""
    q = unpack(p)
    rb = bf16 if round_bf16 else (lambda a: a)
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    n = X.shape[0]
    W2, W3 = rb(q["W2"]), rb(q["W3"])
    h1 = rb(np.tanh(X @ q["W1"].T + q["b1"]))
    h2 = rb(np.tanh(h1 @ W2.T + q["b2"]))
    h3 = rb(np.tanh(h2 @ W3.T + q["b3"]))
    y = h3 @ q["W4"].T + q["b4"]
    err = y - Y
    loss = float(np.sum(err * err) / n)
    dy = 2.0 * err / n
    g = {"W4": dy.T @ h3, "b4": dy.sum(0)}
    dz3 = rb((dy @ q["W4"]) * (1.0 - h3 * h3))
    g["W3"], g["b3"] = dz3.T @ h2, dz3.sum(0)
    dz2 = rb((dz3 @ W3) * (1.0 - h2 * h2))
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    g["W1"], g["b1"] = dz1.T @ X, dz1.sum(0)
    return loss, pack(g)


def init(seed=0):
    """Xavier-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SIZES:
        if name.startswith("W"):
            a = np.sqrt(6.0 / (shape[0] + shape[1]))
            d[name] = rng.uniform(-a, a, shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)
