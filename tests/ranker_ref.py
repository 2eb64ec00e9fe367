"""Float64 CPU reference of the ranker network's loss and gradient.

Written from the definition in include/ivm.h: layers 76 -> 128 -> 128 -> 128
(ReLU) -> 64, mean softmax cross-entropy over the batch; master weights in
one flat array W1[76][128], b1, W2[128][128], b2, W3[128][128], b3,
W4[128][64], b4.  Used to check the library's FP32 training kernels."""
import numpy as np

SHAPES = [(76, 128), (128, 128), (128, 128), (128, 64)]


def unpack(w):
    out, off = [], 0
    for i, o in SHAPES:
        W = w[off:off + i * o].reshape(i, o)
        off += i * o
        b = w[off:off + o]
        off += o
        out.append((W, b))
    assert off == len(w)
    return out


def n_params():
    return sum(i * o + o for i, o in SHAPES)


def loss_and_grad(w, x, y):
    w = np.asarray(w, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    B = x.shape[0]
    layers = unpack(w)
    acts = [x]
    for k, (W, b) in enumerate(layers):
        z = acts[-1] @ W + b
        acts.append(np.maximum(z, 0.0) if k < 3 else z)
    z = acts[-1]
    m = z.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.exp(z - m).sum(axis=1))
    loss = float(np.mean(lse - z[np.arange(B), y]))
    p = np.exp(z - lse[:, None])
    d = p.copy()
    d[np.arange(B), y] -= 1.0
    d /= B
    grads = []
    for k in range(3, -1, -1):
        W, b = layers[k]
        a_in = acts[k]
        grads.append((a_in.T @ d, d.sum(axis=0)))
        if k > 0:
            d = (d @ W.T) * (acts[k] > 0)
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def loss_only(w, x, y):
    return loss_and_grad(w, x, y)[0]
