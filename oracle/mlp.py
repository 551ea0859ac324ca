"""FP64 reference of the order-selection network (32 -> 64 -> 32 -> 32 -> 2,
ReLU, mean squared error) -- TEST INFRASTRUCTURE ONLY.  Plain numpy forward
and backward passes written from the definitions, used to check the CUDA
training kernels' gradients.  Parameter layout: W1[64][32] b1[64] W2[32][64]
b2[32] W3[32][32] b3[32] W4[2][32] b4[2]."""
import numpy as np

DIMS = (32, 64, 32, 32, 2)


def unpack(w):
    w = np.asarray(w, np.float64)
    out, o = [], 0
    for nin, nout in zip(DIMS[:-1], DIMS[1:]):
        W = w[o:o + nin * nout].reshape(nout, nin)
        o += nin * nout
        b = w[o:o + nout]
        o += nout
        out.append((W, b))
    assert o == len(w)
    return out


def forward(w, X):
    a = np.asarray(X, np.float64)
    zs, acts = [], [a]
    layers = unpack(w)
    for i, (W, b) in enumerate(layers):
        z = a @ W.T + b
        a = np.maximum(z, 0.0) if i < len(layers) - 1 else z
        zs.append(z)
        acts.append(a)
    return a, zs, acts


def loss_grad(w, X, Y):
    """Mean over samples and outputs of the squared error, and its gradient."""
    yh, zs, acts = forward(w, X)
    Y = np.asarray(Y, np.float64)
    n = yh.size
    loss = ((yh - Y) ** 2).sum() / n
    delta = 2.0 * (yh - Y) / n
    layers = unpack(w)
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        gW = delta.T @ acts[i]
        gb = delta.sum(0)
        grads.append((gW, gb))
        if i > 0:
            delta = (delta @ W) * (zs[i - 1] > 0)
    g = []
    for gW, gb in reversed(grads):
        g.append(gW.ravel())
        g.append(gb)
    return loss, np.concatenate(g)
