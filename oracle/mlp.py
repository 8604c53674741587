"""Plain numpy reference of the warm start's network (TEST INFRASTRUCTURE ONLY).

in -> hidden -> hidden -> out, ReLU, loss L = (1/B) sum_b sum_o [softplus(z) - t z]
(binary cross-entropy on logits, summed over outputs, averaged over the
batch).  Parameters are packed W1 (in x hidden), b1, W2, b2, W3, b3.

``fp16_points=True`` rounds to float16 exactly where the CUDA network keeps
FP16 values (inputs, weights, ReLU activations, back-propagated dz), so that
the remaining difference is only the order of FP32 accumulation.  Pinned in
tests/test_mlp_oracle.py by central finite differences and a hand-computed
example.
"""
import numpy as np


def shapes(i, h, o):
    return [(i, h), (h,), (h, h), (h,), (h, o), (o,)]


def unpack(flat, i, h, o):
    out, k = [], 0
    for s in shapes(i, h, o):
        n = int(np.prod(s))
        out.append(flat[k:k + n].reshape(s))
        k += n
    return out


def _q(x, on):
    return x.astype(np.float16).astype(np.float64) if on else x


def softplus(z):
    return np.where(z > 0, z + np.log1p(np.exp(-np.abs(z))), np.log1p(np.exp(np.minimum(z, 0))))


def forward(flat, X, i, h, o, fp16_points=False):
    W1, b1, W2, b2, W3, b3 = (_q(p, fp16_points) if p.ndim == 2 else p
                              for p in unpack(np.asarray(flat, np.float64), i, h, o))
    x = _q(np.asarray(X, np.float64), fp16_points)
    z1 = x @ W1 + b1
    a1 = _q(np.maximum(z1, 0), fp16_points)
    z2 = a1 @ W2 + b2
    a2 = _q(np.maximum(z2, 0), fp16_points)
    z3 = a2 @ W3 + b3
    return dict(x=x, W1=W1, W2=W2, W3=W3, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3)


def loss_and_grads(flat, X, T, i, h, o, fp16_points=False):
    f = forward(flat, X, i, h, o, fp16_points)
    T = np.asarray(T, np.float64)
    B = X.shape[0]
    z3 = f["z3"]
    loss = float(np.sum(softplus(z3) - T * z3) / B)
    dz3 = _q((1.0 / (1.0 + np.exp(-z3)) - T) / B, fp16_points)
    gW3 = f["a2"].T @ dz3
    gb3 = dz3.sum(0)
    dz2 = _q((dz3 @ f["W3"].T) * (f["z2"] > 0), fp16_points)
    gW2 = f["a1"].T @ dz2
    gb2 = dz2.sum(0)
    dz1 = _q((dz2 @ f["W2"].T) * (f["z1"] > 0), fp16_points)
    gW1 = f["x"].T @ dz1
    gb1 = dz1.sum(0)
    g = np.concatenate([v.ravel() for v in (gW1, gb1, gW2, gb2, gW3, gb3)])
    return loss, g
