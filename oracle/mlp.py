"""FP64 reference of the warm-start network (test infrastructure only; nothing
in the product imports it).

The paper has no learned component: its initial guess of the implicit step is
an extrapolation from past steps (Sec. 3.3). The network checked here is a
plain multilayer perceptron, written out from its definition:

    x_hat = (x - in_mean) / in_std                         (800 inputs)
    h_1 = relu(W_1 x_hat + b_1), h_2 = relu(W_2 h_1 + b_2), h_3 = relu(W_3 h_2 + b_3)
    y_hat = W_4 h_3 + b_4,  y = out_mean + out_std * y_hat   (192 outputs)
    L = sum over rows and outputs (y_hat - t_hat)^2 / (2 B),  t_hat = (t - out_mean) / out_std

with W_l stored [out x in] and packed with the biases as W1, b1, ..., W4, b4.
Gradients follow the chain rule (backpropagation) in FP64.

`bf16=True` additionally rounds to bfloat16 (round to nearest, ties to even)
exactly where the tensor-core path stores BF16 operands: the normalised
input, the weights, the hidden activations, and the back-propagated output
and hidden gradients that feed the weight-gradient products (the bias
gradients use the unrounded values). With `bf16=False` the arithmetic is
plain FP64 (used for the finite-difference pin).
"""
import numpy as np

DIMS = [(800, 256), (256, 256), (256, 256), (256, 192)]   # (in, out) per layer
NPARAM = sum(i * o + o for i, o in DIMS)


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_bits(a):
    """bfloat16 bit patterns (uint16) of a float array, rounded as bf16_round."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def unpack(params):
    """[(W [out x in], b [out])] views of the packed parameter vector."""
    out, p = [], 0
    for i, o in DIMS:
        W = params[p:p + i * o].reshape(o, i)
        p += i * o
        b = params[p:p + o]
        p += o
        out.append((W, b))
    return out


def _r(a, on):
    return bf16_round(a) if on else np.asarray(a, dtype=np.float64)


def forward(params, x, norm, bf16=True):
    """Raw outputs y [B x 192] and the cache for backward. norm = (in_mean,
    in_std, out_mean, out_std)."""
    in_mean, in_std, out_mean, out_std = (np.asarray(v, dtype=np.float64) for v in norm)
    layers = unpack(np.asarray(params, dtype=np.float64))
    h = _r((np.asarray(x, dtype=np.float64) - in_mean) / in_std, bf16)
    acts = [h]
    for l, (W, b) in enumerate(layers):
        z = h @ _r(W, bf16).T + b
        if l < 3:
            h = _r(np.maximum(z, 0.0), bf16)
            acts.append(h)
        else:
            yhat = z
    return out_mean + out_std * yhat, (acts, yhat, layers)


def loss_and_grad(params, x, t, norm, bf16=True):
    """Loss and its gradient with respect to the packed parameters."""
    _, out_mean, out_std = norm[1], np.asarray(norm[2], np.float64), np.asarray(norm[3], np.float64)
    y, (acts, yhat, layers) = forward(params, x, norm, bf16)
    B = x.shape[0]
    d = yhat - (np.asarray(t, dtype=np.float64) - out_mean) / out_std
    loss = 0.5 * np.sum(d * d) / B
    dz = d / B                                  # dL/dz of the output layer
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, _ = layers[l]
        dz_r = _r(dz, bf16)
        grads[l] = (dz_r.T @ acts[l], dz.sum(axis=0))
        if l > 0:
            dz = (dz_r @ _r(W, bf16)) * (acts[l] > 0)
    g = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return loss, g


def grad_magnitudes(params, x, t, norm, bf16=True):
    """Magnitude sums of the gradient: the backward pass of loss_and_grad with
    every factor replaced by its absolute value, so entry (i, j) of a weight
    gradient is sum_b |dz_b,i| |h_b,j| and entry i of a bias gradient
    sum_b |dz_b,i|, with |dz| propagated as (|dz| |W|) * relu-mask. A bound on
    the rounding error of a gradient entry is a multiple of its magnitude sum
    (each term can carry a BF16 rounding of either factor)."""
    out_mean, out_std = np.asarray(norm[2], np.float64), np.asarray(norm[3], np.float64)
    y, (acts, yhat, layers) = forward(params, x, norm, bf16)
    B = x.shape[0]
    dz = np.abs(yhat - (np.asarray(t, dtype=np.float64) - out_mean) / out_std) / B
    mags = [None] * 4
    for l in range(3, -1, -1):
        W, _ = layers[l]
        dz_r = _r(dz, bf16)
        mags[l] = (dz_r.T @ np.abs(acts[l]), dz.sum(axis=0))
        if l > 0:
            dz = (dz_r @ np.abs(_r(W, bf16))) * (acts[l] > 0)
    return np.concatenate([np.concatenate([mW.ravel(), mb]) for mW, mb in mags])
