"""FP64 CPU oracle of the warm-start MLP -- TEST INFRASTRUCTURE ONLY.

x -> relu(W1 x + b1) -> relu(W2 h1 + b2) -> W3 h2 + b3, loss = mean over all outputs of
((y - (t - mean)/std))^2, and its gradients by the chain rule written out layer by layer.
Weights are [out][in]; batches are rows. Plain numpy matmuls in float64. `adam_step` is the
optimiser update the device applies to those gradients (Kingma & Ba's Adam, written out).

`store` (default: none) is applied wherever a value is stored between steps -- the hidden
activations h1, h2 and the back-propagated dY, dZ2, dZ1 -- so that the oracle can reproduce a
device that keeps those arrays in a narrower format (BF16) while all arithmetic stays FP64.
"""
import numpy as np


def _id(a):
    return a


def forward(params, X, store=_id):
    (W1, b1), (W2, b2), (W3, b3) = [(np.asarray(W, np.float64), np.asarray(b, np.float64)) for W, b in params]
    Z1 = X @ W1.T + b1
    H1 = store(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + b2
    H2 = store(np.maximum(Z2, 0.0))
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss_and_grads(params, X, T, mean=None, std=None, store=_id):
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    Y, (X, Z1, H1, Z2, H2) = forward(params, X, store)
    Tn = T if mean is None else (T - mean) / std
    R = Y - Tn
    loss = float(np.mean(R * R))
    dY = store(2.0 * R / R.size)
    (W1, _), (W2, _), (W3, _) = [(np.asarray(W, np.float64), b) for W, b in params]
    gW3, gb3 = dY.T @ H2, dY.sum(axis=0)
    dZ2 = store((dY @ W3) * (Z2 > 0))
    gW2, gb2 = dZ2.T @ H1, dZ2.sum(axis=0)
    dZ1 = store((dZ2 @ W2) * (Z1 > 0))
    gW1, gb1 = dZ1.T @ X, dZ1.sum(axis=0)
    return loss, [(gW1, gb1), (gW2, gb2), (gW3, gb3)]


def adam_step(param, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, "Adam: A Method for Stochastic Optimization", Algorithm 1),
    FP64, elementwise, in the paper's order: the biased first and second moment estimates, their
    bias corrections by 1 - beta^t (t = 1 for the first update), then the parameter step.
    Returns (param, m, v) as new arrays; the inputs are not modified."""
    p = np.asarray(param, np.float64)
    g = np.asarray(grad, np.float64)
    m_t = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v_t = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m_t / (1.0 - beta1 ** t)
    v_hat = v_t / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m_t, v_t
