"""The FP64 MLP oracle's gradients against central finite differences of its own loss (a
definition-level check: the loss is evaluated directly, the gradients by the hand-written chain rule)."""
import numpy as np

from oracle import mlp


def test_mlp_oracle_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    din, w, dout, B = 5, 7, 4, 6
    params = [(rng.standard_normal((w, din)), rng.standard_normal(w)),
              (rng.standard_normal((w, w)) * 0.5, rng.standard_normal(w)),
              (rng.standard_normal((dout, w)) * 0.5, rng.standard_normal(dout))]
    X = rng.standard_normal((B, din))
    T = rng.standard_normal((B, dout)) * 2 + 1
    mean, std = rng.standard_normal(dout), rng.uniform(0.5, 2.0, dout)
    loss, grads = mlp.loss_and_grads(params, X, T, mean, std)
    h = 1e-6
    for l in range(3):
        for which in (0, 1):
            P = params[l][which]
            G = grads[l][which]
            flat = P.reshape(-1)
            for idx in rng.choice(flat.size, min(12, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp, _ = mlp.loss_and_grads(params, X, T, mean, std)
                flat[idx] = old - h
                lm, _ = mlp.loss_and_grads(params, X, T, mean, std)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - G.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (l, which, idx, fd)
