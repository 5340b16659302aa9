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


# Adam pins: closed forms and invariants of Kingma & Ba's update, none of which restates its
# recursion. A dropped bias correction, a wrong power t, swapped moments, a missing square root or
# a flipped sign each fails at least one of them.

def test_adam_first_step_is_normalised_sign_step():
    # t = 1 from zero moments: the bias corrections turn m and v into g and g^2 exactly
    g = np.array([3.0, -0.25, 1e-3, -40.0, 0.0])
    p0 = np.array([1.0, 2.0, -3.0, 0.5, 7.0])
    lr, eps = 0.01, 1e-8
    p1, m1, v1 = mlp.adam_step(p0, g, np.zeros(5), np.zeros(5), 1, lr, eps=eps)
    assert np.allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_adam_constant_gradient_takes_the_same_step_every_time():
    # with g fixed, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2, so the corrected moments are g and
    # g^2 at every t: each step moves by lr * g / (|g| + eps)
    g = np.array([0.7, -2.0, 5e-4])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 60):
        q, m, v = mlp.adam_step(p, g, m, v, t, 1e-3, eps=1e-12)
        assert np.allclose(q - p, -1e-3 * g / (np.abs(g) + 1e-12), rtol=1e-12, atol=0), t
        p = q


def test_adam_second_step_after_a_sign_flip():
    # g1 = g, g2 = -g: m_2 = -(1 - b1)^2 g and 1 - b1^2 = (1 - b1)(1 + b1), so the corrected first
    # moment is -g (1 - b1)/(1 + b1); v_2 corrects to g^2. Step 2 is +lr (1 - b1)/(1 + b1) sign(g).
    b1, b2, lr = 0.9, 0.999, 0.05
    g = np.array([2.0, -0.5])
    p1, m, v = mlp.adam_step(np.zeros(2), g, np.zeros(2), np.zeros(2), 1, lr, b1, b2, eps=0.0)
    p2, m, v = mlp.adam_step(p1, -g, m, v, 2, lr, b1, b2, eps=0.0)
    assert np.allclose(p2 - p1, lr * (1 - b1) / (1 + b1) * np.sign(g), rtol=1e-12, atol=0)


def test_adam_is_invariant_to_gradient_scale():
    # with eps = 0 the step depends on g only through m / sqrt(v): scaling every g by c > 0 changes nothing
    rng = np.random.default_rng(3)
    gs = rng.standard_normal((6, 8))
    pa = pb = rng.standard_normal(8)
    ma = va = mb = vb = np.zeros(8)
    for t, g in enumerate(gs, start=1):
        pa, ma, va = mlp.adam_step(pa, g, ma, va, t, 1e-2, eps=0.0)
        pb, mb, vb = mlp.adam_step(pb, 1e4 * g, mb, vb, t, 1e-2, eps=0.0)
    assert np.allclose(pa, pb, rtol=1e-12, atol=1e-15)


def test_adam_with_zero_betas_is_sign_descent():
    rng = np.random.default_rng(4)
    p, m, v = rng.standard_normal(5), np.zeros(5), np.zeros(5)
    for t in range(1, 5):
        g = rng.standard_normal(5)
        q, m, v = mlp.adam_step(p, g, m, v, t, 0.1, beta1=0.0, beta2=0.0, eps=0.0)
        assert np.allclose(q - p, -0.1 * np.sign(g), rtol=1e-14, atol=0)
        p = q


def test_adam_minimises_a_quadratic():
    # descent direction and fixed point: on f = 0.5 ||p - p*||^2 the iterates reach p*
    target = np.array([1.5, -2.0, 0.25, 3.0])
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 4001):
        lr = 0.05 if t < 3000 else 0.002
        p, m, v = mlp.adam_step(p, p - target, m, v, t, lr)
    assert np.abs(p - target).max() < 2e-2
