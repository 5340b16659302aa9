"""Pins for the FP64 CPU oracle (oracle/mfs_oracle.c) against facts fixed outside the oracle:
the paper's Example 1, the augmented Lagrangian it minimises (eq. lll, differentiated by
autograd, not by the closed forms), the optimality conditions of a projection, brute-force vertex
enumeration, closed-form optima, a library LP solver (HiGHS) and library sparse products."""
import itertools
import os

import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from oracle.reduced import Reduced
from paper_2203_05027_b300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_blocks(path):
    blocks, cur = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        tok = line.split()
        if tok[0].isalpha():
            cur = tok[0]
            blocks[cur] = []
        else:
            blocks[cur].append([float(t) for t in tok])
    return {k: np.array(v) for k, v in blocks.items()}


def dense_uv(orc):
    ik, jk, ak, FU, FV = orc.uv()
    U = np.zeros((orc.m, orc.o))
    V = np.zeros((orc.n, orc.o))
    U[ik, np.arange(orc.o)] = ak
    V[jk, np.arange(orc.o)] = 1.0
    return U, V, FU, FV


def coo_of(A):
    r, c = np.nonzero(A)
    return r.astype(np.int64), c.astype(np.int64), A[r, c]


def lp_problem(A, b, c, cones=None):
    r, cc, v = coo_of(A)
    m, n = A.shape
    if cones is None:
        cones = [(oracle.CONE_NONNEG, n)]
    return oracle.Oracle(m, n, r, cc, v, b, c, cones)


# ---------------------------------------------------------------- UV decomposition (Sec. IV)

def test_example1_uv_matches_paper():
    g = read_blocks(os.path.join(GOLDEN, "example1.txt"))
    A = g["A"]
    orc = lp_problem(A, np.zeros(3), np.zeros(5))
    U, V, FU, FV = dense_uv(orc)
    assert orc.o == 8
    np.testing.assert_array_equal(U, g["U"])
    np.testing.assert_array_equal(V, g["V"])
    np.testing.assert_array_equal(U @ V.T, A)
    # U U^T = diag(117, 25, 62), V V^T = diag(2, 1, 2, 2, 1): F = (I + diag)^-1
    np.testing.assert_allclose(FU, 1.0 / (1.0 + np.array([117.0, 25.0, 62.0])), rtol=0, atol=0)
    np.testing.assert_allclose(FV, 1.0 / (1.0 + np.array([2.0, 1.0, 2.0, 2.0, 1.0])), rtol=0, atol=0)


def test_uv_definition_random_with_duplicates_and_zeros():
    rng = np.random.default_rng(7)
    m, n, t = 9, 13, 60
    row = rng.integers(0, m, t)
    col = rng.integers(0, n, t)
    val = rng.standard_normal(t)
    val[:5] = 0.0  # explicit zeros are dropped
    A = np.zeros((m, n))
    np.add.at(A, (row, col), val)
    orc = oracle.Oracle(m, n, row, col, val, np.zeros(m), np.zeros(n), [(0, n)])
    U, V, FU, FV = dense_uv(orc)
    assert orc.o == np.count_nonzero(A)
    np.testing.assert_allclose(U @ V.T, A, atol=1e-15)
    UUt, VVt = U @ U.T, V @ V.T
    assert np.count_nonzero(UUt - np.diag(np.diag(UUt))) == 0
    assert np.count_nonzero(VVt - np.diag(np.diag(VVt))) == 0
    np.testing.assert_allclose(FU, np.diag(np.linalg.inv(np.eye(m) + UUt)), rtol=1e-14)
    np.testing.assert_allclose(FV, np.diag(np.linalg.inv(np.eye(n) + VVt)), rtol=1e-14)
    # every column of U and of V has exactly one nonzero
    assert np.all(np.count_nonzero(U, axis=0) == 1) and np.all(np.count_nonzero(V, axis=0) == 1)


def test_invalid_inputs_rejected():
    with pytest.raises(ValueError):
        oracle.Oracle(2, 3, [0], [5], [1.0], np.zeros(2), np.zeros(3), [(0, 3)])
    with pytest.raises(ValueError):
        oracle.Oracle(2, 3, [0], [1], [1.0], np.zeros(2), np.zeros(3), [(0, 2)])


# ---------------------------------------------------------------- the Lagrangian and block steps

def lagrangian(U, V, b, c, mu, x, y, z, lam, gam, dl):
    """Augmented Lagrangian of the reformulated problem (eq. lll), in torch (float64)."""
    Uy_b = U @ y - b
    y_Vx = y - V.T @ x
    z_x = z - x
    return (c @ x + lam @ Uy_b + 0.5 * mu * (Uy_b @ Uy_b) + gam @ y_Vx + 0.5 * mu * (y_Vx @ y_Vx)
            + dl @ z_x + 0.5 * mu * (z_x @ z_x))


def random_setup(seed, cones=None, m=5, n=9, t=22, mu=0.7):
    rng = np.random.default_rng(seed)
    row = rng.integers(0, m, t)
    col = rng.integers(0, n, t)
    val = rng.standard_normal(t)
    b = rng.standard_normal(m)
    c = rng.standard_normal(n)
    if cones is None:
        cones = [(0, 3), (1, 4), (1, 2)]
    orc = oracle.Oracle(m, n, row, col, val, b, c, cones, mu=mu)
    st = dict(x=rng.standard_normal(n), y=rng.standard_normal(orc.o), z=rng.standard_normal(n),
              lam=rng.standard_normal(m), gam=rng.standard_normal(orc.o), delta=rng.standard_normal(n))
    orc.set_state(**st)
    return orc, st, rng


def T(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), dtype=torch.float64)


def grad_of(orc, which, state):
    U, V, _, _ = dense_uv(orc)
    args = {k: T(v) for k, v in state.items()}
    args[which].requires_grad_(True)
    L = lagrangian(T(U), T(V), T(orc.b), T(orc.c), orc.mu, args["x"], args["y"], args["z"],
                   args["lam"], args["gam"], args["delta"])
    (g,) = torch.autograd.grad(L, args[which])
    return g.numpy()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_x_step_minimises_lagrangian(seed):
    orc, st, _ = random_setup(seed)
    g0 = grad_of(orc, "x", st)
    orc.step("x")
    st["x"] = orc.state().x
    g = grad_of(orc, "x", st)
    assert np.abs(g0).max() > 1e-2  # the check is sensitive at a non-minimiser
    assert np.abs(g).max() < 1e-12 * max(1.0, np.abs(g0).max()) * 100


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_y_step_minimises_lagrangian(seed):
    orc, st, _ = random_setup(seed)
    g0 = grad_of(orc, "y", st)
    orc.step("y")
    st["y"] = orc.state().y
    g = grad_of(orc, "y", st)
    assert np.abs(g0).max() > 1e-2
    assert np.abs(g).max() < 1e-10


def in_cone(cones, w, tol=1e-12):
    off = 0
    for kind, s in cones:
        seg = w[off:off + s]
        if kind == 0:
            if seg.min() < -tol:
                return False
        else:
            if np.linalg.norm(seg[1:]) > seg[0] + tol:
                return False
        off += s
    return True


def random_in_cone(rng, cones):
    out = []
    for kind, s in cones:
        if kind == 0:
            out.append(np.abs(rng.standard_normal(s)))
        else:
            t = rng.standard_normal(s - 1)
            out.append(np.concatenate([[np.linalg.norm(t) + abs(rng.standard_normal())], t]))
    return np.concatenate(out)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_z_step_is_constrained_minimiser(seed):
    orc, st, rng = random_setup(seed)
    orc.step("z")
    z = orc.state().z
    assert in_cone(orc.cones, z)
    st["z"] = z
    g = grad_of(orc, "z", st)
    # first-order optimality over K: <g, q - z> >= 0 for all q in K (q = 0 and q = 2z give
    # complementarity <g, z> = 0)
    assert abs(g @ z) < 1e-12
    for _ in range(200):
        q = random_in_cone(rng, orc.cones)
        assert g @ (q - z) >= -1e-12


@pytest.mark.parametrize("seed", [0, 1])
def test_dual_steps_ascend_the_lagrangian(seed):
    """lambda, gamma, delta each move by mu times the gradient of eq. (lll) with respect to it,
    evaluated at the new primal iterate."""
    orc, st, _ = random_setup(seed)
    for name in ("x", "y", "z"):
        orc.step(name)
    s1 = orc.state()
    prim = dict(x=s1.x, y=s1.y, z=s1.z, lam=s1.lam, gam=s1.gam, delta=s1.delta)
    glam, ggam, gdel = (grad_of(orc, w, prim) for w in ("lam", "gam", "delta"))
    for name in ("lambda", "gamma", "delta"):
        orc.step(name)
    s2 = orc.state()
    np.testing.assert_allclose(s2.lam, s1.lam + orc.mu * glam, atol=1e-13)
    np.testing.assert_allclose(s2.gam, s1.gam + orc.mu * ggam, atol=1e-13)
    np.testing.assert_allclose(s2.delta, s1.delta + orc.mu * gdel, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_iteration_ends_in_consistent_state(seed):
    """After any iteration gamma = -U^T lambda; after the next one also
    y = V^T x + U^T F_U (b - A x). The oracle's warm-start mapping must reproduce that state."""
    orc, st, _ = random_setup(seed)
    orc.iterate(1)
    s = orc.state()
    U, V, FU, _ = dense_uv(orc)
    np.testing.assert_allclose(s.gam, -U.T @ s.lam, atol=1e-12)
    y, g = orc.consistent_y_gamma(s.x, s.lam)
    assert np.abs(y - s.y).max() > 1e-3  # an arbitrary start is not yet of that form
    orc.iterate(1)
    s = orc.state()
    np.testing.assert_allclose(s.gam, -U.T @ s.lam, atol=1e-12)
    y, g = orc.consistent_y_gamma(s.x, s.lam)
    np.testing.assert_allclose(y, s.y, atol=1e-12)
    np.testing.assert_allclose(g, s.gam, atol=1e-12)


# ---------------------------------------------------------------- projections (eq. proj)

def test_projection_invariants():
    rng = np.random.default_rng(3)
    for s in (1, 2, 3, 4, 7, 64):
        for _ in range(200):
            w = rng.standard_normal(s) * rng.choice([0.1, 1, 10])
            if s > 1 and rng.random() < 0.3:  # near the tie alpha = +-w1
                w[0] = rng.choice([-1, 1]) * np.linalg.norm(w[1:]) * (1 + 1e-12 * rng.standard_normal())
            p = oracle.proj_lorentz(w)
            pm = oracle.proj_lorentz(-w)
            assert in_cone([(1, s)], p, tol=1e-12)
            np.testing.assert_allclose(oracle.proj_lorentz(p), p, atol=1e-12)   # idempotent
            np.testing.assert_allclose(p - pm, w, atol=1e-12)                   # Moreau
            assert abs(p @ pm) < 1e-10 * max(1.0, w @ w)                         # orthogonal
            for _ in range(5):                                                   # variational ineq.
                q = random_in_cone(rng, [(1, s)])
                assert (w - p) @ (q - p) <= 1e-10 * max(1.0, np.abs(w).max() * np.abs(q).max())
    # size 1 is the nonnegative orthant
    for v in (-2.0, -0.0, 0.0, 3.5):
        assert oracle.proj_lorentz(np.array([v]))[0] == max(v, 0.0)
    # the three cases by hand
    np.testing.assert_array_equal(oracle.proj_lorentz(np.array([-5.0, 3.0, 4.0])), [0, 0, 0])
    np.testing.assert_array_equal(oracle.proj_lorentz(np.array([5.0, 3.0, 4.0])), [5, 3, 4])
    np.testing.assert_allclose(oracle.proj_lorentz(np.array([0.0, 3.0, 4.0])), [2.5, 1.5, 2.0])


def test_nonneg_cone_is_elementwise_max():
    rng = np.random.default_rng(4)
    orc = oracle.Oracle(1, 10, [0], [0], [1.0], [1.0], np.zeros(10), [(0, 6), (1, 4)])
    w = rng.standard_normal(10)
    p = orc.proj_K(w)
    np.testing.assert_array_equal(p[:6], np.maximum(w[:6], 0.0))
    np.testing.assert_array_equal(p[6:], oracle.proj_lorentz(w[6:]))


# ---------------------------------------------------------------- converged solutions

def run_to(orc, tol, max_iter, every=500):
    it = 0
    while it < max_iter:
        orc.iterate(every)
        it += every
        r = orc.residuals()
        if r["kkt"] < tol:
            return r, it
    return orc.residuals(), it


def vertex_enumeration(A, b, c):
    m, n = A.shape
    best, xbest = np.inf, None
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-12:
            continue
        xB = np.linalg.solve(AB, b)
        if xB.min() < -1e-12:
            continue
        x = np.zeros(n)
        x[list(B)] = xB
        if c @ x < best:
            best, xbest = c @ x, x
    return best, xbest


@pytest.mark.parametrize("seed", range(6))
def test_tiny_lp_matches_vertex_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(1, 4)), int(rng.integers(4, 9))
    A = rng.standard_normal((m, n))
    A[rng.random((m, n)) < 0.2] = 0.0
    A[:, 0] = np.where(A[:, 0] == 0, 1.0, A[:, 0])
    x0 = rng.uniform(0.2, 1.0, n)
    b = A @ x0
    c = A.T @ rng.standard_normal(m) + rng.uniform(0.1, 1.0, n)
    best, xbest = vertex_enumeration(A, b, c)
    orc = lp_problem(A, b, c)
    r, it = run_to(orc, 1e-11, 400_000)
    assert r["kkt"] < 1e-11, (r, it)
    assert abs(r["pobj"] - best) < 1e-8 * (1 + abs(best))
    np.testing.assert_allclose(orc.state().x, xbest, atol=1e-7)


def test_identity_constraints_closed_form():
    rng = np.random.default_rng(11)
    n = 6
    b = rng.uniform(0.5, 1.5, n)
    c = rng.standard_normal(n)
    orc = lp_problem(np.eye(n), b, c)
    r, _ = run_to(orc, 1e-12, 200_000)
    s = orc.state()
    np.testing.assert_allclose(s.x, b, atol=1e-10)
    np.testing.assert_allclose(s.lam, -c, atol=1e-10)


def test_single_lorentz_cone_closed_form():
    c = np.array([0.3, -1.2, 0.5])
    A = np.array([[1.0, 0.0, 0.0]])
    orc = lp_problem(A, np.array([1.0]), c, cones=[(1, 3)])
    r, _ = run_to(orc, 1e-12, 400_000)
    cb = c[1:]
    x_star = np.concatenate([[1.0], -cb / np.linalg.norm(cb)])
    np.testing.assert_allclose(orc.state().x, x_star, atol=1e-8)
    assert abs(r["pobj"] - (c[0] - np.linalg.norm(cb))) < 1e-9
    np.testing.assert_allclose(orc.state().lam, [np.linalg.norm(cb) - c[0]], atol=1e-8)


@pytest.mark.parametrize("m,n,tol,iters,obj_tol", [(20, 50, 1e-9, 400_000, 1e-7),
                                                    (200, 500, 1e-5, 100_000, 1e-5)])
def test_small_lp_matches_highs(m, n, tol, iters, obj_tol):
    """The literal iteration reaches the LP optimum that HiGHS (scipy.optimize.linprog) finds.
    The method's fixed-mu ADMM converges slowly, so the full-size small LP is checked at the
    accuracy it reaches in 1e5 iterations."""
    from scipy.optimize import linprog
    prob = I.small_lp(0, m=m, n=n)
    orc = oracle.make_oracle(prob)
    A = sp.coo_matrix((prob["val"], (prob["row"], prob["col"])), shape=(prob["m"], prob["n"])).tocsr()
    ref = linprog(prob["c"], A_eq=A, b_eq=prob["b"], bounds=(0, None), method="highs")
    assert ref.status == 0
    r, it = run_to(orc, tol, iters, every=5000)
    assert r["kkt"] < tol, (r, it)
    assert abs(r["pobj"] - ref.fun) < obj_tol * (1 + abs(ref.fun))
    assert abs(r["dobj"] - ref.fun) < obj_tol * (1 + abs(ref.fun))


# ---------------------------------------------------------------- residuals

def test_residual_norms_match_library_products():
    prob = I.socp(seed=1, n=300, m=120, nnz_per_row=6)
    orc = oracle.make_oracle(prob)
    rng = np.random.default_rng(5)
    x = rng.standard_normal(prob["n"])
    lam = rng.standard_normal(prob["m"])
    orc.set_state(x=x, lam=lam)
    r = orc.residuals()
    A = sp.coo_matrix((prob["val"], (prob["row"], prob["col"])), shape=(prob["m"], prob["n"])).tocsr()
    res = A @ x - prob["b"]
    s = A.T @ lam + prob["c"]
    assert np.isclose(r["nrm_res_p"], np.linalg.norm(res), rtol=1e-13)
    assert np.isclose(r["nrm_atl_c"], np.linalg.norm(s), rtol=1e-13)
    assert np.isclose(r["inf_res_p"], np.abs(res).max(), rtol=1e-13)
    assert np.isclose(r["pobj"], prob["c"] @ x, rtol=1e-13)
    assert np.isclose(r["dobj"], -prob["b"] @ lam, rtol=1e-13)
    # distance to K of s: Moreau gives s - P_K(s) = -P_K(-s)
    ps_neg = orc.proj_K(-s)
    assert np.isclose(r["nrm_sdist"], np.linalg.norm(ps_neg), rtol=1e-12)
    assert np.isclose(r["r_prim"], np.linalg.norm(res) / (1 + np.linalg.norm(prob["b"])), rtol=1e-13)


def spectral_proj_lorentz(w):
    """Projection on one Lorentz cone through its spectral decomposition (the Jordan algebra of the
    cone): w = l1 u1 + l2 u2 with l1,2 = w1 -/+ ||wbar||, u1,2 = (1, -/+ wbar/||wbar||)/2, and the
    projection keeps max(l, 0) of each eigenvalue. Independent of the case split of eq. proj."""
    w = np.asarray(w, float)
    if w.size == 1:
        return np.maximum(w, 0.0)
    a = np.linalg.norm(w[1:])
    d = w[1:] / a if a > 0 else np.zeros(w.size - 1)
    u1 = np.concatenate([[0.5], -0.5 * d])
    u2 = np.concatenate([[0.5], 0.5 * d])
    return max(w[0] - a, 0.0) * u1 + max(w[0] + a, 0.0) * u2


def spectral_proj_K(cones, w):
    out, o = np.empty_like(w), 0
    for kind, size in cones:
        seg = w[o:o + size]
        out[o:o + size] = np.maximum(seg, 0.0) if kind == 0 else spectral_proj_lorentz(seg)
        o += size
    return out


def test_infinity_norm_distances_match_spectral_projection():
    prob = I.socp(seed=3, n=300, m=120, nnz_per_row=6)
    orc = oracle.make_oracle(prob)
    rng = np.random.default_rng(6)
    cones = [tuple(map(int, q)) for q in np.asarray(prob["cones"]).reshape(-1, 2)]
    A = sp.coo_matrix((prob["val"], (prob["row"], prob["col"])), shape=(prob["m"], prob["n"])).tocsr()
    for _ in range(5):
        x = rng.standard_normal(prob["n"]) * rng.choice([0.1, 1.0, 10.0])
        lam = rng.standard_normal(prob["m"])
        orc.set_state(x=x, lam=lam)
        r = orc.residuals()
        s = A.T @ lam + prob["c"]
        dx = x - spectral_proj_K(cones, x)
        ds = s - spectral_proj_K(cones, s)
        assert np.isclose(r["inf_x"], np.abs(x).max(), rtol=1e-15)
        assert np.isclose(r["inf_xdist"], np.abs(dx).max(), rtol=1e-12, atol=1e-14)
        assert np.isclose(r["inf_sdist"], np.abs(ds).max(), rtol=1e-12, atol=1e-14)
        # norm inequalities between the l2 and infinity forms
        assert r["inf_xdist"] <= r["nrm_xdist"] * (1 + 1e-14) <= np.sqrt(prob["n"]) * r["inf_xdist"] * (1 + 1e-12)
        assert r["inf_sdist"] <= r["nrm_sdist"] * (1 + 1e-14) <= np.sqrt(prob["n"]) * r["inf_sdist"] * (1 + 1e-12)


def test_stop_measures_vanish_at_an_exact_optimum():
    """At HiGHS's optimal primal-dual pair both rules read 0 (to rounding), while the printed dual
    residual ||A^T lambda + c|| does not: the cone multiplier must come out of it."""
    from scipy.optimize import linprog
    prob = I.small_lp(1)
    A = sp.coo_matrix((prob["val"], (prob["row"], prob["col"])), shape=(prob["m"], prob["n"])).tocsr()
    ref = linprog(prob["c"], A_eq=A, b_eq=prob["b"], bounds=(0, None), method="highs",
                  options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    assert ref.status == 0
    x = np.maximum(ref.x, 0.0)
    lam = -ref.eqlin.marginals          # HiGHS: c - A^T y >= 0; here c + A^T lambda in K
    orc = oracle.make_oracle(prob)
    orc.set_state(x=x, lam=lam)
    r = orc.residuals()
    assert r["r_scs"] < 1e-8 and r["r_osqp"] < 1e-8
    assert r["nrm_atl_c"] / (1 + r["nrm_c"]) > 1e-2


def test_stop_measures_reduce_to_the_printed_rules():
    """With x in K (no cone violation) and s = A^T lambda + c in the polar cone (P_K s = 0), the two
    measures are the printed SCS and OSQP tests, and "measure <= eps" holds exactly when the printed
    inequalities hold with eps_abs = eps and eps_rel = q eps."""
    rng = np.random.default_rng(7)
    prob = I.small_lp(2)
    A = sp.coo_matrix((prob["val"], (prob["row"], prob["col"])), shape=(prob["m"], prob["n"])).toarray()
    b = prob["b"]
    for trial in range(20):
        x = np.abs(rng.standard_normal(prob["n"])) * rng.choice([1e-3, 1.0])
        lam = rng.standard_normal(prob["m"]) * 0.01
        c = -np.abs(rng.standard_normal(prob["n"])) - np.abs(A.T @ lam) - 0.1   # s <= 0 elementwise
        p = dict(prob, c=c)
        orc = oracle.make_oracle(p)
        orc.set_state(x=x, lam=lam)
        q = float(rng.choice([1.0, 10.0, 100.0]))
        r = orc.residuals(osqp_rel=q)
        res, s = A @ x - b, A.T @ lam + c
        scs = max(np.linalg.norm(res) / (1 + np.linalg.norm(b)), np.linalg.norm(s) / (1 + np.linalg.norm(c)),
                  abs(c @ x + b @ lam) / (1 + abs(c @ x) + abs(b @ lam)))
        assert np.isclose(r["r_scs"], scs, rtol=1e-12)
        for eps in np.geomspace(1e-6, 10.0, 15):
            ok = (np.abs(res).max() <= eps + q * eps * max(np.abs(A @ x).max(), np.abs(b).max(), np.abs(x).max())
                  and np.abs(s).max() <= eps + q * eps * max(np.abs(A.T @ lam).max(), np.abs(c).max()))
            assert (r["r_osqp"] <= eps) == ok or abs(r["r_osqp"] - eps) < 1e-12 * eps


# ---------------------------------------------------------------- reduced form vs literal form

@pytest.mark.parametrize("maker", ["small_lp", "socp"])
def test_reduced_form_tracks_literal_iteration(maker):
    prob = I.small_lp(0) if maker == "small_lp" else I.socp(seed=2, n=400, m=150, nnz_per_row=5)
    orc = oracle.make_oracle(prob, mu=1.0)
    red = Reduced(prob, mu=1.0)
    for _ in range(4):
        orc.iterate(500)
        red.iterate(500)
        s = orc.state()
        for name, a, bb in (("x", red.x, s.x), ("z", red.z, s.z), ("delta", red.delta, s.delta),
                            ("lam", red.lam, s.lam)):
            err = np.abs(a - bb).max() / max(1.0, np.abs(bb).max())
            assert err < 1e-12, (name, err)


@pytest.mark.parametrize("maker", ["small_lp", "socp"])
def test_literal_state_from_a_reduced_state(maker):
    """Seeding Algorithm 1 from an arbitrary reduced state (x, z, delta, lambda, v) -- v not the one
    (x, lambda) imply -- makes the literal iteration follow the separately written reduced loop
    started from the same state; with v = F_U (b - A x) - lambda/mu the seeded y and gamma are the
    C oracle's consistent warm-start state."""
    prob = I.small_lp(1, m=40, n=100) if maker == "small_lp" else I.socp(seed=3, n=300, m=120, nnz_per_row=5)
    mu = 1.7
    rng = np.random.default_rng(5)
    n, m = prob["n"], prob["m"]
    x, z, d = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal(n)
    lam, v = rng.standard_normal(m), rng.standard_normal(m)
    orc = oracle.make_oracle(prob, mu=mu)
    red = Reduced(prob, mu=mu)
    red.x, red.z, red.delta, red.lam, red.v = x.copy(), z.copy(), d.copy(), lam.copy(), v.copy()
    orc.set_reduced_state(x, z, d, lam, v)
    orc.iterate(300)
    red.iterate(300)
    s = orc.state()
    for name, a, bb in (("x", red.x, s.x), ("z", red.z, s.z), ("delta", red.delta, s.delta), ("lam", red.lam, s.lam)):
        assert np.abs(a - bb).max() <= 1e-12 * max(1.0, np.abs(bb).max()), name
    rho = (red.b - red.A @ x) / (1.0 + red.r)
    orc.set_reduced_state(x, z, d, lam, rho - lam / mu)
    y, g = orc.consistent_y_gamma(x, lam)
    s = orc.state()
    assert np.allclose(s.y, y, rtol=0, atol=1e-13) and np.array_equal(s.gam, g)


# ---------------------------------------------------------------- residual-balanced mu (a variant)

@pytest.mark.parametrize("mu0", [1.0, 1e-3, 1e3])
def test_balanced_mu_reaches_the_original_optimum(mu0):
    """Residual balancing changes only the penalty, not the problem: from any starting mu the
    iteration converges to the LP optimum HiGHS finds, and a badly chosen mu is moved towards
    balance (raised from 1e-3, lowered from 1e3) rather than further away."""
    from scipy.optimize import linprog
    prob = I.small_lp(0, m=20, n=50)
    A = sp.coo_matrix((prob["val"], (prob["row"], prob["col"])), shape=(prob["m"], prob["n"])).tocsr()
    ref = linprog(prob["c"], A_eq=A, b_eq=prob["b"], bounds=(0, None), method="highs")
    assert ref.status == 0
    orc = oracle.make_oracle(prob, mu=mu0)
    it, hist = oracle.solve_balanced(orc, 1e-9, 400_000, 25, 4)
    r = orc.residuals()
    assert r["kkt"] <= 1e-9, (it, r["kkt"])
    assert abs(r["pobj"] - ref.fun) < 1e-7 * (1 + abs(ref.fun))
    mus = np.array([h[2] for h in hist])
    assert mus.min() >= mu0 / 256 * (1 - 1e-12) and mus.max() <= mu0 * 256 * (1 + 1e-12)
    if mu0 < 1e-2:
        assert mus[-1] > 10 * mu0
    if mu0 > 1e2:
        assert mus[-1] < 0.1 * mu0


def test_balanced_mu_off_is_the_fixed_mu_iteration():
    prob = I.small_lp(1, m=30, n=80)
    a, b = oracle.make_oracle(prob), oracle.make_oracle(prob)
    it, hist = oracle.solve_balanced(a, 1e-30, 1000, 25, 0)
    b.iterate(1000)
    assert it == 1000 and all(h[2] == 1.0 for h in hist)
    assert np.array_equal(a.state().x, b.state().x) and np.array_equal(a.state().lam, b.state().lam)
