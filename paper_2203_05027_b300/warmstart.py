"""Learned warm start for a parametric LP family.

The family: A fixed (m rows, n columns, a fixed number of nonzeros per column, N(0,1) values),
x0 ~ U[0,1]^n, y0 ~ N(0,1)^m, s0 ~ U[0,1]^n, b0 = A x0, c0 = A^T y0 + s0, K = R^n_+; the
parameter theta ~ N(0, I_p) moves b = b0 + B_b theta and c = c0 + B_c theta, with B_b, B_c
having i.i.d. N(0, sigma^2) entries. Solutions (x, lambda) of sampled members, produced by the
shared-A solver (mfs_shared_*), train the tensor-core MLP (mfs_mlp_*) theta -> (x, lambda);
its prediction then warm-starts the solver (mfs_shared_warm_start_device). Two starts that need no
network, made from the same training solves, are measured beside it: their mean, and the solution
of the training member whose theta is nearest.

Every arithmetic step of solving and training runs in libmfs; this module draws the seeded
family (numpy), moves buffers and records counts, times and prediction errors; torch provides
device memory.
"""
from __future__ import annotations

import time

import numpy as np

from . import instances as I
from . import mfs


def family(seed=0, m=20_000, n=50_000, nnz_per_col=8, p=32, sigma=0.1):
    base = I.lp_from_degrees(m, n, np.full(n, nnz_per_col), [seed, 40], name=f"param_lp_m{m}_n{n}")
    rng = np.random.default_rng([seed, 41])
    Bb = rng.normal(0.0, sigma, (m, p))
    Bc = rng.normal(0.0, sigma, (n, p))
    return {"base": base, "Bb": Bb, "Bc": Bc, "p": p}


def thetas(count, seed, p=32):
    return np.random.default_rng([seed, 42]).standard_normal((count, p))


def data_of(fam, theta):
    base = fam["base"]
    b = base["b"][None, :] + theta @ fam["Bb"].T
    c = base["c"][None, :] + theta @ fam["Bc"].T
    return b, c


def generate(fam, count, seed, tol, max_iter, batch=512, check_every=250):
    """Training data: theta (count x p, FP32) and targets [x | lambda] (count x (n+m), FP32) on the
    device, from cold-start solves to tol with at most max_iter iterations (the iterate is kept either
    way). Continuous batching: `batch` slots of the shared-A solver iterate together; every
    check_every iterations the members that are done leave their slots and the next members enter.
    Returns (theta, targets, iterations per member (-1 if it missed tol), seconds)."""
    import torch
    base = fam["base"]
    n, m = base["n"], base["m"]
    th = thetas(count, seed, fam["p"])
    T = torch.empty((count, n + m), dtype=torch.float32, device="cuda")
    slots = min(batch, count)
    sh = mfs.Shared(base, slots, check_every=check_every, precision="fp32")
    X = torch.empty((slots, n), dtype=torch.float32, device="cuda")
    L = torch.empty((slots, m), dtype=torch.float32, device="cuda")
    member = np.full(slots, -1)
    age = np.zeros(slots, np.int64)
    iters = np.full(count, -1, np.int64)
    nxt = 0

    def enter(sl):
        nonlocal nxt
        idx = np.arange(nxt, nxt + len(sl))
        nxt += len(sl)
        b, c = data_of(fam, th[idx])
        bd = torch.from_numpy(b.astype(np.float32)).cuda()
        cd = torch.from_numpy(c.astype(np.float32)).cuda()
        sh.load_slots(sl, bd.data_ptr(), cd.data_ptr())
        member[sl] = idx
        age[sl] = 0

    t0 = time.perf_counter()
    enter(np.arange(slots))
    done = 0
    while done < count:
        sh.iterate(check_every)
        age += check_every
        kkt = np.array([r["kkt"] for r in sh.residuals()])
        met = kkt <= tol
        fin = np.where((member >= 0) & (met | (age >= max_iter)))[0]
        if len(fin):
            sh.slots_device(fin, X.data_ptr(), L.data_ptr())
            rows = torch.from_numpy(member[fin]).cuda()
            T[rows, :n] = X[:len(fin)]
            T[rows, n:] = L[:len(fin)]
            iters[member[fin]] = np.where(met[fin], age[fin], -1)
            done += len(fin)
            member[fin] = -1
            k = min(len(fin), count - nxt)
            if k:
                enter(fin[:k])
    torch.cuda.synchronize()
    sh.close()
    theta = torch.from_numpy(th.astype(np.float32)).cuda()
    return theta, T, iters, time.perf_counter() - t0


def train_fn(net, theta, T, epochs, lr, batch, lr_final=None):
    """Minibatch Adam over the training rows (already i.i.d. draws, taken in order), the step size
    falling from lr to lr_final (default lr / 20) along a cosine over the epochs."""
    import math
    import torch
    lr_final = lr / 20 if lr_final is None else lr_final
    count = theta.shape[0]
    losses = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * ep / max(epochs - 1, 1)))
        tot, steps = 0.0, 0
        for s0 in range(0, count - batch + 1, batch):
            tot += net.train_step(batch, theta[s0].data_ptr(), T[s0].data_ptr(), a)
            steps += 1
        losses.append(tot / max(steps, 1))
    torch.cuda.synchronize()
    return losses, time.perf_counter() - t0


def eval_loss(net, theta, T, batch):
    """Mean squared error on standardised targets (no update), averaged over full batches."""
    count = theta.shape[0]
    tot, steps = 0.0, 0
    for s0 in range(0, count - batch + 1, batch):
        tot += net.backward(batch, theta[s0].data_ptr(), T[s0].data_ptr())
        steps += 1
    return tot / max(steps, 1)


def predict(net, theta, n, m):
    """MLP prediction (denormalised) split into contiguous x [count][n] and lambda [count][m]."""
    import torch
    count = theta.shape[0]
    Y = torch.empty((count, n + m), dtype=torch.float32, device="cuda")
    for s0 in range(0, count, net.max_batch):
        k = min(net.max_batch, count - s0)
        net.forward(k, theta[s0].data_ptr(), Y[s0].data_ptr(), denormalize=True)
    return Y[:, :n].contiguous(), Y[:, n:].contiguous()


def solve_stream(fam, theta, tol, max_iter, slots=256, check_every=100, warm=None, mu=1.0, precision="fp32",
                 keep=False):
    """Solve the members theta (count x p, host) to tol by continuous batching: `slots` members
    iterate together, each leaves at its first check with relative KKT <= tol (or at max_iter) and
    the next member enters its slot, from the zero start or, with warm = (X, L) (device FP32
    [count][n] and [count][m]), from its row of X and L. Returns (iterations per member, -1 where
    max_iter was reached first; kkt of each member at entry; seconds; with keep, each member's final
    x [count][n] and lambda [count][m] on the device, else None, None)."""
    import torch
    base = fam["base"]
    count = theta.shape[0]
    slots = min(slots, count)
    sh = mfs.Shared(base, slots, mu=mu, check_every=check_every, precision=precision)
    member = np.full(slots, -1)
    age = np.zeros(slots, np.int64)
    iters = np.full(count, -1, np.int64)
    kkt0 = np.full(count, np.nan)
    n, m = base["n"], base["m"]
    Xo = torch.empty((count, n), dtype=torch.float32, device="cuda") if keep else None
    Lo = torch.empty((count, m), dtype=torch.float32, device="cuda") if keep else None
    Xs = torch.empty((slots, n), dtype=torch.float32, device="cuda") if keep else None
    Ls = torch.empty((slots, m), dtype=torch.float32, device="cuda") if keep else None
    nxt = 0

    def enter(sl):
        nonlocal nxt
        idx = np.arange(nxt, nxt + len(sl))
        nxt += len(sl)
        b, c = data_of(fam, theta[idx])
        bd = torch.from_numpy(b.astype(np.float32)).cuda()
        cd = torch.from_numpy(c.astype(np.float32)).cuda()
        if warm is None:
            sh.load_slots(sl, bd.data_ptr(), cd.data_ptr())
        else:
            rows = torch.from_numpy(idx).cuda()
            if isinstance(warm, _RowStart):
                xw, lw = warm[rows]
                xw, lw = xw.contiguous(), lw.contiguous()
            else:
                xw, lw = warm[0][rows].contiguous(), warm[1][rows].contiguous()
            sh.load_slots_warm(sl, bd.data_ptr(), cd.data_ptr(), xw.data_ptr(), lw.data_ptr())
        member[sl] = idx
        age[sl] = 0
        res = sh.residuals()
        kkt0[idx] = [res[q]["kkt"] for q in sl]

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    enter(np.arange(slots))
    done = 0
    while done < count:
        sh.iterate(check_every)
        age += check_every
        kkt = np.array([r["kkt"] for r in sh.residuals()])
        met = kkt <= tol
        fin = np.where((member >= 0) & (met | (age >= max_iter)))[0]
        if len(fin):
            iters[member[fin]] = np.where(met[fin], age[fin], -1)
            if keep:
                sh.slots_device(fin, Xs.data_ptr(), Ls.data_ptr())
                rows = torch.from_numpy(member[fin]).cuda()
                Xo[rows] = Xs[:len(fin)]
                Lo[rows] = Ls[:len(fin)]
            done += len(fin)
            member[fin] = -1
            k = min(len(fin), count - nxt)
            if k:
                enter(fin[:k])
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    sh.close()
    return iters, kkt0, sec, Xo, Lo


def mean_start(T, n):
    """Non-learned start: the mean training target (x-bar, lambda-bar), the same for every member."""
    mu = T.mean(dim=0, keepdim=True)
    return mu[:, :n].contiguous(), mu[:, n:].contiguous()


def nearest_start(theta_train, T, theta, n, chunk=4096):
    """Non-learned start: for each member, the training target of the training theta nearest to its
    own (Euclidean distance in parameter space). theta_train: device FP32 [count][p]; theta: host
    [members][p]. Returns device row indices into T (the starts are gathered when a member enters)."""
    import torch
    q = torch.from_numpy(np.ascontiguousarray(theta, np.float32)).cuda()
    best = torch.empty(q.shape[0], dtype=torch.int64, device="cuda")
    for s0 in range(0, q.shape[0], chunk):
        d = torch.cdist(q[s0:s0 + chunk].double(), theta_train.double())
        best[s0:s0 + chunk] = d.argmin(dim=1)
    return best


class _RowStart:
    """A start given as rows of a target matrix T ([count][n + m]): member i starts from row idx[i]
    (idx None: the same single row 0 of X and L for all)."""

    def __init__(self, X, L, idx=None):
        self.X, self.L, self.idx = X, L, idx

    def __getitem__(self, k):
        import torch
        rows = k if self.idx is None else self.idx[k]
        if self.idx is None:
            rows = torch.zeros_like(k)
        return (self.X[rows], self.L[rows])


def evaluate(fam, net, theta, tol, max_iter, mu=1.0, check_every=100, precision="fp32", slots=256, starts=None):
    """Cold start against warm starts on the members theta (count x p, host), each arm solved by
    continuous batching (solve_stream): per member, the iteration at which the relative KKT residual
    first met tol (-1 if never within max_iter) and the KKT at entry, and the wall time for the whole
    set. Arms: "cold" (zero start), "mlp" (the network's prediction; its inference time included) and
    any further named starts (pairs of device FP32 arrays [count][n], [count][m], or _RowStart)."""
    import torch
    base = fam["base"]
    n, m = base["n"], base["m"]
    out = {}
    its, k0, sec, Xc, Lc = solve_stream(fam, theta, tol, max_iter, slots, check_every, None, mu, precision, keep=True)
    out["cold"] = {"iters": its, "seconds": sec, "kkt0": k0}
    th = torch.from_numpy(np.ascontiguousarray(theta, np.float32)).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xw, Lw = predict(net, th, n, m)
    torch.cuda.synchronize()
    t_pred = time.perf_counter() - t0
    arms = {"mlp": (Xw, Lw)}
    arms.update(starts or {})
    for name, st in arms.items():
        its, k0, sec, _, _ = solve_stream(fam, theta, tol, max_iter, slots, check_every, st, mu, precision)
        rec = {"iters": its, "seconds": sec + (t_pred if name == "mlp" else 0.0), "kkt0": k0}
        if name == "mlp":
            rec["predict_seconds"] = t_pred
        # error of the start against the point where the cold arm ended (per member)
        rows = torch.arange(theta.shape[0], device="cuda")
        Xs, Ls = st[rows] if isinstance(st, _RowStart) else st
        rec["rel_err_x"] = (torch.linalg.vector_norm(Xs - Xc, dim=1) /
                            torch.linalg.vector_norm(Xc, dim=1).clamp_min(1e-30)).cpu().numpy()
        rec["rel_err_lam"] = (torch.linalg.vector_norm(Ls - Lc, dim=1) /
                              torch.linalg.vector_norm(Lc, dim=1).clamp_min(1e-30)).cpu().numpy()
        out[name] = rec
    return out


def _its_summary(a):
    a = np.asarray(a)
    ok = a[a >= 0]
    return {"converged": int(ok.size), "of": int(a.size),
            "mean": float(ok.mean()) if ok.size else None,
            "median": float(np.median(ok)) if ok.size else None,
            "p90": float(np.percentile(ok, 90)) if ok.size else None}


def run(train=50_000, test=1000, m=20_000, n=50_000, nnz_per_col=8, p=32, sigma=0.1, seed=0, data_tol=1e-3,
        data_cap=10_000, data_batch=512, width=512, epochs=100, lr=1e-3, batch=256, eval_tol=1e-6,
        eval_cap=250_000, mu=1.0, single=0, log=print):
    """The whole experiment: generate, fit, train, evaluate warm against cold on held-out members,
    and (single > 0) time that many plain one-at-a-time cold solves. Logs one dict per stage and
    returns the evaluation summary."""
    import json
    import torch
    fam = family(seed, m, n, nnz_per_col, p, sigma)
    base = fam["base"]
    theta, T, its, sec = generate(fam, train, seed + 1, data_tol, data_cap, batch=data_batch)
    log(json.dumps({"stage": "data", "solves": train, "tol": data_tol, "cap": data_cap, "seconds": sec,
                    **_its_summary(its)}))
    thv, Tv, _, _ = generate(fam, max(batch, 512), seed + 5, data_tol, data_cap, batch=max(batch, 512))
    net = mfs.MLP(p, width, n + m, batch, seed=seed)
    net.fit_output_scaling(train, T.data_ptr(), 1e-3)
    losses, tsec = train_fn(net, theta, T, epochs, lr, batch)
    val = eval_loss(net, thv, Tv, batch)
    log(json.dumps({"stage": "train", "epochs": epochs, "steps": epochs * (train // batch), "seconds": tsec,
                    "loss_first": losses[0], "loss_last": losses[-1], "val_loss": val}))
    del Tv
    th_test = thetas(test, seed + 7, p)
    # non-learned starts from the same training solves: their mean, and the nearest training theta's
    Xmean, Lmean = mean_start(T, n)
    near = nearest_start(theta, T, th_test, n)
    starts = {"mean": _RowStart(Xmean, Lmean), "nearest": _RowStart(T[:, :n], T[:, n:], near)}
    res = evaluate(fam, net, th_test, eval_tol, eval_cap, mu=mu, starts=starts)
    summary = {"stage": "evaluate", "tol": eval_tol, "cap": eval_cap, "members": test,
               "train_solves": train, "train_tol": data_tol, "train_cap": data_cap}
    ic = res["cold"]["iters"]
    for arm in ("cold", "mlp", "mean", "nearest"):
        r = res[arm]
        summary[arm] = {"seconds": r["seconds"], "kkt0_median": float(np.median(r["kkt0"])),
                        **_its_summary(r["iters"])}
        if arm != "cold":
            iw = r["iters"]
            both = (ic > 0) & (iw > 0)
            summary[arm]["paired"] = int(both.sum())
            summary[arm]["iters_ratio_median"] = float(np.median(iw[both] / ic[both])) if both.any() else None
            summary[arm]["rel_err_x_median"] = float(np.median(r["rel_err_x"]))
            summary[arm]["rel_err_lam_median"] = float(np.median(r["rel_err_lam"]))
    summary["mlp"]["predict_seconds"] = res["mlp"]["predict_seconds"]
    del T
    torch.cuda.empty_cache()
    log(json.dumps(summary))
    if single > 0:
        b, c = data_of(fam, th_test[:single])
        secs, iters = [], []
        for t in range(single):
            prob = dict(base, b=b[t], c=c[t])
            s = mfs.Solver(prob, mu=mu, check_every=100, precision="fp32")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, it = s.solve(eval_tol, eval_cap)
            torch.cuda.synchronize()
            secs.append(time.perf_counter() - t0)
            iters.append(it)
            s.close()
        log(json.dumps({"stage": "single_cold", "solves": single, "seconds_mean": float(np.mean(secs)),
                        "iters": iters}))
        summary["single_cold_seconds_mean"] = float(np.mean(secs))
    return summary


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="learned warm start: generate, train, evaluate warm vs cold")
    for k, v in (("train", 50_000), ("test", 1000), ("m", 20_000), ("n", 50_000), ("nnz_per_col", 8), ("p", 32),
                 ("seed", 0), ("data_cap", 10_000), ("data_batch", 512), ("width", 512), ("epochs", 100),
                 ("batch", 256), ("eval_cap", 250_000), ("single", 0)):
        ap.add_argument("--" + k.replace("_", "-"), type=int, default=v)
    for k, v in (("sigma", 0.1), ("data_tol", 1e-3), ("lr", 1e-3), ("eval_tol", 1e-6), ("mu", 1.0)):
        ap.add_argument("--" + k.replace("_", "-"), type=float, default=v)
    a = ap.parse_args(argv)
    mfs.load()
    run(**vars(a), log=lambda s: print(s, flush=True))


if __name__ == "__main__":
    main()
