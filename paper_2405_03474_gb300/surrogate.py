"""Surrogate of log det over GP hyperparameters, trained on the estimator's own values.

An addition to the paper's method for hyperparameter search: the MLP of
``csrc/mlp.cu`` maps (log lengthscale, log variance, log noise, log n) to
log det M / n.  Labels come from ``logdet_estimate`` (r_3, randomized-SVD
preconditioner) on the GPU; the estimator stays the fallback (queries outside
the training box) and the reference its error is measured against (audits on
random queries).

Run ``python -m paper_2405_03474_gb300.surrogate --help`` for the label job of the
``surrogate_matern_n262144_d3`` workload (checkpointed to an .npz, resumable).
"""
import argparse
import os
import time

import numpy as np
import torch

from . import _lib, api, inputs


def features(theta, n):
    """(K x 3) hyperparameters (l, v, nu) -> (K x 4) float32 network inputs."""
    theta = np.asarray(theta, dtype=np.float64)
    logn = np.full((theta.shape[0], 1), np.log(float(n)))
    return np.hstack([np.log(theta), logn]).astype(np.float32)


def in_box(theta, box=inputs.THETA_BOX, slack=1e-9):
    """Mask of hyperparameters inside the training box."""
    theta = np.asarray(theta, dtype=np.float64)
    lo = np.array([box["lengthscale"][0], box["variance"][0], box["noise"][0]]) * (1 - slack)
    hi = np.array([box["lengthscale"][1], box["variance"][1], box["noise"][1]]) * (1 + slack)
    return np.all((theta >= lo) & (theta <= hi), axis=1)


class Estimator:
    """The plain estimator at one point cloud: log det M(theta) / n on the GPU."""

    def __init__(self, X, kind, rank=64, power_iters=1, probes=16, t=20, order=3, precision="f16x3_tc",
                 sketch_precision="f16_tc", seed=1):
        self.X = X
        self.n = X.shape[0]
        self.kind, self.rank, self.power_iters = kind, rank, power_iters
        self.opts = dict(order=order, num_probes=probes, probes_per_block=probes, fixed_iters=t, max_iters=t,
                         precision=precision, seed=seed)
        self.sketch_precision = sketch_precision

    def __call__(self, theta):
        """log det / n at theta, or NaN where the operator in the estimator's precision
        is not positive definite (LD_ERR_NOT_SPD from the preconditioner's Cholesky or
        from the CG: the rounding of K exceeds the noise, which happens at the box's
        long-lengthscale, low-noise corner)."""
        l, v, nu = (float(x) for x in theta)
        kern = api.Kernel(self.kind, l, v, nu)
        try:
            P = api.Precond.build(self.X, kern, self.rank, power_iters=self.power_iters, seed=inputs.SEED_SKETCH,
                                  precision=self.sketch_precision)
        except _lib.LogdetError as e:
            if e.status != _lib.LD_ERR_NOT_SPD:
                raise
            return float("nan")
        try:
            res = api.logdet_estimate(self.X, kern, precond=P, **self.opts)
        except _lib.LogdetError as e:
            if e.status != _lib.LD_ERR_NOT_SPD:
                raise
            return float("nan")
        finally:
            P.free()
        return res["logdet"] / self.n


def generate_labels(est, thetas, checkpoint=None, every=32, log=None):
    """Labels est(theta) for each row of thetas, saved every `every` labels to
    `checkpoint` (.npz with thetas, labels, done) and resumed from it: the labels
    already done are reused when their thetas are the first rows of `thetas`, so a
    job also extends a shorter run of the same Sobol sequence."""
    thetas = np.asarray(thetas, dtype=np.float64)
    labels = np.full(len(thetas), np.nan)
    done = 0
    if checkpoint and os.path.exists(checkpoint):
        z = np.load(checkpoint)
        k = min(int(z["done"]), len(thetas))
        if z["thetas"].shape[1:] == thetas.shape[1:] and np.array_equal(z["thetas"][:k], thetas[:k]):
            labels[:k] = z["labels"][:k]
            done = k
    t0 = time.perf_counter()
    for i in range(done, len(thetas)):
        labels[i] = est(thetas[i])
        if checkpoint and ((i + 1) % every == 0 or i + 1 == len(thetas)):
            np.savez(checkpoint + ".tmp.npz", thetas=thetas, labels=labels, done=i + 1)
            os.replace(checkpoint + ".tmp.npz", checkpoint)
            if log:
                log("labels %d/%d (%.1f s)" % (i + 1, len(thetas), time.perf_counter() - t0))
    return labels


class HyperSurrogate:
    """Trained network plus the estimator as fallback and as the reference of its error."""

    def __init__(self, est, box=inputs.THETA_BOX, seed=0):
        self.est = est
        self.box = box
        self.net = api.Surrogate(seed=seed)
        self.device = est.X.device

    def fit(self, thetas, labels, epochs=400, batch=256, lr=2e-3):
        f = torch.as_tensor(features(thetas, self.est.n)).to(self.device)
        y = torch.as_tensor(np.asarray(labels, dtype=np.float32)).to(self.device)
        return self.net.train(f, y, epochs=epochs, batch=batch, lr=lr)

    def predict(self, thetas, want_grad=False):
        """log det / n for each theta; the estimator answers queries outside the box.
        With want_grad, also d(log det / n)/d(log l, log v, log nu)."""
        thetas = np.asarray(thetas, dtype=np.float64)
        f = torch.as_tensor(features(thetas, self.est.n)).to(self.device)
        if want_grad:
            out, dout = self.net.infer(f, want_grad=True)
            g = dout.cpu().numpy()[:, :3].astype(np.float64)
        else:
            out = self.net.infer(f)
            g = None
        pred = out.cpu().numpy().astype(np.float64)
        outside = ~in_box(thetas, self.box)
        for i in np.nonzero(outside)[0]:
            pred[i] = self.est(thetas[i])
        return (pred, g, outside) if want_grad else (pred, outside)

    def audit(self, thetas, tol):
        """Compare against the estimator on `thetas`; returns (max abs error, passed)."""
        pred, _ = self.predict(thetas)
        ref = np.array([self.est(t) for t in thetas])
        err = float(np.max(np.abs(pred - ref)))
        return err, err <= tol


def train_and_evaluate(est, thetas, labels, held_out=64, queries=65536, epochs=800, batch=128, lr=2e-3, seed=0):
    """Fit on labels, then report what the network gains: error against fresh
    estimator values on held-out hyperparameters, time per query of batched
    inference against time per estimate, and an audit."""
    thetas, labels = np.asarray(thetas), np.asarray(labels)
    ok = np.isfinite(labels)  # settings where the estimator's operator was not positive definite carry NaN
    hs = HyperSurrogate(est, seed=seed)
    t0 = time.perf_counter()
    loss = hs.fit(thetas[ok], labels[ok], epochs=epochs, batch=batch, lr=lr)
    t_fit = time.perf_counter() - t0
    test = inputs.sobol_theta(held_out, seed=101)
    t0 = time.perf_counter()
    ref = np.array([est(t) for t in test])
    t_est = (time.perf_counter() - t0) / held_out
    pred, _ = hs.predict(test)
    q = inputs.sobol_theta(queries, seed=202)
    hs.predict(q, want_grad=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hs.predict(q, want_grad=True)
    torch.cuda.synchronize()
    t_q = (time.perf_counter() - t0) / queries
    fin = np.isfinite(ref)
    err = np.abs(pred - ref)[fin]
    ref = ref[fin]
    return {"labels": int(len(labels)), "labels_not_spd": int((~ok).sum()), "train_loss_normalised": loss,
            "fit_s": t_fit, "held_out": held_out, "held_out_not_spd": int((~fin).sum()),
            "max_abs_err_logdet_per_n": float(err.max()),
            "mean_abs_err_logdet_per_n": float(err.mean()),
            "max_rel_err_logdet": float(np.max(err / np.abs(ref))),
            "label_spread": float(np.max(labels[ok]) - np.min(labels[ok])),
            "estimator_s_per_query": t_est, "surrogate_s_per_query_with_grad": t_q,
            "speedup_per_query": t_est / t_q, "queries": queries}


def main():
    ap = argparse.ArgumentParser(description="label job of the surrogate workload (checkpointed), "
                                             "then training and evaluation")
    ap.add_argument("--count", type=int, default=4096)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--checkpoint", default="surrogate_labels.npz")
    ap.add_argument("--rank", type=int, default=None)
    ap.add_argument("--power-iters", type=int, default=None)
    ap.add_argument("--t", type=int, default=20)
    ap.add_argument("--train", action="store_true", help="train and evaluate after labelling")
    args = ap.parse_args()
    w = inputs.WORKLOADS["surrogate_matern_n262144_d3"]
    n = args.n or w["n"]
    X = torch.as_tensor(inputs.points(n, w["d"], "uniform", seed=inputs.SEED_POINTS)).cuda()
    est = Estimator(X, w["kind"], rank=args.rank or w["rank"],
                    power_iters=w["power_iters"] if args.power_iters is None else args.power_iters,
                    probes=w["probes"], t=args.t)
    thetas = inputs.sobol_theta(args.count, seed=0)
    labels = generate_labels(est, thetas, checkpoint=args.checkpoint, log=print)
    if args.train:
        import json
        out = train_and_evaluate(est, thetas, labels)
        out.update({"n": n, "rank": est.rank, "power_iters": est.power_iters, "t": args.t,
                    "probes": w["probes"]})
        print(json.dumps(out))


if __name__ == "__main__":
    main()
