"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle.

This module holds no arithmetic of the estimator: only point clouds, probe
signs and hyperparameter samples drawn from numpy's PCG64 (and scipy's Sobol
sequence), with the shapes and distributions of the workloads below.  The
paper's own workload is synthetic too (Section 3: index points drawn from a
normal distribution; amplitude and lengthscale 1).

Workloads (name -> settings):

* ``matern_n2048_d2``     n=2048 uniform [0,1]^2, Matern-5/2, l=0.2, v=1,
                          nu=1e-2, r_3, rank 64, 32 probes, FP64 dense
* ``rbf_n65536_d3``       n=65536 N(0, I_3), RBF, l=0.5, v=1, nu=1e-3,
                          r_1/r_3/r_5, rank 256, 64 probes, stored dense FP32
* ``matern_n1048576_d4``  n=2^20 uniform [0,1]^4, Matern-5/2, l=0.1, v=1,
                          nu=1e-2, r_3, rank 512, 16 probes per block,
                          matrix-free
* ``rbf_grad_n131072_d2`` n=131072 uniform [0,1]^2, RBF, gradient in
                          (l in [0.05,1], v in [0.5,2], nu in [1e-4,1e-1])
* ``surrogate_matern_n262144_d3``  Matern-5/2 labels at n=262144 uniform
                          [0,1]^3 over Sobol samples of the same box

Seeds: points 0, probes 1, sketch 2 (per workload).
"""
import numpy as np

RBF = 0
MATERN52 = 1

WORKLOADS = {
    "matern_n2048_d2": dict(n=2048, d=2, dist="uniform", kind=MATERN52, lengthscale=0.2,
                            variance=1.0, noise=1e-2, order=3, rank=64, probes=32,
                            power_iters=5),
    "rbf_n65536_d3": dict(n=65536, d=3, dist="normal", kind=RBF, lengthscale=0.5,
                          variance=1.0, noise=1e-3, order=3, rank=256, probes=64,
                          power_iters=5),
    "matern_n1048576_d4": dict(n=1 << 20, d=4, dist="uniform", kind=MATERN52,
                               lengthscale=0.1, variance=1.0, noise=1e-2, order=3,
                               rank=512, probes=16, power_iters=2),
    "rbf_grad_n131072_d2": dict(n=131072, d=2, dist="uniform", kind=RBF, lengthscale=0.2,
                                variance=1.0, noise=1e-2, order=3, rank=128, probes=32,
                                power_iters=2),
    "surrogate_matern_n262144_d3": dict(n=262144, d=3, dist="uniform", kind=MATERN52,
                                        order=3, rank=128, probes=16, power_iters=2),
}

SEED_POINTS = 0
SEED_PROBES = 1
SEED_SKETCH = 2

# hyperparameter box of the gradient / surrogate workloads
THETA_BOX = dict(lengthscale=(0.05, 1.0), variance=(0.5, 2.0), noise=(1e-4, 1e-1))


def points(n, d, dist="uniform", seed=SEED_POINTS):
    """n-by-d float64 point cloud: uniform in [0,1]^d or standard normal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if dist == "uniform":
        return rng.random((n, d))
    if dist == "normal":
        return rng.standard_normal((n, d))
    raise ValueError(dist)


def rademacher(n, s, seed=SEED_PROBES):
    """n-by-s int8 matrix of +-1 (column j is probe j)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (1 - 2 * rng.integers(0, 2, size=(n, s), dtype=np.int8)).astype(np.int8)


def gaussian(n, s, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, s))


def sobol_theta(count, seed=0, box=THETA_BOX):
    """count-by-3 hyperparameters (l, v, nu), scrambled Sobol in log space."""
    import warnings

    from scipy.stats import qmc

    with warnings.catch_warnings():  # counts that are not powers of two are intended here
        warnings.simplefilter("ignore", UserWarning)
        u = qmc.Sobol(d=3, scramble=True, seed=seed).random(count)
    lo = np.log([box["lengthscale"][0], box["variance"][0], box["noise"][0]])
    hi = np.log([box["lengthscale"][1], box["variance"][1], box["noise"][1]])
    return np.exp(lo + u * (hi - lo))
