"""Seeded synthetic inputs of the benchmark and test workloads.

Only NumPy's default generator is used here: none of the library's own
engines, seeding or samplers.  Both the CUDA path and the oracle-based tests
take their inputs from these functions.
"""
import numpy as np

# Distribution mix of the batched substream workload: uniform 25%, normal 35%,
# exponential 15%, gamma 25% (shape log-uniform in [0.1, 100]).
BATCH_MIX = (("uniform", 0.25), ("normal", 0.35), ("exp", 0.15), ("gamma", 0.25))


def batch_workload(n_req=4096, lo=1e3, hi=1e7, seed=99, mix=BATCH_MIX, alpha_range=(0.1, 100.0)):
    """Request table of the batched substream workload: request i uses
    substream i, size floor(10^U) with U uniform in [log10 lo, log10 hi], a
    distribution drawn from `mix` and, for gamma, a log-uniform shape.
    Returns a list of dicts (stream, dist, n, p0, p1, m, pos)."""
    rng = np.random.default_rng(seed)
    lu = rng.uniform(np.log10(lo), np.log10(hi), n_req)
    sizes = np.floor(10.0 ** lu).astype(np.int64)
    names = [m[0] for m in mix]
    probs = np.array([m[1] for m in mix], dtype=np.float64)
    kinds = rng.choice(len(names), size=n_req, p=probs / probs.sum())
    la, ha = np.log10(alpha_range[0]), np.log10(alpha_range[1])
    alphas = 10.0 ** rng.uniform(la, ha, n_req)
    reqs = []
    for i in range(n_req):
        d = names[kinds[i]]
        reqs.append({"stream": i, "dist": d, "n": int(sizes[i]), "p0": float(alphas[i]) if d == "gamma" else 0.0,
                     "p1": 0.0, "m": 0, "pos": 0})
    return reqs


def mixed_requests(n_req, seed, max_n=20000):
    """Small request tables for parity tests: every distribution, sizes
    log-uniform in [1, max_n], substreams spread over [0, 4096), some
    nonzero start words, shapes for gamma (log-uniform [0.1, 100]) and beta
    (a != b), moduli for the bounded requests."""
    rng = np.random.default_rng(seed)
    dists = ["u64", "uniform", "bounded", "normal", "exp", "gamma", "beta"]
    moduli = [6, 1_000_000_007, 2**63 + 1, 0, 1000]
    streams = rng.permutation(4096)[:n_req]
    streams[0] = 0
    reqs = []
    for i in range(n_req):
        d = dists[i % len(dists)]
        n = int(np.floor(10.0 ** rng.uniform(0.0, np.log10(max_n))))
        pos = int(rng.integers(0, 1000)) if i % 3 == 1 else 0
        p0 = p1 = 0.0
        m = 0
        if d == "gamma":
            p0 = float(10.0 ** rng.uniform(-1.0, 2.0))
        elif d == "beta":
            p0, p1 = [(0.5, 2.0), (2.0, 5.0), (3.0, 0.7)][i % 3]
        elif d == "bounded":
            m = moduli[i % len(moduli)]
        reqs.append({"stream": int(streams[i]), "dist": d, "n": n, "p0": p0, "p1": p1, "m": m, "pos": pos})
    return reqs


def upstream_grads(n, seed=1):
    """Upstream gradients dL/dz ~ N(0, 1)."""
    return np.random.default_rng(seed).standard_normal(n)


def mvn_inputs(d, seed=3):
    """Mean and Cholesky factor of the multivariate-normal workload:
    Sigma = W W^T / d + 0.1 I with W a d x d standard-normal matrix, mu ~
    N(0, 1); L = chol(Sigma) (LAPACK through NumPy)."""
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((d, d))
    mu = rng.standard_normal(d)
    sigma = W @ W.T / d + 0.1 * np.eye(d)
    return mu, np.linalg.cholesky(sigma)
