"""Seeded synthetic workloads shaped like the paper's time-series inputs.

The paper clusters UCR time-series sets (Table 1: n from 930 to 19412
series, lengths 46 to 2709, 2 to 60 classes) through the Pearson correlation
matrix of the series (Section 5, Datasets).  Those sets are not shipped
here; these generators make planted-cluster stand-ins with the same shapes.

Every random number comes from one counter-based generator, splitmix64
(Steele, Lea & Flood 2014), evaluated at (seed, stream, counter) with numpy
uint64 arithmetic, so a workload is the same on every machine up to the
last-bit behaviour of ``log``/``cos``/``sqrt`` in the normal transform.  This
module holds no TMFG, APSP or DBHT arithmetic; the oracle and the CUDA path
both consume what it produces.

Factor model: series i of cluster k(i) is x_i(t) = lam_i * f_k(t) + e_i(t)
with f_k(t) ~ N(0,1), lam_i ~ U[lo, hi] and e_i(t) ~ N(0,1) or a unit-variance
Student-t(4); ``walk=True`` integrates each series over t (random walks).
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * _M1
    z = z ^ (z >> np.uint64(27))
    z = z * _M2
    return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: str) -> np.uint64:
    h = hashlib.sha256(f"{int(seed)}:{stream}".encode()).digest()
    return np.uint64(int.from_bytes(h[:8], "little"))


def u64(seed: int, stream: str, count: int, offset: int = 0) -> np.ndarray:
    """``count`` splitmix64 outputs of (seed, stream) starting at ``offset``."""
    key = _stream_key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        return _mix(key + ctr * _GOLDEN)


def uniform(seed: int, stream: str, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (u64(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: str, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller (one normal per pair of uniforms)."""
    u = uniform(seed, stream, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def student_t4_unit(seed: int, stream: str, count: int, offset: int = 0) -> np.ndarray:
    """Student-t with 4 degrees of freedom scaled to unit variance:
    Z / sqrt(V/4) with V = -2 ln(U1 U2) ~ chi^2(4); Var(t_4) = 2."""
    z = normal(seed, stream + "/z", count, offset)
    u = uniform(seed, stream + "/v", 2 * count, 2 * offset)
    v = -2.0 * np.log((1.0 - u[0::2]) * (1.0 - u[1::2]))
    return z / np.sqrt(v / 4.0) / math.sqrt(2.0)


def cluster_sizes(seed: int, n: int, k: int, kind: str = "equal", min_size: int = 2) -> np.ndarray:
    """Planted cluster sizes summing to n: equal, or Dirichlet(1) proportions
    (normalised exponentials) rounded by largest remainder, each >= min_size."""
    if kind == "equal":
        base = np.full(k, n // k, np.int64)
        base[: n - base.sum()] += 1
        return base
    if k * min_size > n:
        raise ValueError("too many clusters for n")
    e = -np.log(1.0 - uniform(seed, "dirichlet", k))
    p = e / e.sum()
    raw = p * n
    sizes = np.floor(raw).astype(np.int64)
    rem = n - sizes.sum()
    order = np.argsort(-(raw - sizes), kind="stable")
    sizes[order[:rem]] += 1
    while sizes.min() < min_size:
        i, j = int(np.argmin(sizes)), int(np.argmax(sizes))
        sizes[i] += 1
        sizes[j] -= 1
    return sizes


def labels_for(seed: int, sizes: np.ndarray) -> np.ndarray:
    """Cluster label of each series, spread over the ids by a seeded shuffle."""
    n = int(sizes.sum())
    block = np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)
    perm = np.argsort(uniform(seed, "perm", n), kind="stable")
    lab = np.empty(n, np.int32)
    lab[perm] = block
    return lab


def factor_series(seed: int, n: int, T: int, k: int, sizes: str = "equal",
                  loading=(0.3, 0.9), noise: str = "normal", walk: bool = False,
                  dtype=np.float64, chunk: int = 2048):
    """Planted-factor series X (n x T) and their labels (see module doc)."""
    sz = cluster_sizes(seed, n, k, sizes)
    lab = labels_for(seed, sz)
    lam = loading[0] + (loading[1] - loading[0]) * uniform(seed, "loading", n)
    F = normal(seed, "factors", k * T).reshape(k, T)
    X = np.empty((n, T), dtype)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        cnt = (r1 - r0) * T
        if noise == "normal":
            e = normal(seed, "noise", cnt, r0 * T)
        elif noise == "t4":
            e = student_t4_unit(seed, "noise", cnt, r0 * T)
        else:
            raise ValueError(noise)
        blk = lam[r0:r1, None] * F[lab[r0:r1]] + e.reshape(r1 - r0, T)
        if walk:
            blk = np.cumsum(blk, axis=1)
        X[r0:r1] = blk
    return X, lab


def pearson_similarity(X: np.ndarray, dtype=np.float32, device: str = "cpu"):
    """The paper's input matrix: Pearson correlation of every pair of series
    (Section 5, Datasets), computed in double (numpy, or torch on ``device``)
    and stored as ``dtype``.  The diagonal is set to 1."""
    if device == "cpu":
        Xc = X - X.mean(axis=1, keepdims=True)
        Xc = Xc / np.sqrt((Xc * Xc).sum(axis=1, keepdims=True))
        S = (Xc @ Xc.T).astype(dtype)
    else:
        import torch
        Xt = torch.as_tensor(X, dtype=torch.float64, device=device)
        Xt = Xt - Xt.mean(dim=1, keepdim=True)
        Xt = Xt / torch.sqrt((Xt * Xt).sum(dim=1, keepdim=True))
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        S = (Xt @ Xt.T).to(tdt)
        S.fill_diagonal_(1.0)
        return S
    np.fill_diagonal(S, 1.0)
    return S


# The five workload shapes (sizes from the paper's range of n and lengths).
CONFIGS = {
    1: dict(n=200, T=256, k=5, sizes="equal", loading=(0.3, 0.9), noise="normal",
            dtype=np.float64, seed=1001),
    2: dict(n=5000, T=1000, k=20, sizes="dirichlet", loading=(0.3, 0.9), noise="normal",
            dtype=np.float32, seed=1002),
    3: dict(n=20000, T=2000, k=50, sizes="dirichlet", loading=(0.3, 0.9), noise="t4",
            dtype=np.float32, seed=1003),
    # raw series for the similarity product: random walks of 40 factors
    4: dict(n=30000, T=4096, k=40, sizes="equal", loading=(0.3, 0.9), noise="normal",
            dtype=np.float32, seed=1004, walk=True),
}


def config_series(cfg: int, n: int | None = None, T: int | None = None):
    """(X float32 n x T, labels) of workload ``cfg`` (raw series; ``n`` and
    ``T`` optionally shrink it)."""
    c = dict(CONFIGS[cfg])
    if n is not None:
        c["n"] = n
    if T is not None:
        c["T"] = T
    X, lab = factor_series(c["seed"], c["n"], c["T"], c["k"], c["sizes"], c["loading"],
                           c["noise"], walk=c.get("walk", False), dtype=np.float32)
    return X, lab


def config_similarity(cfg: int, device: str = "cpu", n: int | None = None):
    """(S, labels) for workload ``cfg``; ``n`` optionally shrinks it while
    keeping every other parameter (used for quick cases)."""
    c = dict(CONFIGS[cfg])
    if n is not None:
        c["n"] = n
    X, lab = factor_series(c["seed"], c["n"], c["T"], c["k"], c["sizes"], c["loading"],
                           c["noise"])
    return pearson_similarity(X, c["dtype"], device), lab


def random_similarity(seed: int, n: int, dtype=np.float32, kind: str = "uniform"):
    """Unstructured symmetric test matrices.  kinds: 'uniform' U(-1,1);
    'quantized' values on a grid of 1/8 (many exact ties, with -0.0 mixed
    in); 'constant' (all off-diagonal entries equal); 'dyadic_additive'
    S[i,j] = a_i + a_j with distinct multiples of 2^-10 (exact in float)."""
    iu = np.triu_indices(n, 1)
    S = np.zeros((n, n), np.float64)
    if kind == "uniform":
        vals = 2.0 * uniform(seed, "sym", len(iu[0])) - 1.0
    elif kind == "quantized":
        vals = np.floor(uniform(seed, "sym", len(iu[0])) * 17.0) / 8.0 - 1.0
    elif kind == "constant":
        vals = np.full(len(iu[0]), 0.25)
    elif kind == "dyadic_additive":
        a = (np.argsort(uniform(seed, "add", n), kind="stable") - n / 2.0) / 1024.0
        vals = a[iu[0]] + a[iu[1]]
    else:
        raise ValueError(kind)
    S[iu] = vals
    S = S + S.T
    np.fill_diagonal(S, 1.0)
    S = S.astype(dtype)
    if kind == "quantized":
        # spread some negative zeros over the zero entries, symmetrically
        z = (S == 0) & (np.arange(n)[:, None] != np.arange(n)[None, :])
        flip = (u64(seed, "negzero", n * n).reshape(n, n) & np.uint64(1)).astype(bool)
        flip = np.triu(flip, 1)
        flip = flip | flip.T
        S[z & flip] = -0.0
    return np.ascontiguousarray(S)


def serving_requests(seed: int, count: int, device: str = "cuda", n_range=(64, 4000),
                     T_range=(128, 2048), k_range=(2, 30), loading=(0.5, 0.9),
                     similarity: bool = True):
    """Clustering requests shaped like the serving workload: n log-uniform in
    n_range, series length T uniform in T_range, planted cluster count k
    uniform in k_range, strong loadings (clean instances).  The sizes come
    from the counter-based generator above; the series themselves are drawn
    with torch's generator seeded from (seed, request), on ``device``, which
    keeps generation of thousands of requests fast (they are reproducible on
    one device type, not across CPU and GPU).  Returns a list of dicts with
    the raw float32 series X (n x T), the float32 Pearson matrix S (unless
    ``similarity`` is False: the pipeline computes it), the labels and the
    shape."""
    import torch
    u = uniform(seed, "req_n", count)
    ns = np.round(np.exp(np.log(n_range[0]) + u * (np.log(n_range[1]) - np.log(n_range[0]))))
    Ts = T_range[0] + (uniform(seed, "req_T", count) * (T_range[1] - T_range[0] + 1)).astype(int)
    ks = k_range[0] + (uniform(seed, "req_k", count) * (k_range[1] - k_range[0] + 1)).astype(int)
    out = []
    for i in range(count):
        n, T, k = int(ns[i]), int(Ts[i]), int(min(ks[i], ns[i] // 2))
        g = torch.Generator(device=device)
        g.manual_seed(int(u64(seed, "req_seed", 1, i)[0] >> np.uint64(1)))
        lab = torch.randint(0, k, (n,), generator=g, device=device)
        lam = loading[0] + (loading[1] - loading[0]) * torch.rand(n, generator=g, device=device)
        F = torch.randn(k, T, generator=g, device=device)
        X = lam[:, None] * F[lab] + torch.randn(n, T, generator=g, device=device)
        rec = {"X": X.contiguous(), "labels": lab, "n": n, "T": T, "k": k}
        if similarity:
            Y = X - X.mean(dim=1, keepdim=True)
            Y = Y / torch.sqrt((Y * Y).sum(dim=1, keepdim=True))
            S = Y @ Y.T
            S.fill_diagonal_(1.0)
            rec["S"] = S.contiguous()
        out.append(rec)
    return out
