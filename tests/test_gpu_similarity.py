"""The device Pearson similarity (tmfg_similarity) against the FP64 oracle.

Every precision must give an exactly symmetric S with a unit diagonal, and
stay within the error its arithmetic allows of the oracle's double-precision
correlations.  The bound used (``tol``) is a worst case with three parts:
  * the float32 rounding of the output: 2^-24;
  * the representation of the unit series y: f32 rounds each entry (2^-24
    relative); the split paths store y = hi + lo + r with |r| <= 2^-18 |y|
    (bf16 halves: 8+8 mantissa bits) or 2^-22 |y| (tf32 halves: 11+11), and
    drop lo.lo' (<= the same bound, Cauchy-Schwarz on unit norms): 3x that;
  * accumulation.  Every partial sum of a dot product of unit vectors is at
    most 1 in size.  The float FMA chain rounds to nearest: <= 2^-24 per
    step, T steps.  The tensor core accumulates in FP32 with truncation, so
    its errors can share a sign: <= 2 ulps (2^-22) per step, where a step is
    one MMA (K = 16 bf16 / 8 tf32 elements, 3 products per K slice) into one
    of the 2 accumulators, whose partial sums add up to at most 1
    (Cauchy-Schwarz over the K slices each one holds): ceil(steps / 2) steps;
    the 2 accumulators are then added in FP32: one more rounding (2^-24).
f64 keeps only the output rounding (1e-7).
"""
import numpy as np
import pytest

import oracle
from paper_2408_09399_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")



def tol(prec, Tlen):
    if prec == "f64":
        return 1e-7
    if prec == "f32":
        return 3 * 2.0 ** -24 + Tlen * 2.0 ** -24
    K, rep = (8, 2.0 ** -22) if prec == "tf32x3" else (16, 2.0 ** -18)
    steps = 3 * -(-Tlen // K)
    return 3 * rep + -(-steps // 2) * 2.0 ** -22 + 2 * 2.0 ** -24


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_09399_gb300 import build
    build.build()
    import paper_2408_09399_gb300 as T
    return T


@pytest.fixture(scope="module")
def ctx(T):
    c = T.tmfg_create(0)
    yield c
    c.close()


def series(n, Tlen, seed=9, walk=True):
    X, _ = W.factor_series(seed, n, Tlen, 7, "equal", (0.3, 0.9), "normal", walk=walk,
                           dtype=np.float32)
    return X


def run(T, ctx, X, prec):
    S = T.tmfg_similarity(ctx, torch.as_tensor(X, device="cuda:0"), prec)
    T.tmfg_sync_status(ctx)
    return S.cpu().numpy()


@pytest.mark.parametrize("prec", ["f64", "f32", "tf32x3", "bf16x3"])
@pytest.mark.parametrize("n,Tlen", [(2, 2), (5, 3), (128, 64), (129, 100), (300, 500),
                                    (383, 1000), (520, 4096)])
def test_similarity_within_tolerance(T, ctx, prec, n, Tlen):
    X = series(n, Tlen, seed=n + Tlen, walk=Tlen > 64)
    S = run(T, ctx, X, prec)
    R = oracle.pearson(X)
    assert np.array_equal(S, S.T)
    assert np.all(np.diag(S) == 1.0)
    off = ~np.eye(n, dtype=bool)
    err = np.abs(S.astype(np.float64) - R)[off].max() if n > 1 else 0.0
    assert err <= tol(prec, Tlen), (prec, n, Tlen, err)


def test_bf16x3_beats_plain_bf16_error_scale(T, ctx):
    """The split keeps ~16 mantissa bits: the error is far below one bf16
    ulp (2^-8 relative) and below the float path's on long random walks."""
    X = series(400, 4096, seed=5)
    R = oracle.pearson(X)
    e3 = np.abs(run(T, ctx, X, "bf16x3") - R).max()
    assert e3 < 2.0 ** -12


def test_strided_tiles_and_many_tiles(T, ctx):
    """n spanning many 128-row tiles with a ragged last tile; every tile pair
    above the diagonal is written once and mirrored."""
    X = series(1100, 300, seed=17)
    R = oracle.pearson(X)
    for prec in ("bf16x3", "tf32x3"):
        S = run(T, ctx, X, prec)
        assert np.array_equal(S, S.T)
        assert np.abs(S - R).max() <= tol(prec, 300)


def test_tiles_per_persistent_cta(T, ctx):
    """More tiles than SMs: each persistent CTA runs several tiles, the
    epilogue of one overlapping the accumulation of the next in the other
    tensor-memory buffer."""
    X = series(2500, 256, seed=29)
    R = oracle.pearson(X)
    for prec in ("bf16x3", "tf32x3"):
        S = run(T, ctx, X, prec)
        assert np.array_equal(S, S.T)
        assert np.all(np.diag(S) == 1.0)
        assert np.abs(S - R).max() <= tol(prec, 256)


def test_constant_or_nonfinite_series_are_errors(T, ctx):
    for bad in ("const", "nan", "inf"):
        X = series(50, 64, seed=3)
        if bad == "const":
            X[7] = 2.5
        elif bad == "nan":
            X[7, 3] = np.nan
        else:
            X[7, 3] = np.inf
        for prec in ("f32", "bf16x3"):
            T.tmfg_similarity(ctx, torch.as_tensor(X, device="cuda:0"), prec)
            with pytest.raises(T.TmfgError) as e:
                T.tmfg_sync_status(ctx)
            assert e.value.code == 3


def test_similarity_feeds_tmfg(T, ctx):
    """S from the device goes straight into tmfg_build; the TMFG equals the
    oracle's on the same float32 S."""
    X = series(300, 1000, seed=23)
    S = T.tmfg_similarity(ctx, torch.as_tensor(X, device="cuda:0"), "bf16x3")
    t = T.tmfg_build(ctx, S, "corr", 1)
    T.tmfg_sync_status(ctx)
    ref = oracle.tmfg(S.cpu().numpy(), "corr", 1)
    assert np.array_equal(t["edges"].cpu().numpy(), ref["edges"])


@pytest.mark.slow
def test_config4_full_size_sampled(T, ctx):
    """n = 30000, T = 4096 random walks (the full workload): bf16x3 and tf32x3
    against the device f64 path (pinned above) on every entry, and the f64
    path against the oracle on sampled rows."""
    X, _ = W.config_series(4)
    Xd = torch.as_tensor(X, device="cuda:0")
    S64 = T.tmfg_similarity(ctx, Xd, "f64")
    T.tmfg_sync_status(ctx)
    rows = np.random.default_rng(1).choice(X.shape[0], 8, replace=False)
    Xs = np.concatenate([X[rows], X[:256]])
    R = oracle.pearson(Xs)
    got = S64[torch.as_tensor(rows, device="cuda:0")][:, :256].cpu().numpy().astype(np.float64)
    assert np.abs(got - R[:8, 8:]).max() <= tol("f64", 4096)
    for prec in ("bf16x3", "tf32x3"):
        S = T.tmfg_similarity(ctx, Xd, prec)
        T.tmfg_sync_status(ctx)
        d = (S - S64).abs().max().item()
        assert d <= tol(prec, 4096) + tol("f64", 4096), (prec, d)
        del S
