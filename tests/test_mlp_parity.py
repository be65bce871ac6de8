"""Proposal network on the GPU (training kernels in FP32, inference on the
tensor cores with BF16 weights) against the FP64 numpy oracle, through the C
interface.

Tolerances: FP32 gradient 1e-5 of the gradient's scale per entry; weights
after full-batch Adam steps 1e-5 of the step size.  Logits against the FP64
evaluation of the inference network (W1, W2, W3 in BF16, biases in FP32):
the kernel carries each activation as a BF16 pair hi + lo, exact to 2^-18 of
its value, and accumulates in FP32, so a logit is within a few 2^-18 of the
network's absolute-value magnitude |W3|^T (|W2|^T (|W1|^T |x| + |b1|) +
|b2|) + |b3|; the bar is 2^-14 of it.
"""
import numpy as np
import pytest

from oracle import mlp_oracle as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    from paper_1705_02876_gb300 import build, kf as kf_
    build.build()
    return kf_


@pytest.fixture(scope="module")
def ctx(kf):
    return kf.Context(0)


def data(seed, n):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 12)).astype(np.float32)
    y = ((X[:, 0] + 0.5 * X[:, 1] - X[:, 2] + 0.3 * rng.normal(size=n)) > 0).astype(np.float32)
    w = M.init_params(rng).astype(np.float32)
    return X, y, w


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [1, 63, 64, 1000, 20000])
def test_gradient_matches_oracle(kf, ctx, n):
    X, y, w = data(1, n)
    g, loss = kf.proposal_gradient(ctx, cu(w), cu(X), cu(y))
    torch.cuda.synchronize()
    g_ref = M.backward(w.astype(np.float64), X, y)
    l_ref = M.loss(w.astype(np.float64), X, y)
    scale = np.abs(g_ref).max()
    assert np.abs(g.cpu().numpy() - g_ref).max() <= 1e-5 * scale, np.abs(g.cpu().numpy() - g_ref).max() / scale
    assert abs(loss - l_ref) <= 1e-5 * (1 + l_ref)


def test_full_batch_adam_steps_match_oracle(kf, ctx):
    X, y, w = data(2, 3000)
    wt = cu(w.copy())
    kf.proposal_train(ctx, wt, cu(X), cu(y), epochs=3, batch=3000, lr=1e-3)
    torch.cuda.synchronize()
    p = w.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in range(1, 4):
        p, m, v = M.adam_step(p, M.backward(p, X, y), m, v, t, lr=1e-3)
    # each Adam step moves a weight by about lr; FP32 gradients near zero can
    # flip the sign of an early step, so compare to the step size
    d = np.abs(wt.cpu().numpy() - p)
    assert np.quantile(d, 0.999) <= 1e-5 and d.max() <= 6e-3


def test_training_learns(kf, ctx):
    X, y, w = data(3, 50000)
    wt = cu(w)
    _, l0 = kf.proposal_gradient(ctx, wt, cu(X), cu(y))
    losses = kf.proposal_train(ctx, wt, cu(X), cu(y), epochs=4, batch=1024, lr=3e-3)
    assert losses[-1] < 0.5 * l0 and losses[-1] < 0.25 and losses[-1] <= losses[0], (l0, losses)
    _, l_final = kf.proposal_gradient(ctx, wt, cu(X), cu(y))
    assert abs(l_final - M.loss(wt.cpu().numpy().astype(np.float64), X, y)) < 1e-4


def abs_magnitude(wi, X):
    """|W3|^T (|W2|^T (|W1|^T |x| + |b1|) + |b2|) + |b3| per row: the scale of
    every partial sum the network forms."""
    p = M.unflatten(wi)
    a1 = np.abs(X) @ np.abs(p["W1"]) + np.abs(p["b1"])
    a2 = a1 @ np.abs(p["W2"]) + np.abs(p["b2"])
    return a2 @ np.abs(p["W3"]) + np.abs(p["b3"][0])


@pytest.mark.parametrize("engine", [None, 1, 2])
@pytest.mark.parametrize("n", [1, 31, 32, 33, 127, 129, 4097, 300_000])
def test_tensor_core_scores_match_oracle(kf, ctx, n, engine):
    """Both tensor-core engines (KF_SCORE_MMA_SYNC = 1, KF_SCORE_TCGEN05 = 2)
    and the automatic choice (None; tcgen05 from 262,144 rows), on partial
    warps and partial 128-row tiles."""
    X, y, w = data(4, n)
    kf.proposal_load(ctx, cu(w))
    z = kf.proposal_score(ctx, cu(X), engine=engine).cpu().numpy().astype(np.float64)
    assert not kf.proposal_status(ctx)  # no bounded wait expired
    wi = M.inference_weights(w)
    z_ref, _ = M.forward(wi, X)
    bound = 2.0 ** -14 * abs_magnitude(wi, X.astype(np.float64))
    assert (np.abs(z - z_ref) <= bound).all(), (np.abs(z - z_ref) / bound).max()
    # the weights are BF16: the scores are far closer to the BF16-weight
    # network than to the FP32 master network
    z_master, _ = M.forward(w.astype(np.float64), X)
    assert np.abs(z_master - z).max() > 8 * np.abs(z - z_ref).max()


def test_score_without_weights_fails(kf):
    c = kf.Context(0)
    with pytest.raises(kf.KFError, match="no proposal"):
        kf.proposal_score(c, cu(np.zeros((4, 12), np.float32)))
    c.close()


def test_load_proposal_as_bytes(kf):
    """kf_load_proposal (weights as bytes) loads the same network as
    kf_proposal_load; a buffer of the wrong size is an argument error."""
    X, _, w = data(5, 257)
    c1, c2 = kf.Context(0), kf.Context(0)
    kf.proposal_load(c1, cu(w))
    torch.cuda.synchronize()
    kf.load_proposal(c2, cu(w).view(torch.uint8))
    torch.cuda.synchronize()
    z1 = kf.proposal_score(c1, cu(X)).cpu().numpy()
    z2 = kf.proposal_score(c2, cu(X)).cpu().numpy()
    assert np.array_equal(z1, z2)
    with pytest.raises(kf.KFError, match="bytes"):
        kf.load_proposal(c2, cu(w[:-1]))
    c1.close()
    c2.close()
