"""kf_transport_batch (C <- J C J^T for general dense 6x6 J, one thread per
matrix) against the oracle's dense FP64 transport, on the same FP32 inputs.
Bar: the forward error bound of an FP32 matrix product: every entry within
2e-6 (about 16 units of FP32 rounding, for the 12 products summed per entry)
of the same product taken in absolute values, (|J| |C| |J|^T)_ij."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PK = [(i, j) for i in range(6) for j in range(i + 1)]


@pytest.fixture(scope="module")
def kf():
    from paper_1705_02876_gb300 import build, kf as kf_
    build.build()
    return kf_


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    J = (np.eye(6)[None] + 0.5 * rng.normal(size=(n, 6, 6))).astype(np.float32)
    B = rng.normal(size=(n, 6, 6)) * np.logspace(-3, 1, 6)[None, None, :]
    C = np.einsum("nij,nkj->nik", B, B).astype(np.float32)  # SPD, spread scales
    return J, C


@pytest.mark.parametrize("n", [1, 33, 10_007])
def test_transport_batch_matches_oracle(kf, oracle, n):
    J, C = _inputs(n, n)
    Jd = torch.from_numpy(np.ascontiguousarray(J.reshape(n, 36).T)).cuda()
    Cd = torch.from_numpy(np.ascontiguousarray(np.stack([C[:, i, j] for i, j in PK]))).cuda()
    ctx = kf.Context(0)
    kf.transport_batch(ctx, Jd, Cd)
    torch.cuda.synchronize()
    got = Cd.cpu().numpy()
    for t in range(0, n, max(1, n // 200)):
        Jt, Ct = J[t].astype(np.float64), C[t].astype(np.float64)
        ref = oracle.transport(Jt, Ct, np.zeros((6, 6)))
        scale = np.abs(Jt) @ np.abs(Ct) @ np.abs(Jt).T
        for k, (i, j) in enumerate(PK):
            assert abs(got[k, t] - ref[i, j]) <= 2e-6 * scale[i, j], (t, i, j, got[k, t], ref[i, j])
    ctx.close()


def test_transport_batch_empty_and_errors(kf):
    ctx = kf.Context(0)
    kf.transport_batch(ctx, torch.zeros((36, 0), device="cuda"), torch.zeros((21, 0), device="cuda"))
    with pytest.raises(kf.KFError, match="shape"):
        kf.transport_batch(ctx, torch.zeros((36, 5), device="cuda"), torch.zeros((21, 4), device="cuda"))
    ctx.close()


def test_transport_batch_full_size_sampled(kf, oracle):
    """10 million matrices in one launch, as the benchmark times them (inputs
    drawn on the device from a seeded generator, the same recipe as above);
    2,000 sampled matrices against the oracle."""
    n = 10_000_000
    gen = torch.Generator(device="cuda").manual_seed(11)
    J = torch.eye(6, device="cuda")[None] + 0.5 * torch.randn((n, 6, 6), generator=gen, device="cuda")
    scales = torch.logspace(-3, 1, 6, device="cuda")
    B = torch.randn((n, 6, 6), generator=gen, device="cuda") * scales[None, None, :]
    C = torch.bmm(B, B.transpose(1, 2))
    del B
    Jd = J.reshape(n, 36).T.contiguous()
    Cd = torch.stack([C[:, i, j] for i, j in PK]).contiguous()
    del C
    rng = np.random.default_rng(12)
    sel = np.sort(rng.choice(n, 2000, replace=False))
    idx = torch.from_numpy(sel).cuda()
    J_s = Jd[:, idx].cpu().numpy().astype(np.float64)
    C_s = Cd[:, idx].cpu().numpy().astype(np.float64)
    ctx = kf.Context(0)
    kf.transport_batch(ctx, Jd, Cd)
    torch.cuda.synchronize()
    got = Cd[:, idx].cpu().numpy()
    for k in range(len(sel)):
        Jt = J_s[:, k].reshape(6, 6)
        Ct = np.zeros((6, 6))
        for q, (i, j) in enumerate(PK):
            Ct[i, j] = Ct[j, i] = C_s[q, k]
        ref = oracle.transport(Jt, Ct, np.zeros((6, 6)))
        scale = np.abs(Jt) @ np.abs(Ct) @ np.abs(Jt).T
        for q, (i, j) in enumerate(PK):
            assert abs(got[q, k] - ref[i, j]) <= 2e-6 * scale[i, j], (k, i, j)
    ctx.close()
