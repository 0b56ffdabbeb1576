"""Surrogate kernels (include/egn_mlp.h) against plain FP64 references on the same
BF16 values, and the surrogate's gradients against a CPU FP64 MLP.

Tolerances: FP32-epilogue GEMM within 1e-5 of the FP64 product relative to
sum |a||b| (FP32 accumulation over k <= 1024); BF16 epilogues within one BF16
rounding (2^-8 relative) of the rounded FP64 result; whole-network gradients
within 1e-2 relative (Frobenius) of an FP64 reference that rounds to BF16 where
the kernels store activations and their gradients (what remains: FP32 against
FP64 accumulation and the odd BF16 tie), and within 1e-1 of the unrounded FP64
reference (the size of the BF16 storage effect on a random-target problem,
where the gradients are small residuals).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_2412_11614_gb300 import _build
    _build.build()
    from paper_2412_11614_gb300 import mlp
    return mlp


def _bf16(rng, shape, scale=1.0):
    import torch
    return torch.tensor(rng.normal(0.0, scale, size=shape), dtype=torch.float32).to(torch.bfloat16)


SHAPES = [(128, 256, 64, 1), (300, 256, 192, 1), (1000, 64, 256, 1), (77, 512, 128, 1), (256, 256, 1024, 4),
          (256, 64, 640, 10), (5, 32, 64, 1)]


@pytest.mark.parametrize("m,n,k,splits", SHAPES)
def test_gemm_f32_matches_fp64(K, m, n, k, splits):
    import torch
    rng = np.random.default_rng(m * 7 + n + k)
    a, b = _bf16(rng, (m, k)), _bf16(rng, (n, k))
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    part = torch.full((splits, m, n), float("nan"), dtype=torch.float32, device="cuda")
    K.gemm(a.cuda(), b.cuda(), part, K.EPI_F32, splits=splits, err=err)
    out = torch.empty((m, n), dtype=torch.float32, device="cuda")
    K.reduce_splits(part, splits, out)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    want = a.double().numpy() @ b.double().numpy().T
    bound = np.abs(a.double().numpy()) @ np.abs(b.double().numpy()).T
    got = out.cpu().double().numpy()
    assert np.all(np.abs(got - want) <= 1e-5 * bound + 1e-30)


@pytest.mark.parametrize("epi", ["bias_relu", "bias", "relu_grad"])
def test_gemm_bf16_epilogues(K, epi):
    import torch
    rng = np.random.default_rng(3)
    m, n, k = 333, 256, 256
    a, b = _bf16(rng, (m, k)), _bf16(rng, (n, k))
    bias = torch.tensor(rng.normal(0, 1, n), dtype=torch.float32)
    aux = _bf16(rng, (m, n))
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty((m, n), dtype=torch.bfloat16, device="cuda")
    code = {"bias_relu": K.EPI_BIAS_RELU, "bias": K.EPI_BIAS, "relu_grad": K.EPI_RELU_GRAD}[epi]
    K.gemm(a.cuda(), b.cuda(), out, code, bias=bias.cuda(), aux=aux.cuda(), err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    acc = a.double().numpy() @ b.double().numpy().T
    if epi == "bias_relu":
        want = np.maximum(acc + bias.double().numpy(), 0.0)
    elif epi == "bias":
        want = acc + bias.double().numpy()
    else:
        want = np.where(aux.double().numpy() > 0, acc, 0.0)
    got = out.cpu().double().numpy()
    scale = np.abs(a.double().numpy()) @ np.abs(b.double().numpy()).T + np.abs(bias.double().numpy())
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-5 * scale)


def test_gemm_rejects_bad_shapes(K):
    import torch
    from paper_2412_11614_gb300 import egn
    a = torch.zeros((64, 96), dtype=torch.bfloat16, device="cuda")  # k not a multiple of 64
    b = torch.zeros((32, 96), dtype=torch.bfloat16, device="cuda")
    out = torch.zeros((64, 32), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(egn.EgnError):
        K.gemm(a, b, out, K.EPI_F32, err=err)
    a = torch.zeros((64, 64), dtype=torch.bfloat16, device="cuda")
    b = torch.zeros((40, 64), dtype=torch.bfloat16, device="cuda")  # n not a multiple of 32
    with pytest.raises(egn.EgnError):
        K.gemm(a, b, out, K.EPI_F32, err=err)
    b = torch.zeros((32, 64), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(egn.EgnError):  # split k needs the FP32 epilogue
        K.gemm(a, b, out, K.EPI_BIAS, bias=torch.zeros(32, device="cuda"), splits=2, err=err)


def test_small_kernels(K):
    import torch
    rng = np.random.default_rng(5)
    x = _bf16(rng, (70, 96))
    xt = torch.empty((96, 128), dtype=torch.bfloat16, device="cuda")
    K.transpose(x.cuda(), 128, xt)
    cs = torch.empty(96, dtype=torch.float32, device="cuda")
    K.colsum(x.cuda(), cs)
    torch.cuda.synchronize()
    t = xt.cpu().double().numpy()
    assert np.array_equal(t[:, :70], x.double().numpy().T) and np.all(t[:, 70:] == 0)
    assert np.allclose(cs.cpu().double().numpy(), x.double().numpy().sum(0), rtol=1e-5, atol=1e-5)
    # head: forward, loss and gradients
    h = torch.relu(_bf16(rng, (50, 64)).float()).to(torch.bfloat16)
    w = torch.tensor(rng.normal(0, 1, 64), dtype=torch.float32)
    b = torch.tensor([0.3], dtype=torch.float32)
    tgt = torch.tensor(rng.normal(0, 1, 50), dtype=torch.float32)
    mask = torch.tensor((rng.uniform(size=50) > 0.2).astype(np.float32))
    y, g, loss = (torch.empty(50, device="cuda"), torch.empty(50, device="cuda"), torch.empty(1, device="cuda"))
    dh = torch.empty((50, 64), dtype=torch.bfloat16, device="cuda")
    dw, db = torch.empty(64, device="cuda"), torch.empty(1, device="cuda")
    K.head(h.cuda(), w.cuda(), b.cuda(), y, target=tgt.cuda(), mask=mask.cuda(), loss=loss, g=g, dh=dh, dw=dw, db=db)
    torch.cuda.synchronize()
    H, W, T, M = h.double().numpy(), w.double().numpy(), tgt.double().numpy(), mask.double().numpy()
    yv = H @ W + 0.3
    gv = 2 * M * (yv - T) / M.sum()
    assert np.allclose(y.cpu().numpy(), yv, rtol=1e-5, atol=1e-5)
    assert abs(loss.item() - np.sum(M * (yv - T) ** 2) / M.sum()) < 1e-5
    assert np.allclose(g.cpu().numpy(), gv, rtol=1e-5, atol=1e-7)
    assert np.allclose(dw.cpu().numpy(), gv @ H, rtol=1e-4, atol=1e-6)
    assert abs(db.item() - gv.sum()) < 1e-6
    dhv = np.where(H > 0, np.outer(gv, W), 0.0)
    assert np.all(np.abs(dh.cpu().double().numpy() - dhv) <= 2.0 ** -8 * np.abs(dhv) + 1e-9)
    # Adam, one step from zero moments
    wm = torch.tensor(rng.normal(0, 1, (32, 64)), dtype=torch.float32, device="cuda")
    w0 = wm.cpu().double().numpy()
    gr = torch.tensor(rng.normal(0, 1, (32, 64)), dtype=torch.float32, device="cuda")
    mo, ve = torch.zeros_like(wm), torch.zeros_like(wm)
    wb = torch.empty((32, 64), dtype=torch.bfloat16, device="cuda")
    wt = torch.empty((64, 32), dtype=torch.bfloat16, device="cuda")
    K.adam(wm, gr, mo, ve, 1e-2, 1, w_bf16=wb, wt_bf16=wt)
    torch.cuda.synchronize()
    G = gr.cpu().double().numpy()
    want = w0 - 1e-2 * G / (np.abs(G) + 1e-8)  # bias-corrected first step: m/c1 = g, sqrt(v/c2) = |g|
    assert np.allclose(wm.cpu().double().numpy(), want, rtol=1e-5, atol=1e-6)
    assert torch.equal(wt.cpu(), wb.cpu().T.contiguous())


def _round_bf16(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float64)).to(torch.bfloat16).double().numpy()


def _fp64_mlp_grads(x, Ws, bs, w_out, b_out, t, mask, bf16_storage=False):
    """Plain FP64 forward/backward of the surrogate's network (ReLU MLP + linear
    output, masked mean-squared loss).  With bf16_storage the activations and
    their gradients are rounded to BF16 where the device kernels store them."""
    q = _round_bf16 if bf16_storage else (lambda a: a)
    hs = [x]
    for W, b in zip(Ws, bs):
        hs.append(q(np.maximum(hs[-1] @ W.T + b, 0.0)))
    y = hs[-1] @ w_out + b_out
    msum = mask.sum()
    loss = np.sum(mask * (y - t) ** 2) / msum
    g = 2 * mask * (y - t) / msum
    dW, db = [None] * len(Ws), [None] * len(Ws)
    dw_out, db_out = g @ hs[-1], g.sum()
    d = q(np.outer(g, w_out) * (hs[-1] > 0))
    for i in reversed(range(len(Ws))):
        dW[i] = d.T @ hs[i]
        db[i] = d.sum(0)
        if i > 0:
            d = q((d @ Ws[i]) * (hs[i] > 0))
    return loss, dW, db, dw_out, db_out


def test_surrogate_gradients_match_fp64_mlp(K):
    import torch
    from paper_2412_11614_gb300 import surrogate as S
    rng = np.random.default_rng(11)
    model = S.Surrogate(seed=4)
    rows = 700
    x = rng.normal(0, 1, (rows, S.N_FEAT))
    t = rng.normal(0, 1, rows)
    model.fit_normalisation(x, t)
    Ws = [w.cpu().to(torch.bfloat16).double().numpy() for w in model.W]
    bs = [b.cpu().double().numpy() for b in model.b]
    w_out, b_out = model.w_out.cpu().double().numpy(), float(model.b_out.item())
    loss = model.train_step(x, t, lr=0.0)  # lr 0: gradients only
    xn = np.zeros((rows, S.F_PAD))
    xn[:, :S.N_FEAT] = (x - model.x_mean) / model.x_std
    xn = torch.tensor(xn, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    tn = (t - model.y_mean) / model.y_std

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    g = [p.cpu().double().numpy() for p in model.grads]
    # (1) the same arithmetic with BF16 storage where the kernels store: tight
    lw, dW, db, dwo, dbo = _fp64_mlp_grads(xn, Ws, bs, w_out, b_out, tn, np.ones(rows), bf16_storage=True)
    assert abs(loss - lw) <= 1e-3 * lw
    for i in range(S.LAYERS):
        assert rel(g[2 * i], dW[i]) < 1e-2, (i, rel(g[2 * i], dW[i]))
        assert rel(g[2 * i + 1], db[i]) < 1e-2, (i, rel(g[2 * i + 1], db[i]))
    assert rel(g[-2], dwo) < 1e-3 and abs(g[-1][0] - dbo) <= 1e-3 * abs(dbo) + 1e-6
    # (2) full FP64: the size of the BF16 storage effect on the gradients
    lw, dW, db, dwo, dbo = _fp64_mlp_grads(xn, Ws, bs, w_out, b_out, tn, np.ones(rows))
    assert abs(loss - lw) <= 1e-2 * lw
    for i in range(S.LAYERS):
        assert rel(g[2 * i], dW[i]) < 1e-1, (i, rel(g[2 * i], dW[i]))
        assert rel(g[2 * i + 1], db[i]) < 1e-1
    assert rel(g[-2], dwo) < 3e-2


def test_surrogate_learns_a_smooth_map(K):
    from paper_2412_11614_gb300 import surrogate as S
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, (4096, S.N_FEAT))
    t = np.sin(2 * x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] + 0.2 * x[:, 3]
    model = S.Surrogate(seed=1)
    model.fit_normalisation(x, t)
    first = model.train_step(x[:1024], t[:1024], lr=1e-3)
    for step in range(300):
        i = (step * 1024) % 4096
        last = model.train_step(x[i:i + 1024], t[i:i + 1024], lr=1e-3)
    assert last < 0.1 * first
    pred = model.predict_rows(x[:512])
    assert np.sqrt(np.mean((pred - t[:512]) ** 2)) < 0.3 * np.std(t)


class _Crash(Exception):
    pass


def test_training_checkpoint_resume_is_bit_identical(K, tmp_path):
    """A training run that dies after step 4 (checkpoints every 3 steps) and is
    resumed from its checkpoint by a fresh model ends with exactly the weights,
    Adam moments and predictions of an uninterrupted run (all kernels are
    deterministic, the sampler state is in the checkpoint)."""
    from paper_2412_11614_gb300 import surrogate as S
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, (3000, S.N_FEAT))
    t = np.cos(3 * x[:, 0]) + x[:, 4] * x[:, 5]
    ref = S.Surrogate(seed=3)
    ref.fit_normalisation(x, t)
    ref_losses = S.train(ref, x, t, steps=8, batch_rows=1024, seed=9)   # 2 batches per epoch, 4 epochs

    ck = str(tmp_path / "ck.npz")

    def die(step, loss):
        if step == 4:
            raise _Crash()

    a = S.Surrogate(seed=3)
    a.fit_normalisation(x, t)
    with pytest.raises(_Crash):
        S.train(a, x, t, steps=8, batch_rows=1024, seed=9, checkpoint=ck, every=3, on_step=die)
    b = S.Surrogate(seed=11)  # other initial weights: everything must come from the checkpoint
    losses = S.train(b, x, t, steps=8, batch_rows=1024, seed=9, checkpoint=ck, every=3)
    assert losses == ref_losses[3:]
    sa, sb = ref.state(), b.state()
    assert sa.keys() == sb.keys()
    for key in sa:
        assert np.array_equal(sa[key], sb[key]), key
    assert np.array_equal(ref.predict_rows(x[:500]), b.predict_rows(x[:500]))
    # the finished checkpoint holds the final step: a rerun trains nothing
    c = S.Surrogate(seed=12)
    assert S.train(c, x, t, steps=8, batch_rows=1024, seed=9, checkpoint=ck, every=3) == []
    assert np.array_equal(c.predict_rows(x[:500]), b.predict_rows(x[:500]))
