"""GPU kernels of the learned row-size predictor (BF16 inputs and weights,
FP32 accumulation) against the FP64 reference in oracle/mlp.py, evaluated on
the same bf16-rounded weights and inputs.

The forward check allows for the kernels rounding the two hidden activations
to bf16 (relative 2^-9 per value): a few 1e-2 of the logit's scale.

The gradient check is element by element.  The reference then takes the
kernel's rounding points too: it rounds h1 and h2 to bf16 in FP64 (so both
sides take the same ReLU and rounding decisions up to FP32-vs-FP64 ties), and
runs oracle/mlp.py's FP64 backward on them.  What remains per entry is FP32
accumulation (at most ~(64 + 160) 2^-24 of the entry's sum of absolute
terms) and, rarely, one bf16 ulp (2^-8) of a single row's activation where
the FP32 and FP64 values straddle a bf16 rounding point.  So every entry must
satisfy |g - g_ref| <= 2^-8 * G_abs + 1e-7, where G_abs is the same backward
run on absolute values (the entry's sum of |terms| over rows)."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2106_14402_gb300 import gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_14402_gb300 import cb as _cb
    _cb.load()
    return _cb


def bf16(a):
    """Round float64/float32 values to bfloat16 (nearest even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["w3"], p["b3"]])


def unflat(v):
    v = np.asarray(v, dtype=np.float64)
    o = 0
    out = {}
    for k, shape in (("W1", (64, 3)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)),
                     ("w3", (64,)), ("b3", (1,))):
        n = int(np.prod(shape))
        out[k] = v[o:o + n].reshape(shape)
        o += n
    return out


def setup_problem(seed=0):
    P = gen.rmat(12, 16, *gen.RMAT_ABCD, seed=400 + seed)
    A = P.with_values(np.ones(P.nnz, np.uint8))
    flops, maxb = oracle.row_stats(A, A)
    nnz = np.diff(oracle.spgemm("or_and_bool", A, A)[0])
    nnza = np.diff(A.row_ptr)
    width = np.full(A.nrows, A.ncols)
    F = np.stack([nnza, flops, maxb, width], 1).astype(np.float64)
    L = mlp.raw_features(nnza, flops, maxb, width)
    norm = np.concatenate([L.mean(0), L.std(0) + 1e-3]).astype(np.float32)
    p = mlp.init_params(seed)
    return A, F, nnz, norm, p


def reference_inputs(F, norm, p):
    """bf16-rounded weights and standardized inputs, as the kernels see them."""
    q = {k: (bf16(v) if k in ("W1", "W2", "w3") else np.asarray(v, np.float32).astype(np.float64))
         for k, v in p.items()}
    mu, sg = norm[:3].astype(np.float64), norm[3:].astype(np.float64)
    X = bf16((mlp.raw_features(F[:, 0], F[:, 1], F[:, 2], F[:, 3]) - mu) / sg)
    return q, X


def test_row_features_match_row_stats(cb):
    A, F, nnz, norm, p = setup_problem()
    dA = cb.DeviceCSR.from_host(A, "or_and_bool")
    feat = cb.row_features(dA, dA).cpu().numpy()
    assert np.array_equal(feat.astype(np.int64), F.astype(np.int64))


def test_forward_and_sizes(cb):
    A, F, nnz, norm, p = setup_problem(1)
    model = cb.MLP(flat(p).astype(np.float32), norm)
    feat = torch.tensor(F, dtype=torch.float32, device="cuda")
    z, pred = model.predict(feat, ncols=A.ncols)
    z = z.cpu().numpy().astype(np.float64)
    q, X = reference_inputs(F, norm, p)
    zr, cache = mlp.forward(q, X)
    scale = np.abs(cache[4]) @ np.abs(q["w3"]) + 1.0
    assert np.all(np.abs(z - zr) <= 3e-2 * scale), np.max(np.abs(z - zr) / scale)
    # the integer size rule applied to the kernel's own logits
    want = mlp.predict_sizes(z, F[:, 1].astype(np.int64), F[:, 2].astype(np.int64), A.ncols)
    assert np.array_equal(pred.cpu().numpy(), want)


def forward_at_kernel_rounding(q, X):
    """oracle/mlp.py's forward with the hidden activations rounded to bf16 where
    the kernels round them; the cache makes backward's ReLU masks h > 0, the
    kernels' masks."""
    a1 = X @ q["W1"].T + q["b1"]
    h1 = bf16(np.maximum(a1, 0.0))
    a2 = h1 @ q["W2"].T + q["b2"]
    h2 = bf16(np.maximum(a2, 0.0))
    z = h2 @ q["w3"] + q["b3"][0]
    return z, (X, h1, h1, h2, h2)


GRAD_RTOL = 2.0 ** -8
GRAD_ATOL = 1e-7


@pytest.mark.parametrize("seed", [2, 5])
def test_gradients_match_fp64_reference(cb, seed):
    A, F, nnz, norm, p = setup_problem(seed)
    model = cb.MLP(flat(p).astype(np.float32), norm)
    feat = torch.tensor(F, dtype=torch.float32, device="cuda")
    g, loss = model.grad(feat, torch.tensor(nnz, dtype=torch.int64, device="cuda"), tau=0.9)
    g = unflat(g.cpu().numpy().astype(np.float64))
    q, X = reference_inputs(F, norm, p)
    z, cache = forward_at_kernel_rounding(q, X)
    L, dz = mlp.loss_and_dz(z, F[:, 1], nnz, 0.9)
    want = mlp.backward(q, cache, dz)
    # the same backward on absolute values: each entry's sum of |terms|
    qa = {k: np.abs(v) for k, v in q.items()}
    Xa, h1, _, h2, _ = cache
    gabs = mlp.backward(qa, (np.abs(Xa), h1, h1, h2, h2), np.abs(dz))
    live = F[:, 1] > 0
    e = np.log2(nnz[live] / F[live, 1]) - mlp.log2_sigmoid(z[live])
    assert np.min(np.abs(e)) > 1e-4, "a row sits on the pinball kink: pick another seed"
    loss_scale = np.mean(np.abs(e))
    assert abs(float(loss.item()) - L) <= 1e-4 * loss_scale + 1e-6
    checked = sharp = 0
    for k in want:
        bound = GRAD_RTOL * gabs[k] + GRAD_ATOL
        bad = np.abs(g[k] - want[k]) > bound
        assert not bad.any(), (k, np.nonzero(bad.ravel())[0][:5], g[k].ravel()[bad.ravel()][:5],
                               want[k].ravel()[bad.ravel()][:5])
        checked += want[k].size
        sharp += int((np.abs(want[k]) > 10 * bound).sum())
    assert checked == cb.MLP_NPARAM
    # the bound discriminates: most entries are over ten times larger than it
    assert sharp > 0.5 * checked


def test_training_lowers_the_loss(cb):
    A, F, nnz, norm, p = setup_problem(3)
    model = cb.MLP(flat(p).astype(np.float32), norm)
    feat = torch.tensor(F, dtype=torch.float32, device="cuda")
    lab = torch.tensor(nnz, dtype=torch.int64, device="cuda")
    _, l0 = model.grad(feat, lab)
    losses = model.train(feat, lab, epochs=30, batch=1024, lr=3e-3)
    _, l1 = model.grad(feat, lab)
    assert losses[-1] < losses[0]
    assert float(l1.item()) < 0.5 * float(l0.item())
    params, nrm, step = model.get()
    assert step > 0 and np.all(np.isfinite(params)) and np.array_equal(nrm, norm)
