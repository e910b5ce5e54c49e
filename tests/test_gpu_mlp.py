"""GPU parity of the tcgen05 surrogate MLP against the FP64 oracle MLP.

The GPU keeps weights and activations in bf16 (8-bit mantissa) with fp32
accumulation; the oracle runs in FP64 on the same bf16-rounded weights and
inputs.  Bound: each of the 5 layers adds a relative rounding of ~2^-8
(activations rounded to bf16) on top of fp32 accumulation, so outputs agree
to ~1e-2 relative and gradients (a second chain of 5 bf16 roundings) to
~3e-2."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def bf16_round(a):
    t = torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32)
    return t.numpy().astype(np.float64)


@pytest.fixture(scope="module")
def ect():
    assert torch.cuda.is_available()
    from paper_1602_03207_gb300 import build, ect as ect_mod
    build.build()
    ect_mod.load_library()
    return ect_mod


def setup_case(ect, B=256, seed=0):
    p = mlp.init(seed)
    rng = np.random.default_rng(seed + 1)
    for l in range(len(p)):
        p[l][1] = rng.normal(scale=0.1, size=p[l][1].shape)
    X = rng.uniform(-1, 1, size=(B, 6))
    T = rng.normal(size=(B, 256))
    pr = [[bf16_round(W), np.asarray(b, np.float32).astype(np.float64)] for W, b in p]
    Xr = bf16_round(X)
    return p, pr, X, Xr, T


def test_num_params(ect):
    assert ect.load_library().ect_mlp_num_params() == sum(W.size + b.size for W, b in mlp.init(0))


# 65536 rows are 512 tiles of 128: each persistent CTA takes several tiles, so the shared-memory
# ring wraps and both TMEM accumulators are reused
@pytest.mark.parametrize("B", [128, 256, 4096, 65536])
def test_forward_matches_oracle(ect, B):
    p, pr, X, Xr, T = setup_case(ect, B)
    s = ect.Surrogate(batch=B)
    s.set_params(ect.mlp_flatten(p))
    x = torch.from_numpy(X.astype(np.float32)).cuda()
    y = torch.empty(B, 256, dtype=torch.float32, device="cuda")
    s.forward(x, y)
    ref, _ = mlp.forward(pr, Xr)
    Y = y.cpu().numpy()
    err = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    assert err <= 1e-2, err
    s.close()


# the weight gradients contract over the batch: 256 rows is one K range per CTA, 16384 and 65536
# split K over the CTAs (64 and 74 ranges of 4 and 14 chunks) and sum the partial products
@pytest.mark.parametrize("B", [256, 16384, 65536])
def test_gradients_match_oracle(ect, B):
    p, pr, X, Xr, T = setup_case(ect, B, seed=3)
    s = ect.Surrogate(batch=B)
    s.set_params(ect.mlp_flatten(p))
    x = torch.from_numpy(X.astype(np.float32)).cuda()
    t = torch.from_numpy(T.astype(np.float32)).cuda()
    g, loss = s.gradients(x, t)
    y, cache = mlp.forward(pr, Xr)
    ref = mlp.backward(pr, cache, y, T)
    assert abs(loss - mlp.loss(y, T)) <= 1e-2 * mlp.loss(y, T)
    G = ect.mlp_unflatten(g)
    for l in range(len(ref)):
        for i in range(2):
            a, r = np.asarray(G[l][i], np.float64), ref[l][i]
            err = np.linalg.norm(a - r) / np.linalg.norm(r)
            assert err <= 3e-2, (l, i, err)
    s.close()


def test_adam_step_matches_oracle_and_training_reduces_loss(ect):
    p, pr, X, Xr, T = setup_case(ect, 256, seed=5)
    T = np.tanh(X @ np.random.default_rng(9).normal(size=(6, 256)))
    s = ect.Surrogate(batch=256)
    s.set_params(ect.mlp_flatten(p))
    x = torch.from_numpy(X.astype(np.float32)).cuda()
    t = torch.from_numpy(T.astype(np.float32)).cuda()
    l0 = s.train_step(x, t, 1e-3, want_loss=True)
    # one Adam step moves every parameter with a non-negligible gradient by ~lr
    q = s.get_params()
    d = np.abs(q - ect.mlp_flatten(p))
    assert np.median(d[d > 0]) == pytest.approx(1e-3, rel=0.05)
    for _ in range(300):
        s.train_step(x, t, 1e-3)
    l1 = s.train_step(x, t, 1e-3, want_loss=True)
    assert l1 < 0.2 * l0, (l0, l1)
    s.close()
