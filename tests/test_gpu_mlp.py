"""GPU parity of the warm-start network kernels (ieti_mlp_*) against the FP64
oracle network of oracle/mlp.py, which applies the same bfloat16 rounding to
every GEMM operand.

Sizes are chosen to be ragged for the 64 x 64 x 32 GEMM tiles: batch 70
(two row tiles, the second with 6 rows), n_in 80 (K tail of 16), hidden 256
(four column tiles), n_out 333.

Tolerances: the kernels accumulate each product in FP32 (at most 256 terms,
about 1e-5 relative), the oracle in FP64 from identically rounded operands. A
bfloat16 activation, or a ReLU decision, can come out differently where the
FP32 and FP64 pre-activations straddle a rounding boundary or zero; that is
rare and is absorbed by relative Frobenius-norm bounds of 2e-3 on the outputs
and on each gradient tensor.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp as om

B, NI, NH, NO = 70, 80, 256, 333


@pytest.fixture(scope="module")
def ieti():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti as m
    return m


def _data(seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, NI))
    T = rng.standard_normal((B, NO))
    return X, T


def _flat(params):
    return np.concatenate([np.ravel(p) for p in params])


def _split(v):
    shapes = [(NH, NI), (NH,), (NH, NH), (NH,), (NO, NH), (NO,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(v[o:o + n].reshape(s).astype(np.float64))
        o += n
    return out


def _net(ieti, params):
    m = ieti.ieti_mlp_create(NI, NH, NO, B)
    # the oracle's parameters, rounded to FP32 as the library stores them
    ieti.ieti_mlp_set_params(m, _flat(params))
    return m


def _f32(params):
    return [np.asarray(p, np.float32).astype(np.float64) for p in params]


def relf(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_forward_matches_oracle(ieti):
    params = _f32(om.init_params(NI, NH, NO, seed=1))
    X, _ = _data(2)
    m = _net(ieti, params)
    try:
        x = torch.tensor(X, dtype=torch.float32, device="cuda")
        y = torch.empty((B, NO), dtype=torch.float32, device="cuda")
        ieti.ieti_mlp_forward(m, x, y)
        y64 = torch.empty((B, NO), dtype=torch.float64, device="cuda")
        ieti.ieti_mlp_forward_f64(m, x, y64)
        Y, _ = om.forward(params, np.asarray(X, np.float32).astype(np.float64))
        assert relf(y.cpu().numpy().astype(np.float64), Y) <= 2e-3
        assert np.array_equal(y64.cpu().numpy(), y.cpu().numpy().astype(np.float64))
    finally:
        ieti.ieti_mlp_destroy(m)


def test_forward_ragged_batches_agree(ieti):
    """Rows do not interact: a batch of 1 and a batch of 70 give the same row."""
    params = _f32(om.init_params(NI, NH, NO, seed=3))
    X, _ = _data(4)
    m = _net(ieti, params)
    try:
        x = torch.tensor(X, dtype=torch.float32, device="cuda")
        y = torch.empty((B, NO), dtype=torch.float32, device="cuda")
        ieti.ieti_mlp_forward(m, x, y)
        y1 = torch.empty((1, NO), dtype=torch.float32, device="cuda")
        ieti.ieti_mlp_forward(m, x[67:68].contiguous(), y1)
        assert torch.equal(y1[0], y[67])
    finally:
        ieti.ieti_mlp_destroy(m)


def test_gradients_match_oracle(ieti):
    params = _f32(om.init_params(NI, NH, NO, seed=5))
    X, T = _data(6)
    m = _net(ieti, params)
    try:
        x = torch.tensor(X, dtype=torch.float32, device="cuda")
        t = torch.tensor(T, dtype=torch.float32, device="cuda")
        loss = ieti.ieti_mlp_backward(m, x, t)
        g = _split(ieti.ieti_mlp_get(m, 1))
        L, G = om.loss_and_grads(params, np.asarray(X, np.float32).astype(np.float64),
                                 np.asarray(T, np.float32).astype(np.float64))
        assert abs(loss - L) <= 1e-4 * L
        for name, a, b in zip(["dW1", "db1", "dW2", "db2", "dW3", "db3"], g, G):
            assert relf(a, b) <= 2e-3, name
    finally:
        ieti.ieti_mlp_destroy(m)


def test_adam_steps_match_oracle(ieti):
    """Three Adam steps applied to the library's own gradients equal the
    oracle's Adam update of the same gradients (FP32 against FP64 arithmetic)."""
    params = _f32(om.init_params(NI, NH, NO, seed=7))
    X, T = _data(8)
    m = _net(ieti, params)
    try:
        x = torch.tensor(X, dtype=torch.float32, device="cuda")
        t = torch.tensor(T, dtype=torch.float32, device="cuda")
        ref = [p.copy() for p in params]
        state = (0, [np.zeros_like(p) for p in ref], [np.zeros_like(p) for p in ref])
        for _ in range(3):
            ieti.ieti_mlp_backward(m, x, t, want_loss=False)
            g = _split(ieti.ieti_mlp_get(m, 1))
            ieti.ieti_mlp_adam(m, 1e-3)
            state = om.adam_step(ref, g, state, 1e-3)
            got = _split(ieti.ieti_mlp_get(m, 0))
            for a, b in zip(got, ref):
                assert np.abs(a - b).max() <= 1e-5 * 1e-3 + 1e-6 * np.abs(b).max()
    finally:
        ieti.ieti_mlp_destroy(m)


def test_fit_single_batch_is_one_backward_and_adam_step(ieti):
    """ieti_mlp_fit with one full batch and one epoch computes the full-batch
    gradient (rows in shuffled order) and takes one Adam step."""
    params = _f32(om.init_params(NI, NH, NO, seed=9))
    X, T = _data(10)
    x = torch.tensor(X, dtype=torch.float32, device="cuda")
    t = torch.tensor(T, dtype=torch.float32, device="cuda")
    m1, m2 = _net(ieti, params), _net(ieti, params)
    try:
        ieti.ieti_mlp_fit(m1, x, t, batch=B, epochs=1, lr=1e-3, normalise=False, seed=3)
        ieti.ieti_mlp_backward(m2, x, t, want_loss=False)
        g1, g2 = ieti.ieti_mlp_get(m1, 1), ieti.ieti_mlp_get(m2, 1)
        assert relf(g1.astype(np.float64), g2.astype(np.float64)) <= 1e-5
        ieti.ieti_mlp_adam(m2, 1e-3)
        p1, p2 = ieti.ieti_mlp_get(m1, 0), ieti.ieti_mlp_get(m2, 0)
        # an update can differ only where the gradient is at FP32 noise level
        assert np.mean(np.abs(p1 - p2) > 1e-7) <= 1e-3
    finally:
        ieti.ieti_mlp_destroy(m1)
        ieti.ieti_mlp_destroy(m2)


def test_fit_normalisation_statistics(ieti):
    rng = np.random.default_rng(11)
    X = rng.standard_normal((300, NI)) * rng.uniform(0.1, 5, NI) + rng.uniform(-3, 3, NI)
    X[:, 7] = 2.5   # constant feature: scale 1
    T = rng.standard_normal((300, NO)) * 0.01
    m = ieti.ieti_mlp_create(NI, NH, NO, 64)
    try:
        ieti.ieti_mlp_set_params(m, _flat(_f32(om.init_params(NI, NH, NO, seed=12))))
        x = torch.tensor(X, dtype=torch.float32, device="cuda")
        t = torch.tensor(T, dtype=torch.float32, device="cuda")
        ieti.ieti_mlp_fit(m, x, t, batch=64, epochs=1, lr=1e-4, normalise=True)
        s = ieti.ieti_mlp_get(m, 2)
        X32, T32 = X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64)
        mean, std = X32.mean(0), X32.std(0)
        assert np.abs(s[:NI] - mean).max() <= 1e-5 * np.abs(mean).max()
        ok = np.arange(NI) != 7
        assert np.abs(s[NI:2 * NI][ok] * std[ok] - 1).max() <= 1e-5
        assert s[NI + 7] == 1.0
        assert abs(s[2 * NI] - np.sqrt(np.mean(T32 ** 2))) <= 1e-5 * np.sqrt(np.mean(T32 ** 2))
    finally:
        ieti.ieti_mlp_destroy(m)


def test_training_reduces_the_loss(ieti):
    """A smooth synthetic map is learned: the last-epoch loss after 150 epochs
    is far below the loss of the first epoch (same normalisation)."""
    rng = np.random.default_rng(13)
    n = 512
    X = rng.standard_normal((n, NI))
    A = rng.standard_normal((NI, 16)) / np.sqrt(NI)
    C = rng.standard_normal((16, NO))
    T = np.tanh(X @ A) @ C
    x = torch.tensor(X, dtype=torch.float32, device="cuda")
    t = torch.tensor(T, dtype=torch.float32, device="cuda")
    m = ieti.ieti_mlp_create(NI, NH, NO, 64)
    try:
        ieti.ieti_mlp_set_params(m, _flat(_f32(om.init_params(NI, NH, NO, seed=14))))
        l1 = ieti.ieti_mlp_fit(m, x, t, batch=64, epochs=1, lr=1e-3, seed=1)
        l150 = ieti.ieti_mlp_fit(m, x, t, batch=64, epochs=150, lr=1e-3, decay=0.98, seed=2)
        assert np.isfinite(l150) and l150 < 0.05 * l1
    finally:
        ieti.ieti_mlp_destroy(m)


def test_invalid_arguments_are_rejected(ieti):
    m = ieti.ieti_mlp_create(4, 8, 3, 5)
    try:
        x = torch.zeros((6, 4), dtype=torch.float32, device="cuda")
        y = torch.zeros((6, 3), dtype=torch.float32, device="cuda")
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_mlp_forward(m, x, y)          # batch 6 > max_batch 5
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_mlp_set_params(m, np.zeros(3))
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_mlp_fit(m, x, y, batch=5, epochs=1, lr=1e-3, decay=1.5)
        assert ieti.ieti_mlp_query(m) == {"n_in": 4, "n_hidden": 8, "n_out": 3, "max_batch": 5,
                                          "nparam": 8 * 4 + 8 + 64 + 8 + 24 + 3}
    finally:
        ieti.ieti_mlp_destroy(m)


def test_forward_combine_is_the_coefficient_sum_of_the_outputs(ieti):
    """lam[b] = out_scale * sum_c coef[b, c] y[b, c m : (c + 1) m] with n_out = 9 * 37."""
    params = _f32(om.init_params(NI, NH, NO, seed=15))
    X, _ = _data(16)
    m = _net(ieti, params)
    try:
        ieti.ieti_mlp_set_scaling(m, np.zeros(NI), np.ones(NI), out_scale=2.5)
        x = torch.tensor(X, dtype=torch.float32, device="cuda")
        y = torch.empty((B, NO), dtype=torch.float32, device="cuda")
        ieti.ieti_mlp_forward(m, x, y)
        coef = torch.tensor(np.random.default_rng(17).standard_normal((B, 9)), device="cuda")
        lam = torch.empty((B, NO // 9), dtype=torch.float64, device="cuda")
        ieti.ieti_mlp_forward_combine(m, x, coef, lam)
        yy = y.cpu().numpy().astype(np.float64) / 2.5       # y already carries out_scale
        ref = 2.5 * np.einsum("bc,bcj->bj", coef.cpu().numpy(), yy.reshape(B, 9, NO // 9))
        assert np.abs(lam.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_mlp_forward_combine(m, x, coef[:, :5].contiguous(), lam)
    finally:
        ieti.ieti_mlp_destroy(m)
