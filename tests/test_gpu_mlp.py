"""The cost model's CUDA kernels (forward, loss, backward, Adam) against the
FP64 oracle network, plus training, checkpointing and selection."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

F, H, V = 34, 16, 5


def split(flat):
    out, o = {}, 0
    for name, shape in omlp.shapes(F, H, V).items():
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape).astype(np.float64)
        o += n
    return out


def problem(seed, M=40):
    rng = np.random.default_rng(seed)
    params = rng.normal(0, 0.3, sum(int(np.prod(s)) for s in omlp.shapes(F, H, V).values())).astype(np.float32)
    X = rng.normal(0, 1, (M, F)).astype(np.float32)
    T = rng.normal(0, 1, (M, V)).astype(np.float32)
    mask = (rng.random((M, V)) < 0.8).astype(np.float32)
    mean = rng.normal(0, 0.5, F).astype(np.float32)
    inv = rng.uniform(0.5, 2.0, F).astype(np.float32)
    return params, X, T, mask, mean, inv


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_loss_and_gradients_match_oracle(lib, seed):
    import torch
    params, X, T, mask, mean, inv = problem(seed)
    m = lib.spmv_model_create(F, H, V, params)
    try:
        lib.spmv_model_set_normalizer(m, mean, inv)
        Xd, Td, Md = (torch.from_numpy(a).cuda() for a in (X, T, mask))
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        grad = torch.zeros(params.size, dtype=torch.float32, device="cuda")
        Y = torch.zeros((X.shape[0], V), dtype=torch.float32, device="cuda")
        lib.spmv_model_forward(m, Xd.data_ptr(), X.shape[0], Y.data_ptr(), 0)
        lib.spmv_model_loss_grad(m, Xd.data_ptr(), Td.data_ptr(), Md.data_ptr(), X.shape[0], loss.data_ptr(),
                                 grad.data_ptr(), 0)
        torch.cuda.synchronize()
        p = split(params)
        Xn = (X.astype(np.float64) - mean) * inv
        Yr, cache = omlp.forward(p, Xn)
        lr = omlp.loss(Yr, T.astype(np.float64), mask.astype(np.float64))
        gr = omlp.backward(p, cache, Yr, T.astype(np.float64), mask.astype(np.float64))
        assert rel_err(Y.cpu().numpy(), Yr) < 1e-5
        assert abs(float(loss.item()) - lr) <= 1e-5 * abs(lr)
        g = split(grad.cpu().numpy())
        for name in omlp.PARAM_NAMES:
            assert rel_err(g[name], gr[name]) < 1e-5, name
    finally:
        lib.spmv_model_destroy(m)


def test_adam_step_matches_oracle(lib):
    import torch
    params, X, T, mask, mean, inv = problem(3)
    rng = np.random.default_rng(3)
    g = rng.normal(0, 1, params.size).astype(np.float32)
    m = lib.spmv_model_create(F, H, V, params)
    try:
        gd = torch.from_numpy(g).cuda()
        p = split(params)
        st = {}
        for t in (1, 2, 3):
            lib.spmv_model_adam_step(m, gd.data_ptr(), 0.01, 0.9, 0.999, 1e-8, 0)
            omlp.adam_step(p, split(g), st, t, lr=0.01)
        got = split(lib.spmv_model_get_params(m))
        for name in omlp.PARAM_NAMES:
            assert rel_err(got[name], p[name]) < 1e-6, name
        assert lib.spmv_model_info(m)[4] == 3
    finally:
        lib.spmv_model_destroy(m)


def test_training_checkpoint_and_select(lib, tmp_path):
    import torch
    from paper_1101_0091_gb300 import selector
    rng = np.random.default_rng(5)
    M = 200
    X = rng.normal(0, 1, (M, selector.N_FEATURES))
    # targets with a learnable structure: the best variant depends on the sign of feature 0
    T = np.stack([X[:, 0], -X[:, 0], 0.5 * X[:, 1]], axis=1)
    data = selector.Dataset(X, T, np.exp(T))
    cm = selector.CostModel(3, hidden=32, seed=1)
    curve = cm.fit(data, epochs=600, lr=3e-3)
    assert curve[-1] < 0.1 * curve[0]
    choice, pred = cm.select(X)
    assert np.array_equal(choice, pred.argmin(axis=1))
    assert np.mean(choice == T.argmin(axis=1)) > 0.9
    path = str(tmp_path / "model.bin")
    cm.save(path)
    cm2 = selector.CostModel.load(path)
    assert np.array_equal(lib.spmv_model_get_params(cm.handle), lib.spmv_model_get_params(cm2.handle))
    assert lib.spmv_model_info(cm2.handle)[4] == lib.spmv_model_info(cm.handle)[4]
    c2, p2 = cm2.select(X)
    assert np.array_equal(choice, c2) and np.array_equal(pred, p2)
    cm.close()
    cm2.close()
    with pytest.raises(lib.SpmvError):
        lib.spmv_model_load(str(tmp_path / "missing.bin"))
