"""The warm-start model's kernels (hub_descriptors, hub_mlp_*) against the FP64 CPU oracle
of the same definitions: descriptors, forward pass, loss, exact gradients and one Adam step."""
import numpy as np
import pytest

import workloads as w
from oracle import mlp as om

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_23612_gb300 import MLP, descriptors  # noqa: E402

DEV = torch.device("cuda:0")
SIZES = [48, 64, 64, 64, 30]    # 3 hidden layers; ragged against the 64-wide tiles below


def _flat(params):
    return np.concatenate([np.concatenate([W.reshape(-1), b]) for W, b in params]).astype(np.float32)


def _unflat(flat, sizes):
    out, o = [], 0
    for nin, nout in zip(sizes[:-1], sizes[1:]):
        W = flat[o:o + nin * nout].reshape(nout, nin)
        o += nin * nout
        b = flat[o:o + nout]
        o += nout
        out.append((W.astype(np.float64), b.astype(np.float64)))
    return out


def _problem(B, seed, sizes=SIZES):
    g = np.random.Generator(np.random.PCG64(seed))
    params = [(W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64))
              for W, b in om.init_params(sizes, seed)]
    X = g.normal(0.3, 2.0, (B, sizes[0])).astype(np.float32)
    T = g.normal(0.1, 0.5, (B, sizes[-1])).astype(np.float32)
    mu_in = X.mean(0).astype(np.float32)
    sd_in = (X.std(0) + 0.1).astype(np.float32)
    mu_out = T.mean(0).astype(np.float32)
    sd_out = (T.std(0) + 0.1).astype(np.float32)
    norm = tuple(v.astype(np.float64) for v in (mu_in, sd_in, mu_out, sd_out))
    return params, X, T, (mu_in, sd_in, mu_out, sd_out), norm


def _model(params, normf, fp16, sizes=SIZES):
    m = MLP(sizes[0], sizes[1], len(sizes) - 2, sizes[-1], fp16=fp16, seed=1)
    m.set_params(_flat(params))
    m.set_normalization(*normf)
    return m


@pytest.mark.parametrize("B", [1, 37, 200])
def test_forward_matches_oracle(B):
    params, X, T, normf, norm = _problem(B, 11)
    y_ref, _ = om.forward(params, X.astype(np.float64), norm)
    for fp16, tol in ((False, 2e-6), (True, 3e-3)):
        m = _model(params, normf, fp16)
        Y = torch.empty((B, SIZES[-1]), dtype=torch.float32, device=DEV)
        m.forward(torch.tensor(X, device=DEV), Y)
        err = np.max(np.abs(Y.cpu().numpy() - y_ref)) / np.max(np.abs(y_ref))
        assert err < tol, (fp16, err)
        m.close()


@pytest.mark.parametrize("fp16", [False, True])
def test_loss_and_gradients_match_oracle(fp16):
    B = 130
    params, X, T, normf, norm = _problem(B, 12)
    loss_ref, grads_ref = om.loss_and_grads(params, X.astype(np.float64), T.astype(np.float64), norm)
    m = _model(params, normf, fp16)
    loss, g = m.loss_grad(torch.tensor(X, device=DEV), torch.tensor(T, device=DEV))
    gref = _flat([(gw, gb) for gw, gb in grads_ref]).astype(np.float64)
    tol = 3e-3 if fp16 else 2e-5
    assert abs(loss - loss_ref) < tol * loss_ref
    # per layer, relative to the layer's largest gradient entry
    o = 0
    for (gw, gb) in grads_ref:
        n = gw.size + gb.size
        err = np.max(np.abs(g[o:o + n] - gref[o:o + n])) / np.max(np.abs(gref[o:o + n]))
        assert err < tol, err
        o += n
    m.close()


def test_gradient_against_finite_differences_of_the_oracle_loss():
    """The oracle's own gradient pinned by central differences (so the GPU check above
    compares with a correct gradient, not just the same formula)."""
    B = 9
    sizes = [5, 7, 6, 3]
    params, X, T, _, norm = _problem(B, 13, sizes)
    _, grads = om.loss_and_grads(params, X.astype(np.float64), T.astype(np.float64), norm)
    h = 1e-6
    for li, (W, b) in enumerate(params):
        for idx in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            Wp = [(w_.copy(), b_.copy()) for w_, b_ in params]
            Wm = [(w_.copy(), b_.copy()) for w_, b_ in params]
            Wp[li][0][idx] += h
            Wm[li][0][idx] -= h
            fd = (om.loss_and_grads(Wp, X, T, norm)[0] - om.loss_and_grads(Wm, X, T, norm)[0]) / (2 * h)
            assert abs(fd - grads[li][0][idx]) < 1e-6 * max(1.0, abs(fd))


def test_adam_step_matches_oracle():
    B = 64
    params, X, T, normf, norm = _problem(B, 14)
    _, grads = om.loss_and_grads(params, X.astype(np.float64), T.astype(np.float64), norm)
    zeros = lambda: [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]  # noqa: E731
    lr = 1e-2
    new_ref, _ = om.adam_step(params, grads, (0, zeros(), zeros()), lr)
    m = _model(params, normf, False)
    m.train_step(torch.tensor(X, device=DEV), torch.tensor(T, device=DEV), lr)
    p1 = m.get_params().astype(np.float64)
    d_ref = _flat(new_ref).astype(np.float64) - _flat(params).astype(np.float64)
    d_gpu = p1 - _flat(params).astype(np.float64)
    g = np.abs(_flat(grads))
    big = g > 1e-4 * g.max()
    # first Adam step: lr * g / (|g| + eps) -- the sign of the gradient, scaled by lr
    assert np.max(np.abs(d_gpu[big] - d_ref[big])) < 1e-3 * lr
    assert np.all(np.abs(d_gpu) <= lr * (1 + 1e-5))
    m.close()


def test_training_reduces_loss_and_is_deterministic():
    B = 256
    params, X, T, normf, _ = _problem(B, 15)
    # a smooth target the network can fit
    T = np.tanh(X[:, :SIZES[-1]] * 0.5).astype(np.float32)
    Xd, Td = torch.tensor(X, device=DEV), torch.tensor(T, device=DEV)
    runs = []
    for _ in range(2):
        m = MLP(SIZES[0], SIZES[1], 3, SIZES[-1], fp16=True, seed=3)
        m.fit_normalization(Xd, Td)
        l0 = m.train_step(Xd, Td, 3e-3)
        for _ in range(300):
            last = m.train_step(Xd, Td, 3e-3)
        runs.append((l0, last, m.get_params()))
        m.close()
    assert runs[0][1] < 0.1 * runs[0][0]
    assert runs[0][1] == runs[1][1]
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


def test_fit_normalization_matches_numpy():
    g = np.random.Generator(np.random.PCG64(5))
    X = g.normal(1.0, 3.0, (333, 48)).astype(np.float32)
    T = g.normal(0.0, 0.2, (333, 30)).astype(np.float32)
    m = MLP(48, 32, 1, 30, fp16=False, seed=0)
    m.fit_normalization(torch.tensor(X, device=DEV), torch.tensor(T, device=DEV))
    # with zero weights and biases the output is mu_out
    m.set_params(np.zeros(m.nparams, dtype=np.float32))
    Y = torch.empty((2, 30), dtype=torch.float32, device=DEV)
    m.forward(torch.tensor(X[:2], device=DEV), Y)
    np.testing.assert_allclose(Y.cpu().numpy()[0], T.astype(np.float64).mean(0), rtol=1e-5, atol=1e-6)
    m.close()


@pytest.mark.parametrize("reps", [(1, 1, 1), (2, 2, 1)])
def test_descriptors_match_oracle(reps):
    L, pti, po = w.synthetic._supercell(w.synthetic.rutile_cell(), reps)
    pti = w.synthetic.displaced(pti, 0.1, 3)
    po = w.synthetic.displaced(po, 0.1, 4)
    pos = np.asarray(list(pti) + list(po))
    sp = np.asarray([0] * len(pti) + [1] * len(po), dtype=np.int32)
    centres = np.arange(len(pti), dtype=np.int32)
    ref = om.descriptors(pos, sp, L, centres)
    out = torch.empty(ref.shape, dtype=torch.float32, device=DEV)
    descriptors(pos, sp, L, centres, out)
    got = out.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
