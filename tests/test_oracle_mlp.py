"""Pins for the warm-start oracle: backpropagated gradients against central finite
differences, Adam against its closed form on a quadratic, descriptors against symmetry and
hand-computed cases, and the D packing round trip."""
import numpy as np

from oracle import mlp as m


def _toy(seed=0):
    g = np.random.default_rng(seed)
    sizes = [6, 8, 8, 3]
    params = m.init_params(sizes, seed)
    X = g.standard_normal((5, 6))
    T = g.standard_normal((5, 3))
    norm = (g.standard_normal(6) * 0.1, 1 + g.uniform(0, 1, 6), g.standard_normal(3), 1 + g.uniform(0, 1, 3))
    return params, X, T, norm


def test_gradients_match_finite_differences():
    params, X, T, norm = _toy()
    loss, grads = m.loss_and_grads(params, X, T, norm)
    eps = 1e-6
    for li, (W, b) in enumerate(params):
        for arr, g in ((W, grads[li][0]), (b, grads[li][1])):
            idx = np.unravel_index(np.arange(arr.size)[:: max(1, arr.size // 7)], arr.shape)
            for k in zip(*idx):
                old = arr[k]
                arr[k] = old + eps
                lp, _ = m.loss_and_grads(params, X, T, norm)
                arr[k] = old - eps
                lm, _ = m.loss_and_grads(params, X, T, norm)
                arr[k] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(fd)), (li, k, fd, g[k])


def test_silu_gradient():
    z = np.linspace(-6, 6, 25)
    fd = (m.silu(z + 1e-6) - m.silu(z - 1e-6)) / 2e-6
    np.testing.assert_allclose(m.silu_grad(z), fd, atol=1e-8)


def test_adam_first_step_is_lr_times_sign():
    # with bias correction the first Adam step moves every parameter by lr * g / (|g| + eps')
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3]))]
    state = (0, [(np.zeros((1, 2)), np.zeros(1))], [(np.zeros((1, 2)), np.zeros(1))])
    new, state = m.adam_step(params, grads, state, lr=0.01)
    np.testing.assert_allclose(new[0][0], [[1.0 - 0.01, -2.0 + 0.01]], atol=1e-7)
    np.testing.assert_allclose(new[0][1], [0.5 - 0.01], atol=1e-4)
    assert state[0] == 1


def test_descriptor_symmetry_and_cases():
    L = np.array([10.0, 10.0, 10.0])
    # a lone atom: no neighbours within 6 bohr except its own images at 10 bohr -> zero
    d = m.descriptors([[1.0, 2.0, 3.0]], [0], L, [0])
    assert np.all(d == 0.0)
    # one neighbour at distance r along +x: radial peak where mu_k ~ r; only the
    # x-odd (Y_1,1) and x^2 terms are non-zero among the harmonics
    r = 2.5
    d = m.descriptors([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]], [0, 1], L, [0])[0]
    fc = 0.5 * (np.cos(np.pi * r / 6.0) + 1)
    mu = np.linspace(0.5, 5.5, 16)
    np.testing.assert_allclose(d[24:40], np.exp(-(r - mu) ** 2 / (2 * 0.16)) * fc, atol=1e-14)
    assert np.all(d[:24] == 0.0)                         # no species-0 neighbours
    k = np.sqrt(3 / (4 * np.pi))
    np.testing.assert_allclose(d[40:43], [0, 0, k * fc], atol=1e-14)
    # mirror image neighbour (-x) cancels the odd harmonics and doubles the even ones
    d2 = m.descriptors([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0], [5.0 - r, 5.0, 5.0]], [0, 1, 1], L, [0])[0]
    np.testing.assert_allclose(d2[40:43], 0.0, atol=1e-14)
    np.testing.assert_allclose(d2[43:48], 2 * d[43:48], atol=1e-14)


def test_pack_unpack_roundtrip():
    g = np.random.default_rng(1)
    A = g.standard_normal((2, 3, 5, 5))
    D = A + np.transpose(A, (0, 1, 3, 2))
    np.testing.assert_allclose(m.unpack_D(m.pack_D(D), 2), D)


def test_descriptor_rotation_covariance():
    """Rotating an environment by 90 degrees about z, (x, y, z) -> (-y, x, z), leaves the
    radial values unchanged and maps the harmonic sums in the fixed way the real Y_1m and
    Y_2m do: Y_1 (y, z, x) -> (x, z, -y); Y_2 (xy, yz, 2z^2-x^2-y^2, xz, x^2-y^2) ->
    (-xy, xz, 2z^2-x^2-y^2, -yz, -(x^2-y^2)).  A swapped or mis-signed component fails."""
    g = np.random.default_rng(7)
    L = np.array([30.0, 30.0, 30.0])
    c = L / 2
    rel = g.uniform(-4.0, 4.0, (7, 3))
    sp = [0] + list(g.integers(0, 2, 6))
    pos = np.vstack([c, c + rel[1:]])
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    pos_r = np.vstack([c, c + rel[1:] @ R.T])
    d = m.descriptors(pos, sp, L, [0])[0]
    dr = m.descriptors(pos_r, sp, L, [0])[0]
    for s in range(2):
        b = 24 * s
        np.testing.assert_allclose(dr[b:b + 16], d[b:b + 16], atol=1e-12)
        y1 = d[b + 16:b + 19]
        np.testing.assert_allclose(dr[b + 16:b + 19], [y1[2], y1[1], -y1[0]], atol=1e-12)
        y2 = d[b + 19:b + 24]
        np.testing.assert_allclose(dr[b + 19:b + 24], [-y2[0], y2[3], y2[2], -y2[1], -y2[4]], atol=1e-12)
    assert np.abs(d[16:24]).max() > 1e-3 and np.abs(d[40:48]).max() > 1e-3   # not a trivial case
