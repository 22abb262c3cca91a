"""FP64 CPU oracle of the warm-start model: local-environment descriptors of a Hubbard atom
and a multilayer perceptron with SiLU activations, its mean-squared-error loss, the exact
gradients by backpropagation, and one Adam step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): it checks the CUDA kernels; the product
never imports it.

The paper gives no such model (it only points to learned U as future work); this is the
plain definition of what the library's kernels compute:
  descriptors (per centre atom I, neighbours J within rc over all periodic images, per
  neighbour species s):
    radial    G_sk = sum_J exp(-(r_IJ - mu_k)^2 / (2 eta^2)) fc(r_IJ),  k = 0..nrad-1
    angular   A_slm = sum_J Y_lm(r_IJ / |r_IJ|) fc(r_IJ),  l = 1 (3 values), l = 2 (5 values)
    fc(r) = (cos(pi r / rc) + 1) / 2 for r < rc, else 0
  network: h_0 = (x - mu_in) / sd_in;  h_l = silu(W_l h_{l-1} + b_l) for the hidden layers;
           y = (W_L h_{L-1} + b_L) * sd_out + mu_out,  silu(z) = z / (1 + exp(-z))
  loss:    mean over batch and outputs of ((y - t) / sd_out)^2
"""
from __future__ import annotations

from math import pi, sqrt
import numpy as np


def descriptor_params(rc: float = 6.0, nrad: int = 16, eta: float = 0.4):
    return dict(rc=rc, mu=np.linspace(0.5, rc - 0.5, nrad), eta=eta)


def _real_ylm_unit(l, u):
    x, y, z = u[..., 0], u[..., 1], u[..., 2]
    if l == 1:
        k = sqrt(3.0 / (4.0 * pi))
        return np.stack([k * y, k * z, k * x], axis=-1)
    k1, k0, k2 = 0.5 * sqrt(15.0 / pi), 0.25 * sqrt(5.0 / pi), 0.25 * sqrt(15.0 / pi)
    return np.stack([k1 * x * y, k1 * y * z, k0 * (2 * z * z - x * x - y * y), k1 * x * z, k2 * (x * x - y * y)], axis=-1)


def descriptors(pos, species, L, centers, nspecies: int = 2, rc: float = 6.0, nrad: int = 16, eta: float = 0.4):
    """pos (natoms, 3) bohr, species (natoms,) in 0..nspecies-1, L (3,) orthogonal cell,
    centers: indices of the centre atoms.  Returns (len(centers), nspecies * (nrad + 8))."""
    pos = np.asarray(pos, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    mu = np.linspace(0.5, rc - 0.5, nrad)
    nf = nrad + 8
    out = np.zeros((len(centers), nspecies * nf))
    tr = [range(-int(np.ceil(rc / L[a])) - 1, int(np.ceil(rc / L[a])) + 2) for a in range(3)]
    for ci, I in enumerate(centers):
        for J in range(len(pos)):
            for t1 in tr[0]:
                for t2 in tr[1]:
                    for t3 in tr[2]:
                        d = pos[J] + np.array([t1, t2, t3]) * L - pos[I]
                        r = float(np.sqrt(d @ d))
                        if r < 1e-8 or r >= rc:
                            continue
                        fc = 0.5 * (np.cos(pi * r / rc) + 1.0)
                        s = int(species[J])
                        base = s * nf
                        out[ci, base:base + nrad] += np.exp(-(r - mu) ** 2 / (2 * eta * eta)) * fc
                        u = d / r
                        out[ci, base + nrad:base + nrad + 3] += _real_ylm_unit(1, u) * fc
                        out[ci, base + nrad + 3:base + nrad + 8] += _real_ylm_unit(2, u) * fc
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, X, norm):
    """params: list of (W (out, in), b (out,)); norm: (mu_in, sd_in, mu_out, sd_out).
    Returns (y, cache)."""
    mu_in, sd_in, mu_out, sd_out = norm
    h = (np.asarray(X, dtype=np.float64) - mu_in) / sd_in
    cache = [h]
    zs = []
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        zs.append(z)
        h = silu(z) if li < len(params) - 1 else z
        cache.append(h)
    y = h * sd_out + mu_out
    return y, (cache, zs)


def loss_and_grads(params, X, T, norm):
    """MSE in normalised output units, and its exact gradient for every W and b."""
    mu_in, sd_in, mu_out, sd_out = norm
    y, (cache, zs) = forward(params, X, norm)
    B, nout = y.shape
    r = (y - T) / sd_out
    loss = float(np.mean(r * r))
    dh = 2.0 * r / (B * nout)          # d loss / d (normalised output) = d loss / d h_L
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        dz = dh if li == len(params) - 1 else dh * silu_grad(zs[li])
        grads[li] = (dz.T @ cache[li], dz.sum(axis=0))
        dh = dz @ W
    return loss, grads


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015) with bias correction; state = (t, m list, v list)."""
    t, ms, vs = state
    t += 1
    new = []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, ms, vs):
        out = []
        for p, g, m, v in ((W, gW, mW, vW), (b, gb, mb, vb)):
            m[...] = beta1 * m + (1 - beta1) * g
            v[...] = beta2 * v + (1 - beta2) * g * g
            mh = m / (1 - beta1 ** t)
            vh = v / (1 - beta2 ** t)
            out.append(p - lr * mh / (np.sqrt(vh) + eps))
        new.append(tuple(out))
    return new, (t, ms, vs)


def init_params(sizes, seed):
    """Seeded uniform init U(-1/sqrt(in), 1/sqrt(in)) for W and b (the usual default)."""
    g = np.random.Generator(np.random.PCG64(seed))
    params = []
    for nin, nout in zip(sizes[:-1], sizes[1:]):
        k = 1.0 / sqrt(nin)
        params.append((g.uniform(-k, k, (nout, nin)), g.uniform(-k, k, nout)))
    return params


def pack_D(D):
    """(nspin, natoms, 5, 5) -> (natoms, nspin * 15): upper triangles, row by row."""
    D = np.asarray(D)
    iu = np.triu_indices(5)
    return np.concatenate([D[s][:, iu[0], iu[1]] for s in range(D.shape[0])], axis=1)


def unpack_D(Y, nspin):
    """Inverse of pack_D (symmetric fill)."""
    Y = np.asarray(Y, dtype=np.float64)
    iu = np.triu_indices(5)
    out = np.zeros((nspin, Y.shape[0], 5, 5))
    for s in range(nspin):
        out[s][:, iu[0], iu[1]] = Y[:, 15 * s:15 * (s + 1)]
        out[s][:, iu[1], iu[0]] = Y[:, 15 * s:15 * (s + 1)]
    return out
