"""Test helpers: put one seeded workload into both the CUDA library (through the C ABI) and
the CPU oracle.  The two sides share only the workload's inputs."""
import numpy as np

from oracle import hubbard as o


def torch_dev():
    import torch
    return torch.device("cuda:0")


def make_hub(wl, prec=0, kidx=0, complex_=None):
    import torch
    from paper_2507_23612_gb300 import Hub
    kpt = wl.kpts[kidx]
    cplx = bool(np.any(np.asarray(kpt) != 0)) if complex_ is None else complex_
    hb = Hub(wl.n, wl.L, wl.fd_half_order, kpt=kpt, complex_=cplx, prec=prec)
    hb.set_veff(torch.tensor(wl.veff, dtype=torch.float64, device=torch_dev()))
    hb.set_atoms(wl.atoms)
    return hb


def oracle_ham(wl, kidx=0, D=None):
    g = o.Grid(wl.n, wl.L, wl.kpts[kidx], wl.fd_half_order)
    return o.Hamiltonian(g, wl.veff, wl.atoms, D)


def to_dev(X_cols, dtype):
    """(ncol, Nd) numpy -> torch CUDA tensor of the same layout."""
    import torch
    return torch.tensor(np.ascontiguousarray(X_cols), device=torch_dev()).to(dtype).contiguous()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def rel_elem(a, b):
    """Element-by-element error: max over elements of |a - b| divided by the RMS magnitude
    of the reference row the element belongs to (one orbital of a [ncol, Nd] block, one row
    of a matrix; a vector is one row).  A single wrong element stands out against its own
    orbital's scale instead of being averaged into a whole-block norm."""
    a = np.asarray(a)
    b = np.asarray(b)
    if b.ndim == 1:
        a, b = a[None, :], b[None, :]
    a = a.reshape(-1, a.shape[-1]) if a.ndim > 2 else a
    b = b.reshape(-1, b.shape[-1]) if b.ndim > 2 else b
    rms = np.sqrt(np.mean(np.abs(b) ** 2, axis=1))
    scale = np.maximum(rms, 1e-300 + 1e-30 * float(np.max(rms)))
    return float(np.max(np.max(np.abs(a - b), axis=1) / scale))
