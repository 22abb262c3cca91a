"""Molecular-dynamics steps of the DFT+U SCF (Sec. II.B, last paragraph): the starting
occupation matrices of a step from the atomic guess plus a second-order extrapolation of the
previous steps' residuals, or from the trained occupation model, the previous orbitals
reused; and checkpoints of an SCF (orbitals, D, metadata) to resume it.

Orchestration only: every SCF runs in the library (hub_scf_*), the extrapolation is
hub_extrapolate_occupations.
"""
from __future__ import annotations

import numpy as np

from .binding import HUB_F64, extrapolate_occupations
from .warmstart import scf_solve


def trajectory_scf(steps, prec: int = HUB_F64, start: str = "extrapolated", reuse_orbitals: bool = True,
                   tol_e_atom: float = 1e-5, tol_D: float = 1e-4, model=None, solve=None):
    """SCF at every step of a trajectory (a list of workloads on one grid).  The starting D of
    a step is the atomic guess (start="atomic"), the second-order extrapolation of the
    previous steps' converged D (start="extrapolated", hub_extrapolate_occupations with
    coefficients fitted to the positions; Sec. II.B), or the prediction of a trained
    OccupationModel (start="mlp", model=...).  With reuse_orbitals the previous step's
    converged orbitals start the next SCF.  solve(wl, prec, D0=..., X0=..., tol_e_atom=...,
    tol_D=...) runs one SCF (default scf_solve, the library's SCF driver) and returns its
    iterations, convergence, E, D, orbitals X and wall time.  Returns per step: iterations,
    E, the starting D, the extrapolation coefficients and the wall time."""
    solve = solve or (lambda wl, prec, **kw: scf_solve(wl, prec, keep_orbitals=True, **kw))
    if start not in ("atomic", "extrapolated", "mlp") or (start == "mlp" and model is None):
        raise ValueError("start must be atomic, extrapolated or mlp (with a model)")
    D_hist, R_hist, X, out = [], [], None, []
    for wl in steps:
        R = np.array([a.pos for a in wl.atoms])
        coef = (0.0, 0.0)
        if start == "extrapolated" and D_hist:
            h = min(3, len(D_hist))
            D0, coef = extrapolate_occupations(D_hist[-h:], wl.D0, R_hist[-h:] + [R])
        elif start == "mlp":
            D0 = model.predict(wl.atoms, wl.L)
        else:
            D0 = wl.D0
        r = solve(wl, prec, D0=D0, tol_e_atom=tol_e_atom, tol_D=tol_D,
                  X0=X if (reuse_orbitals and X is not None) else None)
        X = r["X"]
        D_hist.append(r["D"])
        R_hist.append(R)
        out.append({"iterations": r["iterations"], "converged": r["converged"], "E": r["E"],
                    "D0": np.asarray(D0), "D": r["D"], "alpha_beta": coef, "seconds": r["seconds"]})
    return out


def save_scf_checkpoint(path, Xs, D, meta=None):
    """Orbital blocks (one [ncol, Nd] tensor or array per spin), the occupation matrices and
    a small metadata dict (iteration, energy, seeds) in one .npz file."""
    arrays = {f"X{s}": (x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x))
              for s, x in enumerate(Xs)}
    np.savez(path, D=np.asarray(D, dtype=np.float64), nspin=len(Xs),
             meta=np.array(repr(dict(meta or {}))), **arrays)


def load_scf_checkpoint(path, device=None, dtype=None):
    """(Xs as device tensors, D, meta) of save_scf_checkpoint; with device None the blocks
    stay numpy arrays."""
    import ast
    z = np.load(path, allow_pickle=False)
    Xs = [z[f"X{s}"] for s in range(int(z["nspin"]))]
    if device is not None:
        import torch
        Xs = [torch.tensor(x, device=device, dtype=dtype).contiguous() for x in Xs]
    return Xs, z["D"], ast.literal_eval(str(z["meta"]))
