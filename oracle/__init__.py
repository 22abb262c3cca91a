"""CPU oracle for the DFT+U CheFSI hot path: test infrastructure, not product code.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
reference legs) may import this package.  The CUDA library never imports, links or calls
it, and it imports nothing from the library.
"""
from . import density_scf, hubbard, mlp  # noqa: F401
