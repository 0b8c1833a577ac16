"""CPU FP64 oracle for the RGF selected inversion -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import this package.  The product path (the CUDA library and its Python binding) never imports,
links or executes anything here; the two share no code, only the seeded inputs of ``workloads``.

Contents (numpy complex128 throughout, one energy at a time, LAPACK ``inv`` as the only primitive
beyond matrix products):

* ``dense``       -- the plain definition the method reaches exactly (Eq. 2 with Table I's
                     G-row: M = E S - H - Sigma^R, B = Sigma^<): G^R = M^-1, G^< = G^R B G^A,
                     restricted to the block-tridiagonal pattern.  Tiny sizes only.
* ``leads``       -- lead (contact) retarded self-energies by Sancho-Rubio decimation
                     (ref. of Sigma^R in Table I's G-row; the decimation itself is the
                     Lopez Sancho-Sancho-Rubio iteration).
* ``rgf``         -- the forward/backward block recursion (block Gaussian elimination of Sec. IV-A,
                     Eq. 6's "stabilized Gaussian elimination"; the selected-inversion algorithm the
                     paper cites for Eq. 2) for G^R, G^<, G^> and the observables of Sec. II-B
                     (current, density, contact currents, transmission).

Pins (tests/test_oracle_*.py, all ``-m "not gpu"``): the recursion against ``dense`` on tiny
random inputs; the decimation against the closed-form self-energy of a clean strip and against a
long truncated lead solved densely; the clean strip's integer transmission and Landauer current;
the invariants G^> - G^< = G^R - G^A, anti-Hermitian G^<, PSD spectral function, exact current
continuity, and the equilibrium (fluctuation-dissipation) case.
"""
from .dense import dense_selected  # noqa: F401
from .leads import sancho_rubio, lead_self_energy, fermi  # noqa: F401
from .rgf import rgf_energy, solve, observables, integrate  # noqa: F401
