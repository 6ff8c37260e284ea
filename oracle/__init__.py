"""FP64 CPU oracle for the SplitSolve hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct numpy/scipy code in complex128.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it.  The CUDA library never calls it, and it never calls the CUDA
library; the only code both sides share is the seeded input generator
(``synth``), which holds none of the method's arithmetic.

Modules (each function cites the passage it follows):

* :mod:`oracle.leads`     -- lead cells, Sancho-Rubio doubling, self-energies
                             (decimation is named in Sec. 3A; the doubling
                             steps are the standard ones the citation points to).
* :mod:`oracle.dense`     -- the plain definition: dense (E S - H - Sigma) x = Inj
                             (Eq. wf, Eq. negf), Green's-function corners,
                             Caroli transmission, bond currents.
* :mod:`oracle.alg1`      -- Algorithm 1 (block-column inversion) and the
                             Sherman-Morrison-Woodbury steps 1-4 (Eq. x), in the
                             paper's order, for pins of the readings.
* :mod:`oracle.rgf`       -- recursive Green's-function corners for devices too
                             large for a dense matrix.
* :mod:`oracle.channels`  -- open-channel count from the lead's quadratic pencil
                             (the one-neighbour case of Eq. bound).
* :mod:`oracle.chol`      -- rank-revealing pivoted Cholesky (Gamma = V V^H).
* :mod:`oracle.mlp`       -- FP64 forward/backward/Adam of the warm-start MLP.
* :mod:`oracle.warm`      -- Dyson residual and seeded fixed-point iteration of
                             the surface Green's function.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an identity or brute force, except where its docstring says
"parity unpinned".
"""
from . import leads, dense, alg1, rgf, channels, chol, mlp, warm  # noqa: F401

__all__ = ["leads", "dense", "alg1", "rgf", "channels", "chol", "mlp", "warm"]
