"""FP64 CPU oracle for the e-ph scattering + coupled-BTE hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import it.  The CUDA library never links, calls or reads
anything here, and this package imports nothing from the CUDA path: the two share
only the seeded input generators (``paper_2109_08547_gb300.synthetic``).

Every function follows the paper's statement of the method (arXiv 2109.08547,
"Electrons, phonons, and interactions", "Coupled and decoupled BTEs",
"Transport coefficients") step by step, in the paper's order and notation, in
plain double precision.  Library primitives used as steps: numpy.linalg.eigh
(Hermitian eigen-decomposition) and matrix products.
"""
from .ephb_oracle import *  # noqa: F401,F403
from . import mlp_oracle  # noqa: F401
