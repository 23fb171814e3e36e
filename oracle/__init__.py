"""FP64 CPU oracle of the neural in-scattering estimator (arXiv 2401.14051).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference leg may import or run anything in this package.  The product
package ``paper_2401_14051_gb300`` never imports it and shares no code with it; both take
their inputs from the seeded generators in ``synth``.
"""
from .nis_oracle import *  # noqa: F401,F403
