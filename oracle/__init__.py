"""FP64 CPU oracle of the constrained local approximate ideal restriction (CLAIR) AMG method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute
anything in this package.  Its only users are ``tests/``, ``__graft_entry__.smoke()``
(as the checker of one small GPU run) and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference`` arm, which time the oracle as it stands on the host cores).

It shares no code with the CUDA library: it is written from the paper's definitions
(Sections 2-4, Algorithm 1) in plain numpy/scipy, in float64, and every function cites
the passage it follows.  The only module both sides use is ``workloads`` (seeded input
generators, which hold none of the method's arithmetic).
"""
from .clair_oracle import *  # noqa: F401,F403
from . import adjoint  # noqa: F401
