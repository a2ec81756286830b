"""FP64 CPU oracle for the per-DM-trial periodicity search.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline / reference legs of ``bench.py``
import anything from this package.  The CUDA library never calls it, and it
shares no code, tables or constants with the CUDA library.

The paper (Yu et al., "A PRESTO-based Parallel Pulsar Search Pipeline Used
for FAST Drift Scan Data") names the pipeline steps -- RFI masking,
dedispersion over many DM values, FFT, periodicity/acceleration search,
sifting (Sect. 1 list of five steps; Sect. 2 steps 1-7) -- and the DM plans
(Tables 2-3), but states none of their mathematics.  Each function here
writes out the textbook definition of its step, in plain NumPy, with the
reading taken wherever the paper is silent stated in its docstring.

Pinning: every function is checked in ``tests/test_oracle_*.py`` against
something other than itself (closed forms, brute force, the plan tables'
printed counts, library special functions, Parseval).  Functions without
such a pin say "parity unpinned" in their docstring.
"""

from . import plan, dedisperse, spectrum, response, harmsum, stats, sift, search  # noqa: F401
