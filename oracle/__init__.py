"""CPU FP64 oracle for the ORI/RED scattering system (test infrastructure only).

This package is the independent checker of the GPU library.  It is plain,
slow and written to be read against the paper (Ramm & Tran, "A fast
algorithm for solving scalar wave scattering problem by billions of
particles"): every function cites the equation or section it restates.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import it.  The product path (``paper_1602_04691_gb300``)
never imports it and shares no code with it; the only module both sides use
is the seeded input generator ``paper_1602_04691_gb300.inputs``, which holds
none of the method's arithmetic.

Every function here is pinned by a ``-m "not gpu"`` test to something other
than itself (worked values printed in the paper, closed forms, invariants,
brute force on tiny grids).  No function is "parity unpinned".
"""

from .ori_oracle import *  # noqa: F401,F403
