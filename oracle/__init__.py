"""Plain, slow, FP64 CPU oracle for the NSPT/TEK polynomial-matrix hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
library's product path never calls it, and it shares no code with the CUDA
kernels: it is written from the paper's definitions (Eqs. 1-5 and the five
FFT-CONV steps of Sec. 2) with numpy matmul / tensordot as the only library
steps.

Modules
-------
polymat : the star product (Eq. 5) naive and by direct DFT (Sec. 2, Steps 1-5),
          its backward (the truncated correlation), helpers on series.
tek     : twist phases (Eq. 1), the order-truncated TEK action, the staple and
          drift of Eqs. 2-3, exp-star and one Langevin step.
noise   : the Langevin step's traceless Hermitian noise drawn from the
          counter-based generator Philox4x32-10 (its published definition), for
          the library's seeded noise call.

Every function is pinned by ``tests/test_oracle_pins.py`` (``noise``: by
``tests/test_oracle_noise.py``, with the generator's published known-answer
vectors) against closed forms,
library routines on special cases, brute force or exact arithmetic; none of the
functions is "parity unpinned".
"""
from . import noise, polymat, tek  # noqa: F401
