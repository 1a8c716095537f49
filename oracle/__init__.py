"""FP64 CPU oracle for the AAA-Gaussians renderer (arXiv 2504.12811).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline / reference legs of `bench.py` may import this package.  The
product path (`paper_2504_12811_gb300`) never imports it, and the two share no
code: the only common module is the seeded input generator
`paper_2504_12811_gb300.scenes`, which draws inputs and holds no step of the
method.

The oracle is a plain, slow, obviously-correct restatement of what the paper
computes, in float64 on the float32 inputs, with plain PyTorch CPU ops (so
autograd gives the analytic gradient of the same definition).  Every function
cites the section / equation it follows; where the paper leaves a choice
open, the function states the reading it takes.

Pins (tests/test_oracle_pins.py) tie each function to something other than
itself: closed forms, library routines (scipy rotations and spherical
harmonics), brute-force sampling, the plane form of Eq. 4-5, finite
differences, invariants.  No function here is "parity unpinned".
"""
from .aaa import *  # noqa: F401,F403
from .aaa import __all__  # noqa: F401
