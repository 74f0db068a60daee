"""FP64 CPU oracle for LoRADS (arXiv 2403.09133).

TEST INFRASTRUCTURE ONLY: a plain, slow restatement of the paper used to check the CUDA
library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the library.
"""
from .sdp import SDP  # noqa: F401
from .lorads import Params, kkt_report  # noqa: F401
from .lorads import lorads as solve  # noqa: F401
