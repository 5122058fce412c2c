"""FP64 CPU oracle of the boosted-frame PIC step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The CUDA library never does, and this
package never imports the library.
"""
from .oracle import Oracle, build_oracle, GridParams, PlasmaParams, LaserParams  # noqa: F401
