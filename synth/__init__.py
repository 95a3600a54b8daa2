"""Seeded synthetic inputs for the CVS-ADC(2) hot path.

This package draws random numbers and lays them out; it holds none of the
method's arithmetic.  The CPU oracle, the tests, ``bench.py`` and the smoke
check all take their inputs from here, so the CUDA path and the oracle see
bit-identical bytes.
"""

from .generate import (  # noqa: F401
    Instance,
    WORKLOADS,
    core_energies,
    make_instance,
    make_kramers_instance,
    make_spinfree_instance,
    batched_shapes,
    physical_scale,
)
