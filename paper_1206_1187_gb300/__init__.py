"""GB300 (sm_103a) implementation of the alpha_{2,3} random variate generator
of Beliakov, Johnstone, Creighton and Wilkin, "Parallel random variates
generator for GPUs based on normal numbers" (Algorithm BB, Eq. 2, Eq. 3).

The compute path is the C-ABI library ``libbcn_rng.so`` (include/bcn_rng.h);
``paper_1206_1187_gb300.rng`` binds it.  Importing this package does not load
the library; the first use of an API name does, and fails loudly if the
library is not built.
"""
from __future__ import annotations

_API = {"Stream", "generate_at", "generate_at_ptr", "fill_constant", "resolve_tune",
        "make_tune", "Tune", "RNGError", "version", "SEED_MIN", "SEED_MAX", "PERIOD",
        "MAX_N"}


def __getattr__(name):
    if name in _API:
        from . import rng
        return getattr(rng, name)
    raise AttributeError(name)
