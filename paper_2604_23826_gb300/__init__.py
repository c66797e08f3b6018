"""GB300-native sufficient-statistics pass (n, X^T 1, X^T X in one streaming pass).

The compute lives in libsuffstats.so (hand-written CUDA for sm_103a behind the
C ABI of include/stats.h); ``binding`` is its thin ctypes binding.
"""
from .binding import *  # noqa: F401,F403
from .binding import load, Config, Ctx, Raw, Analysis, StatsError  # noqa: F401
