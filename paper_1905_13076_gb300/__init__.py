"""GB300-native periodic Parareal (PP-PC) with a multi-harmonic coarse solve
for the periodic eddy-current problem M du/dt + K(u) u = f(t), u(0) = u(T).

The compute path is the CUDA library ``libpppc.so`` (C ABI in
``include/pppc.h``); this package only marshals arguments to it.
"""

from ._lib import PPPCError, load  # noqa: F401
from .solver import PPPC, Material, PPPCBatch, from_problem  # noqa: F401
