"""GB300-native CG spectral-element RHS / Runge-Kutta hot path of the NUMA
dynamical core (Mueller et al., Sec. 2).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through the C-ABI declared in ``include/numa.h``; ``numa`` is its
thin ctypes binding.  Submodules are imported lazily so that ``inputs`` can
be used without the compiled library.
"""
