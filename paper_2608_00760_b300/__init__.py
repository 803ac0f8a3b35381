"""B300-native differentiable multigrid solver for -div(D grad u) + mu u = q.

The solver (forward V-cycle solve, JVP and the analytically derived VJP through
the whole grid hierarchy, arXiv 2608.00760 Secs. 2.2-2.4) lives in hand-written
sm_103a CUDA kernels behind the C ABI declared in ``include/dmg.h``
(``libdmg.so``). ``paper_2608_00760_b300.dmg`` is a thin ctypes binding with the
same names; ``paper_2608_00760_b300.autograd`` wraps it in a
``torch.autograd.Function``. The shared library is loaded on first use and
its absence raises an error: there is no CPU fallback.
"""

__all__ = ["dmg", "autograd", "inputs"]
