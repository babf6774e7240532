"""GB300 (sm_103a) multigrid for the elliptic solves of arXiv:1809.08857.

The solver lives in the CUDA library ``libmg.so`` (C ABI, ``include/mg.h``);
``paper_1809_08857_gb300.mg`` is its thin ctypes binding.  Importing this
package loads nothing; the binding raises if the library is missing.
"""
__all__ = ["workloads", "mg"]
