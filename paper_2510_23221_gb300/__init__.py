"""GB300-native BlocKOA hot path: block-CG basis solve, combination, operator action.

The compute path lives in ``libblockoa.so`` (CUDA for sm_103a) behind a C ABI;
``paper_2510_23221_gb300.blockoa`` is its thin ctypes binding.  Importing this
package does not load the library; the binding loads it on first use and
raises if it is missing.
"""
__all__ = ["synth", "blockoa"]
