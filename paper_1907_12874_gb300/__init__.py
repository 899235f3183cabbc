"""BiCGStab with k right-hand sides on GB300 (sm_103a): CUDA library + thin binding.

Krasnopolsky, "Revisiting Performance of BiCGStab Methods for Solving Systems
with Multiple Right-Hand Sides" (arXiv:1907.12874): the CSR SpMM over an
RHS-interleaved block and the merged vector operations of the classical,
Reordered and Pipelined BiCGStab forms.  The solver runs only in the CUDA
library ``libbicgk.so``; the first call into ``bicgk`` loads it (building it
if its sources are newer) and raises if that fails.
"""
from . import bicgk, inputs  # noqa: F401

__all__ = ["bicgk", "inputs"]
