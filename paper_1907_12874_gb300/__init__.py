"""BiCGStab with k right-hand sides on GB300 (sm_103a).

Krasnopolsky, "Revisiting Performance of BiCGStab Methods for Solving Systems
with Multiple Right-Hand Sides" (arXiv:1907.12874).
"""
from . import inputs  # noqa: F401

__all__ = ["inputs"]
