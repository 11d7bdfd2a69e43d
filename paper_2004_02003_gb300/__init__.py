"""GB300-native BTO (Boundary Termination Optimization) Lagrangian flow-map
extraction: per-cycle RK4 advection of a seeded particle set through one
block's uniform-grid velocity field, termination of particles that leave the
block, and basis-flow output at the end of each interval.

The compute path is the C-ABI library ``libbto`` (hand-written sm_103a CUDA);
``paper_2004_02003_gb300.bto`` is its thin ctypes binding. Importing this
package loads nothing; the binding loads the library on first use and raises
if it is missing.
"""
__all__ = ["bto", "inputs"]
