"""GB300 (sm_103a) implementation of the per-timestep microscopic vehicle
update of arxiv 2406.10661 (a GPU-accelerated large-scale traffic simulator).

Modules:
  scenario  seeded synthetic road networks, demand and parameters (inputs)
  binding   ctypes binding of the C ABI in include/moss.h (Simulation, Batch)
  serving   continuous-batching request loop over the C ABI

The compiled library is loaded on first use of ``binding`` and must exist;
there is no CPU fallback.
"""
__all__ = ["scenario", "binding"]
