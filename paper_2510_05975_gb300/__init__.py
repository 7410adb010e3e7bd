"""alpha-CNG on GB300: exact-candidate alpha-convergent neighbourhood graph build and batched
beam search (arXiv 2510.05975), as hand-written sm_103a CUDA behind a C ABI (libcng.so).

``cng`` is the thin ctypes binding; ``synth`` the seeded workload generators.  Importing the
package does not touch the GPU; the CUDA library loads on first use and raises if it is
missing.
"""
