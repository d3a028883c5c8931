"""CPU FP64 oracle of the hybrid mesh-Gaussian renderer.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library in paper_2506_06988_b300/.
"""
