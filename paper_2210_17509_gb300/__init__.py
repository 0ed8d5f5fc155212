"""GB300-native GRMHD method-of-lines hot path (Valencia formulation, GRaM-X).

The compute path is the CUDA library ``libgrmhd.so`` (sources in ``csrc/``,
C ABI in ``include/grmhd.h``).  ``paper_2210_17509_gb300.grmhd`` is the thin
binding with the same entry-point names; it raises if the library is missing.
``paper_2210_17509_gb300.inputs`` holds the seeded synthetic input generators.
"""
