"""GB300 (sm_103a) batched Lennard-Jones local minimisation and Basin Hopping.

``paper_2510_25938_gb300.lj_bh`` is the ctypes binding of the CUDA library
(include/lj_bh.h); ``paper_2510_25938_gb300.inputs`` makes seeded synthetic
starting structures; ``paper_2510_25938_gb300.build`` compiles the library;
``paper_2510_25938_gb300.molden`` reads and writes Molden geometry files and
``python -m paper_2510_25938_gb300 input.molden`` (cli.py) runs Basin Hopping
on a structure read from one, writing the accepted structures.
Nothing is imported eagerly, so the input generators work without torch/CUDA.
"""
