"""GB300-native ADMM solver for periodic micromechanics cells (Zhou & Bhattacharya,
"Accelerated computational micromechanics", Section 2).

The solver itself is the C-ABI library ``librve.so`` built from ``csrc/``; the
Python module :mod:`paper_2010_06697_gb300.rve` is a thin ctypes binding with the
same entry-point names.  :mod:`paper_2010_06697_gb300.synth` builds the seeded
synthetic inputs.  Importing this package loads nothing; the binding loads the
library on first use and raises if it has not been built.
"""
