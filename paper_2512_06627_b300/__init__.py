"""B300-native exact-simulation (ES) engine for combinational equivalence checking.

``circuits`` holds the seeded input generators (AIGs, miters, mutants).  The
engine itself is the C-ABI library ``liblec_es.so`` built from ``csrc/`` and
bound by ``lec_es``; importing this package does not load it.
"""
