"""B300-native ISAAC volume ray caster (Matthes et al., 2016).

``synth`` generates seeded inputs; ``isaac`` binds the CUDA C-ABI library
``libisaac_b300.so`` (built by ``build.py``) and fails loudly if it is missing.
"""
__version__ = "0.1.0"
