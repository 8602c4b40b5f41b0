"""Seeded synthetic workload generators (CNF instances, initial logits).

This package holds input generation only: it draws random instances and writes
them as DIMACS text.  It contains none of the sampler's arithmetic (no
relaxation, no gradients, no verification), so both the CUDA path and the CPU
oracle may consume its output.
"""
from .generators import (  # noqa: F401
    TseitinInstance, PlantedSATInstance,
    tseitin_random_circuit, planted_3sat, fig1_example_dimacs,
    dimacs_text, normal_logits, mlp_params, normal_vector,
)
