"""Seeded synthetic inputs shared by the tests, the smoke check and bench.py.

This package holds NO arithmetic of the method: it only draws uniform
residues mod p and lengths with numpy's PCG64 generator, so that the oracle
and the CUDA path are fed identical inputs.  The paper uses no dataset; these
workloads stand in for the five benchmark configurations (shapes, sizes and
value distributions as listed in ``workloads.configs``).
"""

from .configs import (CONFIGS, Config, uniform_residues, config1_inputs,
                      config2_input, config3_inputs, config4_lengths,
                      config4_inputs, config5_schedule, modulus, elem_dtype)

__all__ = ["CONFIGS", "Config", "uniform_residues", "config1_inputs",
           "config2_input", "config3_inputs", "config4_lengths",
           "config4_inputs", "config5_schedule", "modulus", "elem_dtype"]
