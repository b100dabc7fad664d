"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This package draws mechanisms and cell states. It holds none of the
integrator's arithmetic: no rates, no thermodynamic functions of T, no ODE.
The one exception is the sign of the standard reaction enthalpy at 298.15 K,
a sum of drawn formation enthalpies, which only orients each reaction.
"""
from .mechfile import Mechanism, read_mech, write_mech
from .mechgen import generate_mechanism, nasa7_of_linear, with_falloff, with_nasa7, with_plog
from . import states

__all__ = ["Mechanism", "read_mech", "write_mech", "generate_mechanism", "with_falloff", "with_plog", "with_nasa7", "nasa7_of_linear", "states"]
