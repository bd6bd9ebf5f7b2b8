"""Seeded synthetic inputs (phantoms, exact sinograms, detector counts).

Input generation only, shared by the tests and the benchmark; it contains no
reconstruction arithmetic.
"""
from . import phantoms, acquisition  # noqa: F401
