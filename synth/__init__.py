"""Seeded synthetic inputs shaped like the paper's test problems.

This package only draws and lays out input data (initial fields, edge and
material descriptions). It contains none of the method's arithmetic and is
shared by the tests, the benchmark and the smoke check.
"""
from .generators import *  # noqa: F401,F403
