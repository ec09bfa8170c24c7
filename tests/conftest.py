"""Shared pytest configuration.

Markers: ``gpu`` -- needs a CUDA GPU (the parity tests proper, through the C ABI).
Everything else runs on the CPU: the oracle against its pins, host logic, and
the C ABI's symbol table.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU; calls the library through its C ABI")
    config.addinivalue_line("markers", "slow: long-running CPU test")
