"""Test configuration: the `gpu` marker and import paths.

Tests marked ``gpu`` need a GB300 and the CUDA library built by ``__graft_entry__.build()``;
everything else runs on the CPU.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built liblbm.so")
    config.addinivalue_line("markers", "slow: long-running CPU oracle physics checks")
