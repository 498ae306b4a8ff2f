"""Loads (building if needed) the product library for tests."""
import os

from paper_2608_03778_gb300 import _build


def ensure_built():
    _build.build()
    return _build.LIB
