"""Kernel-level entry points of the C-ABI (bound lazily by ``load``)."""
from __future__ import annotations


def bind(lib):
    """Declare argument types of the kernel-level entry points present in lib."""
    return lib
