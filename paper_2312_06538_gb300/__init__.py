"""Coherent Ray-Space Hierarchy (arXiv 2312.06538) on NVIDIA GB300.

The path (ray hashing and sorting, sphere-cone hierarchy build, culling
traversal, closest-hit tests) runs in libcrsh.so, a C-ABI library of
hand-written sm_103a CUDA kernels (include/crsh.h).  `crsh` binds it with
ctypes; `pipeline` holds device buffers in torch tensors and issues the calls.
"""
import importlib

from . import crsh  # noqa: F401

__all__ = ["crsh", "pipeline"]


def __getattr__(name):
    if name == "pipeline":
        return importlib.import_module(".pipeline", __name__)
    raise AttributeError(name)
