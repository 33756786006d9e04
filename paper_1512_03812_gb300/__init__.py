"""GB300 (sm_103a) implementation of the HMC molecular-dynamics hot path of
the two-flavour Wilson-fermion Schwinger model (arXiv:1512.03812).

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/schwinger.h``); ``binding`` wraps it for torch tensors and
``autograd`` exposes the action S(U) as a torch.autograd.Function.
Importing this package does not load the library; the first call does.
"""
from .binding import (CG, MD, Lattice, NotConverged, SchwingerError, LAMBDA_2MN,  # noqa: F401
                      launch_count, load, library_path)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the CUDA library in-tree for sm_103a."""
    from . import _build
    return _build.build(force=force, verbose=verbose)
