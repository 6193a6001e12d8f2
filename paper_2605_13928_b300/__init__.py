"""Exact t-SNE on B300 (sm_103a): kNN, perplexity calibration, exact KL gradient.

The compute path is the CUDA library ``libtsne.so`` built from ``csrc/``; this
package only marshals arguments to its C ABI.  Importing the package does not
load the library; the first call that needs it does, and raises if it is missing.
"""
from . import synth  # noqa: F401

__all__ = ["synth"]
