"""GB300-native coherent-receiver DSP chain (arXiv 2108.07004, Sec. 2).

Importing the package is cheap: the CUDA library is loaded by
``paper_2108_07004_gb300.rx`` on first use, and fails loudly when the
compiled library is missing.
"""

__all__ = ["synth", "formats", "rx"]
