"""GB300-native implicit grey flux-limited-diffusion radiation step.

Importing the package loads nothing; ``paper_1306_0645_gb300.fld`` binds the
CUDA library (libfld.so) and ``paper_1306_0645_gb300.synth`` builds inputs.
"""
__all__ = ["fld", "synth", "serving"]
