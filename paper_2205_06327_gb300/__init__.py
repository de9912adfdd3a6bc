"""GB300-native multislice ptychography loss/gradient (arxiv 2205.06327 hot path).

Submodules load lazily: ``synth`` (seeded inputs) needs only numpy; ``api``
and ``autograd`` load the CUDA library ``libptycho.so`` and fail loudly if it
is missing.
"""
__all__ = ["synth", "api", "autograd"]
