"""B300-native recursive clutter-whitening preprocessor (Kennedy, arXiv:1408.3526).

Submodules:
  stream  -- WhitenStream, the per-stream front end over the C ABI (libwhiten.so)
  scenes  -- seeded synthetic infrared scenes (input generation only)
  build   -- nvcc build of libwhiten.so for sm_103a

Importing the package loads nothing; ``WhitenStream`` loads the CUDA library
on first use and raises if it is missing.
"""

__all__ = ["WhitenStream"]


def __getattr__(name):
    if name == "WhitenStream":
        from .stream import WhitenStream
        return WhitenStream
    raise AttributeError(name)
