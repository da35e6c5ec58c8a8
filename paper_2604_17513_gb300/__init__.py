"""GB300-native batched deformable + frictional-contact time step (FLASH,
arxiv 2604.17513): CUDA kernels behind a C ABI (include/flash.h), this thin
binding, and seeded synthetic scenes."""
from . import scenes  # noqa: F401

__all__ = ["scenes", "flash", "build"]
