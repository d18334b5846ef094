"""Seeded synthetic surveillance video for the CoG workloads.

This package holds only input generation (counter-based hashing, a smooth
background texture, camera noise, moving objects, dynamic background): none
of the background-subtraction method's arithmetic.  Both the FP64 oracle and
the CUDA path consume its frames.  ``scene.Scene`` renders on the CPU with
numpy; ``gpu.render_frames`` is the bit-identical CUDA twin used when a
workload is too large to render on the host.
"""
from .scene import Scene, sm64, workload  # noqa: F401
