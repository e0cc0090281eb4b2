"""GB300-native hot path of the LOFAR lunar nanosecond-pulse pipeline.

arXiv:1612.06592: tied-array beamforming toward the Moon, ionospheric
de-dispersion by a STEC phase, inverse polyphase filter bank back to 5 ns
samples, envelope trigger.  The work is done by hand-written CUDA kernels for
sm_103a behind the C ABI of include/lp.h (library ``_build/liblp.so``); the
Python module :mod:`paper_1612_06592_gb300.lp` is a ctypes binding with the
same entry-point names.  Build with :func:`build`.
"""

from .build import build, LIB  # noqa: F401
