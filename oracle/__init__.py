"""FP64 CPU oracle of the lunar nanosecond-pulse hot path (arXiv:1612.06592).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously correct
statement of what the GPU path computes: beamforming toward the Moon (Sec. 3,
"Computing Requirements", first paragraph), ionospheric de-dispersion by a
STEC-dependent phase in the frequency domain (Sec. 3, third paragraph),
inversion of the polyphase filter bank back to 5 ns samples (Sec. 2 and Sec. 3,
second paragraph) and the amplitude trigger (Sec. 2, Fig. 1).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` (plus its ``--impl reference`` arm) may import it.  The product
package never imports it, and this package never imports the product package:
the two share no code.  Everything is numpy float64 / complex128; the FFT, the
Bessel function and the filter are written out here, not taken from a library.
"""

from .lofar import *  # noqa: F401,F403
