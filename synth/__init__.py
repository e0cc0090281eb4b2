"""Seeded synthetic station data for the lunar nanosecond-pulse pipeline.

This package only makes inputs: station geometry, beam directions, integer
Gaussian noise in the subband domain and dispersed broadband pulses passed
through a forward polyphase filter bank (the station's analysis side, which is
not part of the pipeline).  It holds none of the pipeline's arithmetic (no
beamforming, no de-dispersion, no synthesis, no trigger) and imports neither
the oracle nor the GPU package; both of those import it.
"""

from .stations import *  # noqa: F401,F403
