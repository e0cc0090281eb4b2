"""Coherent power gain of the final beams in two-stage beamforming, relative to
single-stage beamforming, from the FP64 oracle (Sec. 4, network paragraph: the
effect of the two stages on the final beams).

For each final beam b, a unit plane wave from its own direction is formed into
8 preliminary beams (compact station groups, all toward the pointing centre)
and then into beam b at the group centres; the gain is |beam|^2 / S^2 (1 for a
single stage).  Geometry: the 48 stations and 50 hexagonal beams of the
48 x 488 x 50 workload; frequencies: the lowest, central and highest of its
subbands.  Writes two_stage_gain.json beside this script.

    python tests/golden/two_stage_gain.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402


def gains(groups: int = 8):
    w = synth.PRECISION
    enu, dirs, _ = synth.make_geometry(w)
    grp = synth.station_groups(enu, groups)
    s0 = synth.pointing_enu()
    kk = np.array([0, w.subbands // 2, w.subbands - 1])
    nu = O.sky_frequencies(w.first_bin, w.subbands)[kk]
    cen = O.group_centres(enu, grp, groups)
    w1 = O.prebeam_weights(nu, enu, grp, np.tile(s0, (groups, 1)))
    out = np.zeros((len(kk), len(dirs)))
    for b, sb in enumerate(dirs):
        tau = enu @ sb / O.C_LIGHT
        x = np.exp(2j * np.pi * nu[:, None] * tau[None, :])[None, :, None, :]   # [1, K, 1, S]
        pb = O.prebeam(x, w1)
        beam = O.beamform(pb, O.geometric_weights(nu, cen, sb[None]), np.ones((len(kk), 1)))
        out[:, b] = np.abs(beam[0, 0, 0, :, 0]) ** 2 / enu.shape[0] ** 2
    offs = np.degrees(np.arccos(np.clip(dirs @ s0, -1, 1)))
    return nu, offs, out, np.bincount(grp).tolist()


def main():
    nu, offs, g, sizes = gains()
    res = {"source": "tests/golden/two_stage_gain.py (FP64 oracle)", "groups": 8,
           "group_sizes": sizes, "frequencies_mhz": (nu / 1e6).round(4).tolist(),
           "beam_offset_deg": offs.round(4).tolist(),
           "power_gain": g.round(5).tolist(),
           "summary": {f"{f / 1e6:.2f} MHz": {"min": float(r.min()), "median": float(np.median(r)),
                                              "max": float(r.max())} for f, r in zip(nu, g)}}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "two_stage_gain.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res["summary"], indent=1))


if __name__ == "__main__":
    main()
