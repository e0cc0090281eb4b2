"""Peak of a dispersed pulse recovered by each de-dispersion chain, relative to
the same pulse undispersed through the same inversion, from the FP64 oracle
(Sec. 3, second and third paragraphs).

Chains: (1) the per-subband STEC phase, then the FIR synthesis (the realtime
path); (2) the same plus the channel-domain fine filter; (3) the FIR synthesis
of the undispersed-phase subbands, then full-rate de-dispersion of the 200 MHz
series; (4) the LSMR inversion, then full-rate de-dispersion (the paper's
order).  One pulse (synthetic, through the station-side PPF) at the true STEC,
for two bands.  Writes dedispersion_chains.json beside this script.

    python tests/golden/dedispersion_chains.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import synth  # noqa: E402

CASES = [(25.0, 60, 192), (40.0, 12, 488)]       # (STEC [TECU], first bin, subbands)


def _pulse_frames(tec, first_bin, K, F):
    """Subband frames of one broadband pulse (F frames, pulse at frame 40)."""
    w = synth.Workload("chain", 1, 1, K, first_bin, 1, (tec,), F, "int16", 1.0)
    h = synth.analysis_filter()
    n0 = 40 * O.M + 100
    m_lo, m_hi, xs = synth.pulse_subbands(synth.Pulse(n0, 5.0e4, tec, 0.0, 0), w, h, 0)
    frames = np.zeros((F, K), dtype=complex)
    frames[m_lo:m_hi] = xs
    return frames


def chains(tec, first_bin, K):
    F = 256 + 16
    disp, ref = _pulse_frames(tec, first_bin, K, F), _pulse_frames(0.0, first_bin, K, F)
    nu = O.sky_frequencies(first_bin, K)
    nu_ref = 0.5 * (nu[0] + nu[-1])
    g, h = O.synthesis_filter(), O.prototype_filter()
    fir = lambda fr: O.ippf(fr[1:], first_bin, g).reshape(-1)        # 15 history frames
    peak = lambda u: float(np.abs(u).max())
    d = O.dedispersion_weights(nu, [tec], nu_ref)[:, 0]
    r = O.fine_dedispersion_taps(nu, [tec], nu_ref)[:, 0]
    fine = np.concatenate([np.zeros((O.FINE_TAPS - 1, K)), disp * d[None]])
    out = {
        "subband phase + FIR": peak(fir(disp * d[None])) / peak(fir(ref)),
        "subband phase + fine filter + FIR":
            peak(fir(O.fine_dedisperse(fine, r))) / peak(fir(ref)),
        "FIR + full-rate": peak(O.fullrate_dedisperse(fir(disp), tec, nu_ref)) / peak(fir(ref)),
        "LSMR + full-rate": peak(O.fullrate_dedisperse(O.lsmr_invert(disp, first_bin, h)
                                                      .reshape(-1), tec, nu_ref))
        / peak(O.lsmr_invert(ref, first_bin, h).reshape(-1)),
    }
    return {k: round(v, 4) for k, v in out.items()}


def main():
    res = {"source": "tests/golden/dedispersion_chains.py (FP64 oracle)",
           "cases": [{"tec_tecu": t, "first_bin": b, "subbands": k, "peak_ratio": chains(t, b, k)}
                     for t, b, k in CASES]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dedispersion_chains.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res["cases"], indent=1))


if __name__ == "__main__":
    main()
