"""Writes the oracle-derived golden fixtures in this folder.

Calls only ``oracle/`` and the ``synth`` input generators (never the CUDA
library).  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import swim  # noqa: E402


def noise_pair_64():
    ref, mov = synth.noise_pair(64, (-3, 5))
    lv = swim.Level(64, 0.65, swim.APOD_HANN, 1.0, 3.0)
    res = swim.match_pair(mov, ref, lv)
    return {
        "source": "64x64 worked example: blurred seed-0 white noise (sigma 1.5 px), moving = "
                  "circular shift by (dy, dx) = (-3, +5) plus N(0, 0.1) noise; Hann taper, "
                  "whitening exponent 0.65, SNR exclusion radius 3 px.  Written by the FP64 "
                  "oracle (tests/golden/make_golden.py).",
        "level": {"n": 64, "whiten_exponent": 0.65, "apod": "hann", "snr_exclusion_radius": 3.0},
        "result": res,
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "noise_pair_64.json"), "w") as f:
        json.dump(noise_pair_64(), f, indent=2)
    print("wrote noise_pair_64.json")
