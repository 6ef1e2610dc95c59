"""Writes tests/golden/fx_tiny.json: the FP64 oracle's visibilities for one
tiny seeded block, stored so that later changes to the oracle (or to the
seeded generator) show up as a failed comparison. Calls only oracle/ and
synth/. Run from the repository root:  python tests/golden/make_golden.py"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

# 3 stations x 2 pols, 1 subband at 150 MHz, 16 channels, 4 taps, 6 spectra,
# complex int16 noise (sigma 100) plus one tone on channel 5 with delays
CASE = dict(seed=7, fmt=synth.CI16, SB=1, N=3, C=16, T=4, S=6, sigma=100.0,
            tone_channel=5, tone_amp=60.0, delays=[1.5e-6, -2.0e-6, 0.25e-6])


def compute(case=CASE):
    tau = np.array(case["delays"])
    tone = synth.Tone(amp=case["tone_amp"], channel=case["tone_channel"], delays=tau)
    blk = synth.make_block(case["seed"], case["fmt"], case["SB"], case["N"], case["C"], case["S"],
                           n_taps=case["T"], sigma=case["sigma"], tones=[tone])
    vis = oracle.fx(blk.fmt, blk.raw, case["T"], case["C"], case["S"], blk.taps, synth.SAMPLE_RATE_HZ,
                    blk.centres, tau, tau)
    return blk, tau, vis


if __name__ == "__main__":
    _, _, vis = compute()
    out = {"doc": "oracle.fx visibilities [SB][C][B][4][re, im] for CASE; written by make_golden.py",
           "case": CASE, "vis": np.round(vis, 9).tolist()}
    with open(os.path.join(HERE, "fx_tiny.json"), "w") as f:
        json.dump(out, f, indent=0)
