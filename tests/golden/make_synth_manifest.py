"""Writes tests/golden/synth_manifest.json: the SHA-256 of the synthetic
frames the benchmark and the tests use (a few frames of each workload), from
the seeded generator paper_1602_05975_gb300/synth.py.

    python tests/golden/make_synth_manifest.py

The digests depend on the generator's floating-point DCT round trip; they
were written on an x86_64 host (numpy float64), and tests/test_synth_manifest.py
checks them there.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_1602_05975_gb300 import synth  # noqa: E402

# (what, width, height, bit depth, chroma format, quantiser (None: drawn), seed)
ENTRIES = [
    ("352x288 8-bit 4:2:0, the correctness frame", 352, 288, 8, 420, 32, 0),
    ("1920x1080 8-bit 4:2:0, filter workload frame 0", 1920, 1080, 8, 420, None, 1000),
    ("3840x2160 10-bit 4:2:0, filter workload frame 0", 3840, 2160, 10, 420, None, 2000),
    ("3840x2160 10-bit 4:2:0, filter workload frame 7", 3840, 2160, 10, 420, None, 2007),
    ("640x360 8-bit 4:2:0, search workload frame 0", 640, 360, 8, 420, None, 3000),
    ("1280x720 8-bit 4:2:0, search workload frame 1", 1280, 720, 8, 420, None, 3001),
    ("1920x1080 8-bit 4:4:4, format workload frame 0", 1920, 1080, 8, 444, None, 5000),
    ("3840x2160 12-bit 4:2:0, format workload frame 0", 3840, 2160, 12, 420, None, 6000),
]


def manifest():
    out = []
    for what, w, h, bd, fmt, q, seed in ENTRIES:
        f = synth.make_frame(w, h, bd, q, seed, fmt)
        out.append(dict(what=what, width=w, height=h, bitdepth=bd, chroma=fmt, q=q, seed=seed,
                        drawn_q=int(f.q), sha256=synth.frame_digest(f)))
    return out


if __name__ == "__main__":
    path = os.path.join(HERE, "synth_manifest.json")
    with open(path, "w") as fh:
        json.dump(manifest(), fh, indent=1)
        fh.write("\n")
    print(path)
