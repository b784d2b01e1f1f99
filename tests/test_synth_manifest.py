"""The synthetic inputs are the recorded ones: every frame listed in
tests/golden/synth_manifest.json (written by make_synth_manifest.py from the
seeded generator) regenerates to the same SHA-256.  The generator holds no
step of the method; a change of its recipe (or of numpy's seeded streams)
shows up here before it silently changes what the oracle and the GPU are
compared on."""
import json
import os
import platform

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(platform.machine() not in ("x86_64", "AMD64"),
                    reason="digests recorded on x86_64 (the floating-point DCT round trip)")
def test_synthetic_frames_match_manifest():
    from paper_1602_05975_gb300 import synth
    entries = json.load(open(os.path.join(HERE, "golden", "synth_manifest.json")))
    assert len(entries) >= 8
    for e in entries:
        f = synth.make_frame(e["width"], e["height"], e["bitdepth"], e["q"], e["seed"], e["chroma"])
        assert int(f.q) == e["drawn_q"], e["what"]
        assert synth.frame_digest(f) == e["sha256"], e["what"]


def test_digest_sees_every_part():
    """The digest changes with any sample of either plane set, the
    parameters or the quantiser."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(64, 64, 8, 32, seed=1)
    d0 = synth.frame_digest(f)
    for part in ("src", "rec"):
        planes = [p.copy() for p in getattr(f, part)]
        planes[2][3, 4] ^= 1
        g = synth.Frame(f.width, f.height, f.bitdepth, f.q,
                        *( (tuple(planes), f.rec) if part == "src" else (f.src, tuple(planes)) ),
                        f.params)
        assert synth.frame_digest(g) != d0
    p = f.params.copy()
    p[0, 0, 4] ^= 1
    assert synth.frame_digest(synth.Frame(f.width, f.height, 8, f.q, f.src, f.rec, p)) != d0
    assert synth.frame_digest(synth.Frame(f.width, f.height, 8, 16, f.src, f.rec, f.params)) != d0
