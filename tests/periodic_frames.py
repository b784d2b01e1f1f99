"""Search inputs whose tables are known by construction: frames that
tile one pattern, so that every filter block's tables are those of a block
of a small frame the oracle can search (used by the GPU parity tests and
pinned against the oracle on small frames)."""
import numpy as np


def periodic_search_case(ref, sizes, bd, seed, coded=False):
    """Frames that tile one 128x128 luma pattern (64x64 chroma), every frame
    an even number of filter blocks high and wide.  A filter block's table
    entries depend only on its pixels and a 2-pixel halo (section 5 on
    eq. 7-12), so each block of such a frame has the tables of the block of
    the same class in a 4x4-block tile of the pattern: class 0 on the first
    row (column), 3 on the last, 1 and 2 on odd and even rows in between.
    The oracle computes the 16 blocks of that 256x256 frame; the full
    tables are gathered from them by class and the oracle selects the
    presets on them.  With `coded`, the 128-combination search (section 5
    with section 4's skip semantics) over a coded-residual map that tiles a
    16x16 pattern of 8x8 flags whose first 8x8 quadrant is uncoded (those
    filter blocks skipped); a block's skip flag and tables follow its class
    the same way."""
    from paper_1602_05975_gb300 import synth
    small = synth.make_frame(256, 256, bd, 32, seed=seed)
    pat = [p[:128, :128] for p in small.rec[:1]] + [p[:64, :64] for p in small.rec[1:]]
    pat_s = [p[:128, :128] for p in small.src[:1]] + [p[:64, :64] for p in small.src[1:]]
    tile = lambda ps, ry, rx: tuple(np.ascontiguousarray(np.tile(p, (ry, rx))) for p in ps)
    damping, lam = 5, 1   # a small lambda: N = 8 and ids of every class
    if coded:
        rng = np.random.default_rng(seed)
        cpat = (rng.random((16, 16)) < 0.6).astype(np.uint8)
        cpat[:8, :8] = 0
        dl_s, dc_s, sk_s = ref.distortion_coded(tile(pat, 2, 2), tile(pat_s, 2, 2), bd, damping,
                                                np.tile(cpat, (2, 2)))
    else:
        dl_s, dc_s = ref.distortion(tile(pat, 2, 2), tile(pat_s, 2, 2), bd, damping)
    cases = []
    for w, h in sizes:
        rows, cols = h // 64, w // 64
        assert rows % 2 == 0 and cols % 2 == 0
        cls = lambda i, n: 0 if i == 0 else 3 if i == n - 1 else 1 if i % 2 else 2
        idx = np.array([cls(by, rows) * 4 + cls(bx, cols) for by in range(rows) for bx in range(cols)])
        dl, dc = dl_s[idx], dc_s[idx]
        case = dict(rec=tile(pat, h // 128, w // 128), src=tile(pat_s, h // 128, w // 128),
                    dl=dl, dc=dc, damping=damping, lam=lam)
        if coded:
            case["coded"] = np.ascontiguousarray(np.tile(cpat, (h // 128, w // 128)))
            case["skipped"] = sk_s[idx]
            case["exp"] = ref.select_presets_general(dl, dc, 128, sk_s[idx], lam)
        else:
            case["exp"] = ref.select_presets(dl, dc, lam)
        cases.append(case)
    return cases
