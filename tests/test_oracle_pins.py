"""Pins of the CPU oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: numbers the
paper prints (tests/golden/paper_values.json), closed forms, exact rational
arithmetic, brute force, geometry, or a library routine.  No GPU.
"""
import decimal
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "paper_values.json")))


# --------------------------------------------------------------------------
# Section 2: line geometry (Fig. 1 reading R1)
# --------------------------------------------------------------------------
def _lines(ref, d):
    lines = {}
    for i in range(8):
        for j in range(8):
            lines.setdefault(ref.line_number(d, i, j), []).append((i, j))
    return lines


def test_line_cardinalities_printed(ref):
    g = GOLDEN["line_cardinality"]
    lines = _lines(ref, 1)
    assert len(lines[0]) == g["N_1_0"]
    assert len(lines[4]) == g["N_1_4"]


def test_lines_partition_block(ref):
    g = GOLDEN["cardinality_range"]
    for d in range(8):
        lines = _lines(ref, d)
        assert sorted(lines) == list(range(len(lines)))  # contiguous numbering
        assert sum(len(v) for v in lines.values()) == 64
        for v in lines.values():
            assert g["min"] <= len(v) <= g["max"]
            assert g["lcm"] % len(v) == 0


def test_operation_counts_printed(ref):
    """90 line sums; 34 multiplies (one per distinct cardinality of a
    direction); 82 additions (lines - 1 per direction)."""
    g = GOLDEN["search_op_counts"]
    nlines = [len(_lines(ref, d)) for d in range(8)]
    assert sum(nlines) == g["line_sums"]
    distinct = [len({len(v) for v in _lines(ref, d).values()}) for d in range(8)]
    assert sum(distinct) == g["multiplies_for_s_d"]
    assert sum(n - 1 for n in nlines) == g["additions_for_s_d"]
    assert 8 - 1 == g["comparisons"]


def _line_angle(pixels):
    """Orientation (degrees, in [0, 180)) of a set of (row, col) points, with
    angles measured counter-clockwise from the +column axis, row up."""
    pts = np.array([(j, -i) for (i, j) in pixels], float)
    pts -= pts.mean(0)
    w, v = np.linalg.eigh(pts.T @ pts)
    vx, vy = v[:, -1]
    return math.degrees(math.atan2(vy, vx)) % 180.0


def test_direction_angles(ref):
    """d = 0 is the 45-degree diagonal (Fig. 2 caption: the 45-degree
    direction), directions turn by about 22.5 degrees per step, and d+4 is
    perpendicular to d (the contrast of Algorithm 1 compares them)."""
    ang = []
    for d in range(8):
        longest = max(_lines(ref, d).values(), key=len)
        ang.append(_line_angle(longest))
    for d in range(8):
        expect = (45.0 - 22.5 * d) % 180.0
        diff = min(abs(ang[d] - expect), 180 - abs(ang[d] - expect))
        assert diff < 5.0, (d, ang[d], expect)
        perp = abs(ang[d] - ang[(d + 4) % 8]) % 180
        assert abs(perp - 90.0) < 1e-6 or abs(perp - 90.0) < 5.0


def test_direction_costs_dihedral_symmetry(ref):
    """The eight directions are a symmetric fan (Fig. 1: d = 0 at 45
    degrees, 22.5-degree steps): transposing a block maps the lines of d
    onto those of (8 - d) mod 8, mirroring its columns onto those of
    (4 - d) mod 8, and a half turn maps every direction's lines onto
    themselves, so the costs s_d permute exactly (a line formula wrong for
    one direction, or a floor where its mirror image takes a ceiling, breaks
    this)."""
    rng = np.random.default_rng(12)
    for _ in range(200):
        x = rng.integers(-128, 128, (8, 8))
        s = ref.direction_costs(x)
        st = ref.direction_costs(x.T)
        sf = ref.direction_costs(x[:, ::-1])
        sr = ref.direction_costs(x[::-1, ::-1])
        for d in range(8):
            assert st[(8 - d) % 8] == s[d]
            assert sf[(4 - d) % 8] == s[d]
            assert sr[d] == s[d]


# --------------------------------------------------------------------------
# Section 2: costs, eq. 1-5, Algorithm 1
# --------------------------------------------------------------------------
def _e2_direct(ref, x, d):
    """E_d^2 straight from eq. 1-2 with exact rational line means."""
    lines = _lines(ref, d)
    e2 = Fraction(0)
    for pix in lines.values():
        vals = [int(x[i, j]) for (i, j) in pix]
        mu = Fraction(sum(vals), len(vals))
        e2 += sum((Fraction(v) - mu) ** 2 for v in vals)
    return e2


def test_e2_identity_exact(ref):
    """Eq. 3: 840*E_d^2 = 840*sum x^2 - 840*s_d, in exact rationals."""
    rng = np.random.default_rng(1)
    blocks = [rng.integers(-128, 128, (8, 8)) for _ in range(150)]
    blocks += [np.full((8, 8), -128), np.full((8, 8), 127),
               np.where(np.indices((8, 8)).sum(0) % 2 == 0, 127, -128)]
    for x in blocks:
        s = ref.direction_costs(x)
        sumsq = int((x.astype(np.int64) ** 2).sum())
        for d in range(8):
            assert Fraction(840) * _e2_direct(ref, x, d) == 840 * sumsq - int(s[d])


def test_argmin_e_equals_argmax_s(ref):
    rng = np.random.default_rng(2)
    for _ in range(200):
        x = rng.integers(-128, 128, (8, 8))
        s = ref.direction_costs(x)
        e = [_e2_direct(ref, x, d) for d in range(8)]
        assert e.index(min(e)) == int(np.argmax(s))  # both first on ties


def test_perfectly_directional_block(ref):
    """A block constant along the lines of d* is found as d* with E = 0
    (section 2's definition of a perfectly directional block)."""
    rng = np.random.default_rng(3)
    for dstar in range(8):
        for _ in range(20):
            lines = _lines(ref, dstar)
            vals = rng.choice(np.arange(-128, 128), size=len(lines), replace=False)
            x = np.zeros((8, 8), np.int64)
            for k, pix in lines.items():
                for (i, j) in pix:
                    x[i, j] = vals[k]
            s = ref.direction_costs(x)
            assert _e2_direct(ref, x, dstar) == 0
            assert s[dstar] == 840 * int((x ** 2).sum())
            raw = (x + 128).astype(np.uint16)
            d, v = ref.find_dir_block(raw, 8)
            assert d == dstar
            assert v >= 0


def test_constant_block_ties_to_zero(ref):
    for c in (0, 77, 128, 255):
        d, v = ref.find_dir_block(np.full((8, 8), c, np.uint16), 8)
        assert d == 0 and v == 0  # strict '>' in Algorithm 1


def test_45_degree_line_block(ref):
    """Fig. 2: a block containing a 45-degree line selects the 45-degree
    direction (d = 0 under the reading of Fig. 1)."""
    for off in range(-3, 4):
        x = np.full((8, 8), 40, np.uint16)
        for i in range(8):
            j = 7 - i + off
            if 0 <= j < 8:
                x[i, j] = 200
        d, _ = ref.find_dir_block(x, 8)
        assert d == 0


def test_int32_claim(ref):
    """Section 2: with centred 8-bit pixels, 840*s_d fits a signed 32-bit
    integer.  Cauchy-Schwarz gives s_d <= 840*sum x^2 <= 840*64*128^2."""
    g = GOLDEN["int32_claim"]
    extremes = [np.full((8, 8), g["centred_min"]), np.full((8, 8), g["centred_max"])]
    rng = np.random.default_rng(4)
    extremes += [rng.choice([g["centred_min"], g["centred_max"]], (8, 8)) for _ in range(200)]
    for x in extremes:
        s = ref.direction_costs(x)
        assert s.max() < g["bound_exclusive"]
        assert s.max() <= 840 * int((np.asarray(x, np.int64) ** 2).sum())


def test_high_bitdepth_search_downscales(ref):
    """Section 2: higher bit depths are searched at 8 bits."""
    rng = np.random.default_rng(5)
    for _ in range(100):
        x8 = rng.integers(0, 256, (8, 8)).astype(np.uint16)
        low = rng.integers(0, 4, (8, 8)).astype(np.uint16)
        x10 = (x8 << 2) | low
        assert ref.find_dir_block(x8, 8) == ref.find_dir_block(x10, 10)
        x12 = (x8 << 4) | rng.integers(0, 16, (8, 8)).astype(np.uint16)
        assert ref.find_dir_block(x8, 8) == ref.find_dir_block(x12, 12)


def test_contrast_nonnegative_and_definition(ref):
    rng = np.random.default_rng(6)
    for _ in range(300):
        raw = rng.integers(0, 256, (8, 8)).astype(np.uint16)
        d, v = ref.find_dir_block(raw, 8)
        s = ref.direction_costs(raw.astype(np.int64) - 128)
        assert v >= 0
        assert v == s[d] - s[(d + 4) % 8]
        assert s[d] == s.max() and d == int(np.argmax(s))


# --------------------------------------------------------------------------
# Eq. 7: the constraint function
# --------------------------------------------------------------------------
def test_constrain_properties_exhaustive(ref):
    """Anti-symmetry (stated after eq. 7), f(0) = 0, sign and magnitude
    bounds, zero strength, and the damping-controlled zero point: with
    S*2^(D - floor log2 S) in [2^D, 2^(D+1)), f(d) > 0 for 0 < d < 2^D and
    f(d) = 0 for d >= 2^(D+1)."""
    for S in range(0, 80):
        lo = int(math.floor(math.log2(S))) if S > 0 else 0
        for D in range(max(lo, 0), 11):
            if D - lo > 10:
                continue
            for d in list(range(-1100, 1101, 7)) + list(range(-40, 41)):
                f = ref.constrain(d, S, D)
                assert ref.constrain(-d, S, D) == -f
                if S == 0 or d == 0:
                    assert f == 0
                    continue
                assert f == 0 or np.sign(f) == np.sign(d)
                assert abs(f) <= min(abs(d), S)
                if abs(d) >= 2 ** (D + 1):
                    assert f == 0
                if 0 < abs(d) < 2 ** D:
                    assert f != 0


def test_constrain_small_differences_linear(ref):
    """'For small differences, f(d, S, D) = d': f(d) = d for |d| up to a
    threshold of at least 1 whenever S >= 1 (over the dampings the paper
    allows, D >= 2), and f is unimodal in d >= 0 (rises as d, then falls
    to 0)."""
    for S in range(1, 80):
        lo = int(math.floor(math.log2(S)))
        for D in range(max(lo, 2), lo + 8):
            vals = [ref.constrain(d, S, D) for d in range(0, 2 ** (D + 1) + 2)]
            assert vals[1] == 1
            k = 0
            while k + 1 < len(vals) and vals[k + 1] == k + 1:
                k += 1
            tail = vals[k:]
            assert all(a >= b for a, b in zip(tail, tail[1:]))
            assert max(vals) <= S


def test_constrain_damping_monotone(ref):
    """Fig. 2 (bottom): larger damping moves the zero point out; |f| never
    shrinks as D grows."""
    for S in range(1, 64):
        lo = int(math.floor(math.log2(S)))
        for D in range(lo, lo + 6):
            for d in range(0, 600, 3):
                assert ref.constrain(d, S, D + 1) >= ref.constrain(d, S, D)


def test_constrain_large_damping_reaches_strength(ref):
    """Fig. 2 (top): the strength caps the correction; with damping large
    enough the cap S is reached."""
    for S in range(1, 80):
        assert max(ref.constrain(d, S, 14) for d in range(0, 200)) == S


# --------------------------------------------------------------------------
# Eq. 8 rounding, eq. 13 adjustment, section 3.2 parameters
# --------------------------------------------------------------------------
def test_round16_ties_away_from_zero(ref):
    table = {8: 1, -8: -1, 24: 2, -24: -2, 7: 0, -7: 0, 9: 1, -9: -1, 0: 0,
             23: 1, -23: -1, 25: 2}
    for s, r in table.items():
        assert ref.round16(s) == r
    ctx = decimal.Context(rounding=decimal.ROUND_HALF_UP)
    for s in range(-4000, 4001):
        expect = int(ctx.quantize(decimal.Decimal(s) / 16, decimal.Decimal(1)))
        assert ref.round16(s) == expect


def test_adjust_strength(ref):
    g = GOLDEN["contrast_thresholds"]
    for S in range(0, 16):
        prev = -1
        for v in [0, 1, g["zero_below"] - 1, g["zero_below"], 5000, 65535, 65536,
                  131071, 131072, 10 ** 6, 10 ** 7, 2 ** 28, 2 ** 30, 2 ** 31 - 1]:
            a = ref.adjust_strength(S, v)
            if v < g["zero_below"]:
                assert a == 0
            assert 0 <= a <= S
            assert a >= prev
            prev = a
        # saturation: floor(log2(v/2^16)) >= 12 gives the factor 16/16
        assert ref.adjust_strength(S, g["log_unit"] * 2 ** g["max_log"]) == S
        assert ref.adjust_strength(S, 2 ** 31 - 1) == S
    for v in range(1024, 2 ** 20, 997):
        assert [ref.adjust_strength(S, v) for S in range(16)] == \
            sorted(ref.adjust_strength(S, v) for S in range(16))


def test_adjust_strength_rounds_to_nearest(ref):
    """Eq. 13 prints floor((S (4 + i) + 8) / 16): the strength scaled by
    (4 + i) / 16, rounded to the nearest integer with halves up, where
    i = min(floor(log2 floor(v / 2^16)), 12) (reading R3: 0 below 2^16).
    Checked for every i and S against exact fractions."""
    from fractions import Fraction
    for i in range(13):
        v = 1024 if i == 0 else (1 << 16) << i          # floor(log2(v / 2^16)) = i
        for S in range(16):
            exact = Fraction(S * (4 + i), 16)
            want = int(exact + Fraction(1, 2))          # floor(x + 1/2): nearest, halves up
            assert ref.adjust_strength(S, v) == want, (S, i)


def test_chroma_damping_example(ref):
    g = GOLDEN["chroma_damping_example"]
    e = ref.block_params(g["chroma_primary"], 0, g["luma_damping"], True, 8)
    assert e.damping == g["chroma_damping"]
    e = ref.block_params(2, 0, g["luma_damping"], True, 8)
    assert e.damping == g["luma_damping"] - 1
    for D in range(3, 7):
        for S in range(16):
            for chroma in (False, True):
                e = ref.block_params(S, 0, D, chroma, 8, 2 ** 31 - 1)
                if e.pri:
                    assert e.damping >= int(math.floor(math.log2(e.pri)))


def test_twelve_bit_example(ref):
    g = GOLDEN["twelve_bit_example"]
    vals = [ref.block_params(S, 0, 3, True, 12).pri for S in range(16)]
    assert vals == g["primary_values"]
    damp = sorted({ref.block_params(1, 0, D, False, 12, 2 ** 31 - 1).damping
                   for D in range(3, 7)})
    assert [damp[0], damp[-1]] == g["damping_range"]
    # taps keep alternating after scaling: parity follows the 8-bit value
    for S in range(16):
        assert ref.block_params(S, 0, 3, True, 12).parity == S % 2


def test_bitdepth_scaling(ref):
    """Section 3.2: at bit depth 8+k strengths are scaled by 2^k and D is
    offset by k.  D - floor(log2 S) is then unchanged, so the zero point of
    f scales by exactly 2^k and f itself by 2^k up to the finer flooring:
    |f(2^k d, 2^k S, D + k) - 2^k f(d, S, D)| < 2^k."""
    for k in (2, 4):
        for S in range(1, 20):
            lo = int(math.floor(math.log2(S)))
            for D in range(max(lo, 2), lo + 5):
                zero = next(d for d in range(1, 4096) if ref.constrain(d, S, D) == 0)
                zero_k = next(d for d in range(1, 1 << 16)
                              if ref.constrain(d, S << k, D + k) == 0)
                assert zero_k == zero << k
                for d in range(-300, 301, 5):
                    assert abs(ref.constrain(d << k, S << k, D + k)
                               - (ref.constrain(d, S, D) << k)) < (1 << k)
    for bd in (10, 12):
        for S in range(1, 16):
            for D in range(3, 7):
                for chroma in (False, True):
                    e8 = ref.block_params(S, 4, D, chroma, 8, 2 ** 31 - 1)
                    eb = ref.block_params(S, 4, D, chroma, bd, 2 ** 31 - 1)
                    assert eb.pri == e8.pri << (bd - 8) and eb.sec == e8.sec << (bd - 8)
                    assert eb.damping - eb.pri.bit_length() == e8.damping - e8.pri.bit_length()


# --------------------------------------------------------------------------
# Eq. 8-12: the filter
# --------------------------------------------------------------------------
def _probe_weights(ref, d, pri, sec):
    """Weight (in sixteenths) that the oracle gives each offset of the 5x5
    neighbourhood, read back through a single tap of height 16 at 12 bits
    (where f(16) = 16 for the probed strengths, so y - x = w)."""
    w = {}
    for dr in range(-2, 3):
        for dc in range(-2, 3):
            if dr == 0 and dc == 0:
                continue
            plane = np.full((9, 9), 2000, np.uint16)
            plane[4 + dr, 4 + dc] = 2016
            e = ref.block_params(pri, sec, 6, False, 12, 2 ** 31 - 1)
            y = ref.filter_sample(plane, 4, 4, d, e)
            if y != 2000:
                w[(dr, dc)] = y - 2000
    return w


def test_tap_geometry_and_weights(ref):
    """Figs. 3-4 (figures missing): 4 primary taps on a line through the
    filtered pixel along d, weights (b near, a far) = (4, 2) for even and
    (3, 3) for odd strengths (caption of Fig. 3), and 8 secondary taps
    that are the primary taps of d +- 2 (the cross 45 degrees off d)."""
    pw = GOLDEN["primary_weights"]
    prim = {}
    for d in range(8):
        even = _probe_weights(ref, d, 14, 0)
        odd = _probe_weights(ref, d, 15, 0)
        assert len(even) == 4 and set(even) == set(odd)
        for (dr, dc), wt in even.items():
            assert (-dr, -dc) in even  # symmetric pairs
            near = max(abs(dr), abs(dc)) == 1
            assert wt == (pw["even"]["b"] if near else pw["even"]["a"])
            assert odd[(dr, dc)] == (pw["odd"]["b"] if near else pw["odd"]["a"])
        # the far taps lie on the centre's line of direction d (Fig. 1)
        for (dr, dc) in even:
            if max(abs(dr), abs(dc)) == 2:
                for i in range(2, 6):
                    for j in range(2, 6):
                        if 0 <= i + dr < 8 and 0 <= j + dc < 8:
                            assert ref.line_number(d, i + dr, j + dc) == ref.line_number(d, i, j)
        # and all four are collinear with the centre
        pts = [(0, 0)] + list(even)
        ang = _line_angle(pts)
        longest = max(_lines(ref, d).values(), key=len)
        diff = abs(ang - _line_angle(longest))
        assert min(diff, 180 - diff) < 10
        prim[d] = set(even)
    for d in range(8):
        secw = _probe_weights(ref, d, 0, 4)
        expect = prim[(d + 2) % 8] | prim[(d + 6) % 8]
        assert set(secw) == expect and len(secw) == 8
        for (dr, dc), wt in secw.items():
            assert wt == (2 if max(abs(dr), abs(dc)) == 1 else 1)


@pytest.mark.parametrize("bd", [8, 10])
def test_filter_frame_dihedral_symmetry(ref, bd):
    """Figs. 3-4 (figures missing) and R8: the taps of each direction are
    those of its mirror images, so filtering a transposed (or mirrored)
    frame with the correspondingly mapped directions, contrasts and
    per-block parameters gives the transposed (mirrored) output, sample for
    sample, luma and 4:2:0 chroma, frame edges included.  A tap offset wrong
    in one direction's table fails it."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(30 + bd)
    h, w = 128, 192
    y, u, v = synth.random_frame_planes(rng, w, h, bd)
    prm = synth.random_params(rng, w, h)
    dirs = rng.integers(0, 8, (h // 8, w // 8)).astype(np.uint8)
    var = rng.integers(0, 1 << 20, (h // 8, w // 8)).astype(np.int32)
    oy, ou, ov = ref.filter_frame(y, u, v, bd, prm, dirs, var)
    # transpose: d -> (8 - d) mod 8
    ty, tu, tv = ref.filter_frame(y.T, u.T, v.T, bd, prm.transpose(1, 0, 2),
                                  ((8 - dirs.astype(int)) % 8).astype(np.uint8).T, var.T)
    assert (ty == oy.T).all() and (tu == ou.T).all() and (tv == ov.T).all()
    # mirrored columns: d -> (4 - d) mod 8
    fy, fu, fv = ref.filter_frame(y[:, ::-1], u[:, ::-1], v[:, ::-1], bd, prm[:, ::-1],
                                  ((4 - dirs.astype(int)) % 8).astype(np.uint8)[:, ::-1],
                                  var[:, ::-1])
    assert (fy == oy[:, ::-1]).all() and (fu == ou[:, ::-1]).all() and (fv == ov[:, ::-1]).all()


def test_zero_strength_identity(ref):
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(7)
    for bd in (8, 10):
        y, u, v = synth.random_frame_planes(rng, 48, 40, bd)
        prm = synth.random_params(rng, 48, 40)
        prm[..., 0:4] = 0
        oy, ou, ov = ref.filter_frame(y, u, v, bd, prm)
        assert (oy == y).all() and (ou == u).all() and (ov == v).all()


def test_constant_frame_fixed_point(ref):
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(8)
    for bd in (8, 10):
        for c in (0, 100, (1 << bd) - 1):
            y = np.full((40, 56), c, np.uint16)
            u = np.full((20, 28), c, np.uint16)
            prm = synth.random_params(rng, 56, 40)
            oy, ou, ov = ref.filter_frame(y, u, u, bd, prm)
            assert (oy == c).all() and (ou == c).all() and (ov == c).all()


def test_constant_along_direction_unchanged(ref):
    """With only primary taps, a plane constant along d (rows, columns,
    diagonals) gives every primary difference 0, so y = x."""
    rng = np.random.default_rng(9)
    ii, jj = np.indices((12, 12))
    along = {0: ii + jj, 2: ii, 4: ii - jj, 6: jj}
    for d, key in along.items():
        vals = rng.integers(0, 256, 40)
        plane = vals[key + 15].astype(np.uint16) if d == 4 else vals[key].astype(np.uint16)
        for pri in (1, 7, 15):
            e = ref.block_params(pri, 0, 4, False, 8, 2 ** 31 - 1)
            for i in range(12):
                for j in range(12):
                    assert ref.filter_sample(plane, i, j, d, e) == plane[i, j]


def test_clip_to_taps(ref):
    """Eq. 9-12: twelve taps one above the pixel raise the raw sum to 24
    sixteenths (round(1.5) = 2) but the clip holds y at x + 1; with one tap
    set active the sum is 12 sixteenths and rounds to 1."""
    plane = np.full((9, 9), 101, np.uint16)
    plane[4, 4] = 100
    for d in range(8):
        e = ref.block_params(15, 4, 6, False, 8, 2 ** 31 - 1)
        assert ref.filter_sample(plane, 4, 4, d, e) == 101
        e = ref.block_params(14, 0, 6, False, 8, 2 ** 31 - 1)
        assert ref.filter_sample(plane, 4, 4, d, e) == 101
        e = ref.block_params(0, 4, 6, False, 8, 2 ** 31 - 1)
        assert ref.filter_sample(plane, 4, 4, d, e) == 101


def test_weights_exceed_unity(ref):
    """Section 3.2: the primary and secondary weights together exceed unity,
    so without the clip a pixel can move by more than any contributing
    neighbour differs from it.  Every tap one step delta above x, except the
    far primary tap of d = 2 (along the row), set so far above that f = 0
    for it while it keeps the clip range open: y moves by more than delta
    (round(22 delta / 16) under the weights read from Figs. 3-4)."""
    for delta in (2, 4):
        plane = np.full((9, 9), 100 + delta, np.uint16)
        plane[4, 4] = 100
        plane[4, 6] = 250
        e = ref.block_params(14, 4, 6, False, 8, 2 ** 31 - 1)
        y = ref.filter_sample(plane, 4, 4, 2, e)
        assert y - 100 > delta
        assert y - 100 == ref.round16(22 * delta)


def test_out_of_frame_taps_are_ignored(ref):
    """Section 3.1: a tap outside the frame is ignored (f = 0, not in the
    clip range).  Ignoring it is the same as an in-frame tap equal to the
    filtered pixel (f(0) = 0 and x is already in the range), so filtering at
    the border equals filtering inside a frame padded with the pixel's own
    value."""
    rng = np.random.default_rng(10)
    plane = rng.integers(0, 256, (16, 16)).astype(np.uint16)
    for d in range(8):
        for pri, sec in ((15, 4), (9, 2), (0, 1)):
            e = ref.block_params(pri, sec, 5, False, 8, 2 ** 31 - 1)
            for (i, j) in [(0, 0), (0, 7), (1, 15), (15, 15), (14, 3), (7, 0), (8, 14)]:
                x = int(plane[i, j])
                padded = np.full((20, 20), x, np.uint16)
                padded[2:18, 2:18] = plane
                assert ref.filter_sample(plane, i, j, d, e) == \
                    ref.filter_sample(padded, i + 2, j + 2, d, e)


def test_output_within_neighbourhood_range(ref):
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(11)
    for bd in (8, 10):
        y, u, v = synth.random_frame_planes(rng, 32, 24, bd)
        prm = synth.random_params(rng, 32, 24)
        oy, _, _ = ref.filter_frame(y, u, v, bd, prm)
        yp = np.pad(y.astype(np.int64), 2, mode="edge")
        for i in range(24):
            for j in range(32):
                nb = yp[i:i + 5, j:j + 5]
                assert nb.min() <= oy[i, j] <= nb.max()


# Readings R8 and R9 typed here from their statement, independently of the
# oracle's tables: the primary taps at distance 1 and 2 along direction d
# (row, column offsets, each used with both signs), primary weights (near,
# far) = (4, 2) for an even and (3, 3) for an odd strength, secondary taps
# the primary taps of d + 2 and d - 2 with weights (2, 1).
_R8_TAPS = {0: ((-1, 1), (-2, 2)), 1: ((0, 1), (-1, 2)), 2: ((0, 1), (0, 2)),
            3: ((0, 1), (1, 2)), 4: ((1, 1), (2, 2)), 5: ((1, 0), (2, 1)),
            6: ((1, 0), (2, 0)), 7: ((1, 0), (2, -1))}


def _reading_weights(d, kind, parity):
    """{(dr, dc): weight} of the primary (kind 0) or secondary (kind 1) taps
    of direction d under readings R8/R9."""
    if kind == 0:
        dirs, (wn, wf) = (d,), ((4, 2) if parity == 0 else (3, 3))
    else:
        dirs, (wn, wf) = ((d + 2) % 8, (d + 6) % 8), (2, 1)
    out = {}
    for dd in dirs:
        (nr, nc), (fr, fc) = _R8_TAPS[dd]
        for sg in (1, -1):
            out[(sg * nr, sg * nc)] = wn
            out[(sg * fr, sg * fc)] = wf
    return out


def _py_filter_frame(ref, y, u, v, bd, prm):
    """An independent frame-level evaluator written from the paper in
    Python: the taps and weights of readings R8/R9 typed above, eq. 7 from
    its text, the block/plane plumbing of sections 2-4 re-derived here (the
    oracle supplies only the directions, pinned separately)."""
    wmap = {}
    for d in range(8):
        wmap[(d, 0, 0)] = _reading_weights(d, 0, 0)
        wmap[(d, 0, 1)] = _reading_weights(d, 0, 1)
        wmap[(d, 1, 0)] = _reading_weights(d, 1, 0)

    def f(diff, S, D):
        if S == 0:
            return 0
        sh = D - (S.bit_length() - 1)
        a = abs(diff)
        m = min(a, max(0, S - a // (1 << sh)))
        return m if diff >= 0 else -m

    def adj(S, v):
        if v < 1024:
            return 0
        q = v >> 16
        i = min(q.bit_length() - 1, 12) if q else 0
        return (S * (4 + i) + 8) >> 4

    h, w = y.shape
    dirs, var = ref.find_dir(y, bd)
    outs = []
    for plane, sub in ((y, 0), (u, 1), (v, 1)):
        ph, pw = plane.shape
        out = np.zeros_like(plane)
        for i in range(ph):
            for j in range(pw):
                by, bx = (i << sub) // 8, (j << sub) // 8
                d = int(dirs[by, bx])
                fb = prm[(i << sub) // 64, (j << sub) // 64]
                if sub == 0:
                    Sp, Ss, D = adj(int(fb[0]), int(var[by, bx])), int(fb[1]), int(fb[4])
                else:
                    Sp, Ss, D = int(fb[2]), int(fb[3]), int(fb[4]) - 1
                if Sp and D < Sp.bit_length() - 1:
                    D = Sp.bit_length() - 1
                par = Sp & 1
                k = bd - 8
                Sp, Ss, D = Sp << k, Ss << k, D + k
                x = int(plane[i, j])
                tot, lo, hi = 0, x, x
                for kind, S in ((0, Sp), (1, Ss)):
                    wm = wmap[(d, 0, par)] if kind == 0 else wmap[(d, 1, 0)]
                    for (dr, dc), wt in wm.items():
                        m, n = i + dr, j + dc
                        if 0 <= m < ph and 0 <= n < pw:
                            p = int(plane[m, n])
                            tot += wt * f(p - x, S, D)
                            lo, hi = min(lo, p), max(hi, p)
                r = (abs(tot) + 8) // 16
                yv = x + (r if tot >= 0 else -r)
                out[i, j] = min(hi, max(lo, yv))
        outs.append(out)
    return outs


@pytest.mark.parametrize("w,h,bd", [(8, 8, 8), (16, 16, 10), (24, 16, 8), (72, 72, 10)])
def test_filter_frame_brute_force(ref, w, h, bd):
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(w * 1000 + h + bd)
    y, u, v = synth.random_frame_planes(rng, w, h, bd)
    if w == 72:  # smoother content exercises the contrast adjustment
        fr = synth.make_frame(w, h, bd, 32, seed=3)
        y, u, v = fr.rec
    prm = synth.random_params(rng, w, h)
    got = ref.filter_frame(y, u, v, bd, prm)
    exp = _py_filter_frame(ref, y, u, v, bd, prm)
    for g_, e_ in zip(got, exp):
        assert (g_ == e_).all()


def test_filter_frame_all_strengths(ref):
    """Every strength pair x damping x bit depth on one 16x16 frame."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(12)
    for bd in (8, 10):
        y, u, v = synth.random_frame_planes(rng, 16, 16, bd)
        exp_cache = None
        for pri in (0, 1, 2, 3, 7, 8, 15):
            for sec in (0, 1, 2, 4):
                for D in (3, 6):
                    prm = np.zeros((1, 1, 8), np.uint8)
                    prm[0, 0, :5] = (pri, sec, pri, sec, D)
                    got = ref.filter_frame(y, u, v, bd, prm)
                    exp = _py_filter_frame(ref, y, u, v, bd, prm)
                    for g_, e_ in zip(got, exp):
                        assert (g_ == e_).all(), (bd, pri, sec, D)
        del exp_cache


# --------------------------------------------------------------------------
# Section 5: strength search
# --------------------------------------------------------------------------
def test_distortion_matches_filtered_sse(ref):
    """D_{b,q} is the SSE against the source of the frame filtered with pair
    q everywhere; D_{b,(0,0)} is the unfiltered SSE."""
    from paper_1602_05975_gb300 import synth
    fr = synth.make_frame(80, 72, 8, 32, seed=21)
    dl, dc = ref.distortion(fr.rec, fr.src, 8, 4)
    nb = dl.shape[0]
    assert nb == 4
    for q in (0, 5, 22, 63):
        p, s = q // 4, synth.SEC_VALUES[q % 4]
        prm = np.zeros((2, 2, 8), np.uint8)
        prm[..., :5] = (p, s, p, s, 4)
        oy, ou, ov = ref.filter_frame(*fr.rec, 8, prm)
        for b in range(nb):
            by, bx = divmod(b, 2)
            sl = np.s_[by * 64:(by + 1) * 64, bx * 64:(bx + 1) * 64]
            slc = np.s_[by * 32:(by + 1) * 32, bx * 32:(bx + 1) * 32]
            el = ((oy[sl].astype(np.int64) - fr.src[0][sl]) ** 2).sum()
            ec = sum(((o[slc].astype(np.int64) - s_[slc]) ** 2).sum()
                     for o, s_ in ((ou, fr.src[1]), (ov, fr.src[2])))
            assert dl[b, q] == el and dc[b, q] == ec
    # q = 0 is (0, 0): no filtering
    assert dl[0, 0] == ((fr.rec[0][:64, :64].astype(np.int64) - fr.src[0][:64, :64]) ** 2).sum()


def _brute_greedy(dl, dc, lam):
    B = dl.shape[0]
    full = (dl[:, :, None] + dc[:, None, :]).reshape(B, 4096)
    chosen, totals = [], []
    cur = np.full(B, np.iinfo(np.int64).max)
    for _ in range(8):
        tot = np.minimum(cur[:, None], full).sum(0)
        t = int(np.argmin(tot))  # first minimum
        chosen.append(t)
        totals.append(int(tot[t]))
        cur = np.minimum(cur, full[:, t])
    J = {n: totals[n - 1] + lam * B * int(math.log2(n)) for n in (1, 2, 4, 8)}
    best = min((1, 2, 4, 8), key=lambda n: (J[n], n))
    ids = np.argmin(full[:, chosen[:best]], axis=1)
    return chosen, best, J[best], ids, full


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_greedy_matches_brute_force(ref, seed):
    rng = np.random.default_rng(seed)
    B = int(rng.integers(1, 7))
    hi = [5, 50, 10 ** 6, 10 ** 9][seed]  # small ranges force ties
    dl = rng.integers(0, hi, (B, 64)).astype(np.int64)
    dc = rng.integers(0, hi, (B, 64)).astype(np.int64)
    lam = int(rng.integers(0, hi))
    out = ref.select_presets(dl, dc, lam)
    chosen, n, J, ids, _ = _brute_greedy(dl, dc, lam)
    assert list(out["presets"]) == chosen
    assert out["npresets"] == n and out["cost"] == J
    assert (out["block_ids"] == ids).all()


def test_greedy_pair_not_better_than_exhaustive(ref):
    """Greedy J(2) is never below the exhaustive optimum over all preset
    pairs (B <= 4)."""
    rng = np.random.default_rng(30)
    for _ in range(3):
        B = 3
        dl = rng.integers(0, 1000, (B, 64)).astype(np.int64)
        dc = rng.integers(0, 1000, (B, 64)).astype(np.int64)
        out = ref.select_presets(dl, dc, 0)
        full = (dl[:, :, None] + dc[:, None, :]).reshape(B, 4096)
        best_pair = min(int(np.minimum(full[:, [a]], full).sum(0).min())
                        for a in range(4096))
        assert out["costs"][1] >= best_pair
        assert out["costs"][0] == int(full.sum(0).min())


def test_greedy_lambda_extremes(ref):
    rng = np.random.default_rng(31)
    dl = rng.integers(0, 10 ** 6, (20, 64)).astype(np.int64)
    dc = rng.integers(0, 10 ** 6, (20, 64)).astype(np.int64)
    assert ref.select_presets(dl, dc, 10 ** 12)["npresets"] == 1
    out = ref.select_presets(dl, dc, 0)
    assert out["npresets"] == 8
    ties = ref.select_presets(np.zeros((5, 64), np.int64), np.zeros((5, 64), np.int64), 0)
    assert ties["npresets"] == 1 and list(ties["presets"]) == [0] * 8
    assert (ties["block_ids"] == 0).all()


# --------------------------------------------------------------- section 5: preset re-optimisation
def _constructed_tables():
    """Three blocks, luma-only costs (chroma 0): options X = 1, Y = 2, Z = 3
    (luma indices); every other option costs 1000.  The best single preset
    is Z, greedy then adds X, but {X, Y} costs nothing."""
    dl = np.full((3, 64), 1000, np.int64)
    dc = np.zeros((3, 64), np.int64)
    dl[0, [1, 2, 3]] = [0, 10, 4]
    dl[1, [1, 2, 3]] = [10, 0, 4]
    dl[2, [1, 2, 3]] = [0, 0, 0]
    return dl, dc


def test_refinement_escapes_greedy_trap(ref):
    dl, dc = _constructed_tables()
    g = ref.select_presets(dl, dc, 0)
    assert list(g["presets"][:2]) == [3 * 64, 1 * 64]            # Z, then X
    p, total, passes = ref.refine_presets(dl, dc, g["presets"][:2], 8)
    assert sorted(int(t) >> 6 for t in p) == [1, 2] and total == 0
    assert passes == 2                                            # one changing pass, one quiet


def _total(dl, dc, presets):
    d = dl[:, np.asarray(presets) >> 6] + dc[:, np.asarray(presets) & 63]
    return int(d.min(axis=1).sum())


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_refinement_is_a_local_optimum_and_never_worse(ref, seed):
    rng = np.random.default_rng(seed)
    dl = rng.integers(0, 500, (5, 64)).astype(np.int64)
    dc = rng.integers(0, 500, (5, 64)).astype(np.int64)
    g = ref.select_presets(dl, dc, 0)
    for n in (2, 4):
        start = g["presets"][:n].copy()
        p, total, _ = ref.refine_presets(dl, dc, start, 16)
        assert total == _total(dl, dc, p) <= _total(dl, dc, start)
        # brute force: no single replacement lowers the total
        for k in range(n):
            best = min(_total(dl, dc, np.concatenate([p[:k], [t], p[k + 1:]]))
                       for t in range(4096))
            assert best == total


def test_refinement_keeps_a_local_optimum_and_zero_passes_is_greedy(ref):
    rng = np.random.default_rng(9)
    dl = rng.integers(0, 300, (4, 64)).astype(np.int64)
    dc = rng.integers(0, 300, (4, 64)).astype(np.int64)
    g = ref.select_presets(dl, dc, 5)
    r0 = ref.select_presets_refined(dl, dc, 5, 0)
    assert r0["cost"] == g["cost"] and r0["npresets"] == g["npresets"]
    assert list(r0["presets"][:g["npresets"]]) == list(g["presets"][:g["npresets"]])
    p, total, _ = ref.refine_presets(dl, dc, g["presets"][:2], 16)
    p2, total2, passes2 = ref.refine_presets(dl, dc, p, 16)
    assert list(p2) == list(p) and total2 == total and passes2 == 1


def test_refined_selection_cost_not_above_greedy(ref):
    dl, dc = _constructed_tables()
    for lam in (0, 1, 3, 100):
        g = ref.select_presets(dl, dc, lam)
        r = ref.select_presets_refined(dl, dc, lam, 8)
        assert r["cost"] <= g["cost"]
    r = ref.select_presets_refined(dl, dc, 0, 8)
    assert r["cost"] == 0 and r["npresets"] == 2


# --------------------------------------------------------------- section 4: skip semantics
def _skip_case(seed=11, w=192, h=128, bd=8):
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(seed)
    f = synth.make_frame(w, h, bd, 32, seed=seed)
    params = synth.random_params(rng, w, h)
    params[..., 0] = np.maximum(params[..., 0], 3)      # every block really filters
    params[..., 2] = np.maximum(params[..., 2], 3)
    return f, params, rng


def _block(planes, fby, fbx, sub=0):
    s = 64 >> sub
    return planes[sub > 0 and 1 or 0][fby * s:(fby + 1) * s, fbx * s:(fbx + 1) * s]


def test_skipped_filter_block_is_not_filtered(ref):
    """Section 4: a filter block without coded residual has CDEF disabled,
    whatever its parameters and skip-condition bits."""
    f, params, _ = _skip_case()
    params[..., 5] = 3
    coded = np.ones((f.height // 8, f.width // 8), np.uint8)
    coded[0:8, 8:16] = 0                                   # filter block (0, 1) has none
    out = ref.filter_frame(*f.rec, 8, params, coded=coded)
    full = ref.filter_frame(*f.rec, 8, params)
    assert np.array_equal(out[0][0:64, 64:128], f.rec[0][0:64, 64:128])
    for k in (1, 2):
        assert np.array_equal(out[k][0:32, 32:64], f.rec[k][0:32, 32:64])
    assert not np.array_equal(full[0][0:64, 64:128], f.rec[0][0:64, 64:128])
    # other filter blocks are untouched by the map
    assert np.array_equal(out[0][:, 128:], full[0][:, 128:])


def test_uncoded_8x8_filtered_only_with_skip_condition(ref):
    """Section 4: in a coded filter block an 8x8 block without residual is
    filtered only when the preset's skip-condition bit is set (per plane
    group; chroma follows the co-located luma block)."""
    f, params, _ = _skip_case()
    coded = np.ones((f.height // 8, f.width // 8), np.uint8)
    coded[2, 3] = 0                                        # luma rows 16..23, cols 24..31
    params[..., 5] = 0
    off = ref.filter_frame(*f.rec, 8, params, coded=coded)
    full = ref.filter_frame(*f.rec, 8, params)
    assert np.array_equal(off[0][16:24, 24:32], f.rec[0][16:24, 24:32])
    assert np.array_equal(off[1][8:12, 12:16], f.rec[1][8:12, 12:16])
    m = np.ones(off[0].shape, bool)
    m[16:24, 24:32] = False
    assert np.array_equal(off[0][m], full[0][m])
    params[..., 5] = 1                                     # luma skip condition only
    lum = ref.filter_frame(*f.rec, 8, params, coded=coded)
    assert np.array_equal(lum[0], full[0])
    assert np.array_equal(lum[1][8:12, 12:16], f.rec[1][8:12, 12:16])
    params[..., 5] = 2                                     # chroma only
    chro = ref.filter_frame(*f.rec, 8, params, coded=coded)
    assert np.array_equal(chro[1], full[1]) and np.array_equal(chro[2], full[2])
    assert np.array_equal(chro[0][16:24, 24:32], f.rec[0][16:24, 24:32])


def test_zero_strengths_with_skip_condition_mean_19_and_7(ref):
    """Section 4: (0, 0) with the skip-condition bit set filters with primary
    19 and secondary 7; without it, (0, 0) is the identity."""
    f, params, _ = _skip_case(seed=12)
    params[..., 0:4] = 0
    params[..., 5] = 0
    ident = ref.filter_frame(*f.rec, 8, params)
    assert all(np.array_equal(a, b) for a, b in zip(ident, f.rec))
    params[..., 5] = 3
    mapped = ref.filter_frame(*f.rec, 8, params)
    explicit = params.copy()
    explicit[..., 5] = 0
    explicit[..., 0], explicit[..., 1], explicit[..., 2], explicit[..., 3] = 19, 7, 19, 7
    assert all(np.array_equal(a, b) for a, b in zip(mapped, ref.filter_frame(*f.rec, 8, explicit)))
    assert not np.array_equal(mapped[0], f.rec[0])


def test_all_coded_map_equals_no_map(ref):
    f, params, rng = _skip_case(seed=13, bd=10)
    params[..., 5] = rng.integers(0, 4, params.shape[:2])
    coded = np.ones((f.height // 8, f.width // 8), np.uint8) * 7
    a = ref.filter_frame(*f.rec, 10, params, coded=coded)
    b = ref.filter_frame(*f.rec, 10, params)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_skip_bits_out_of_range_rejected(ref):
    f, params, _ = _skip_case(seed=14)
    params[0, 0, 5] = 4
    with pytest.raises(ValueError):
        ref.filter_frame(*f.rec, 8, params)


# --------------------------------------------------------------- section 5 with section 4's skip bits
def _sse_blocks(out, src, sub):
    s = 64 >> sub
    planes = (0,) if sub == 0 else (1, 2)
    h, w = out[planes[0]].shape
    res = []
    for by in range(-(-h // s)):
        for bx in range(-(-w // s)):
            e = 0
            for k in planes:
                d = out[k][by * s:(by + 1) * s, bx * s:(bx + 1) * s].astype(np.int64) - \
                    src[k][by * s:(by + 1) * s, bx * s:(bx + 1) * s].astype(np.int64)
                e += int((d * d).sum())
            res.append(e)
    return res


@pytest.mark.parametrize("bd", [8, 10])
def test_coded_distortion_is_sse_of_decoder_output(ref, bd):
    """Each of the 128 entries is the squared error of what the decoder
    outputs (section 4 semantics) for that preset."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(192, 72, bd, 32, seed=40 + bd)
    rng = np.random.default_rng(bd)
    coded = (rng.random((9, 24)) < 0.5).astype(np.uint8)
    coded[:, 16:] = 0                                     # filter blocks 2 and 5 skipped
    dl, dc, sk = ref.distortion_coded(f.rec, f.src, bd, 5, coded)
    assert list(sk) == [0, 0, 1, 0, 0, 1]
    params = np.zeros(f.params.shape, np.uint8)
    params[..., 4] = 5
    for q in range(128):
        k, p, s = q >> 6, (q & 63) >> 2, q & 3
        params[..., 0] = params[..., 2] = p
        params[..., 1] = params[..., 3] = (0, 1, 2, 4)[s]
        params[..., 5] = 3 * k
        out = ref.filter_frame(*f.rec, bd, params, coded=coded)
        assert _sse_blocks(out, f.src, 0) == list(dl[:, q]), q
        assert _sse_blocks(out, f.src, 1) == list(dc[:, q]), q
    # skipped blocks: every entry is the unfiltered error
    assert (dl[sk == 1] == dl[sk == 1][:, :1]).all()


def test_coded_tables_with_every_block_coded(ref):
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(128, 64, 8, 16, seed=44)
    dl, dc, sk = ref.distortion_coded(f.rec, f.src, 8, 4, None)
    old_l, old_c = ref.distortion(f.rec, f.src, 8, 4)
    assert not sk.any()
    assert (dl[:, 1:64] == old_l[:, 1:]).all() and (dl[:, 65:] == old_l[:, 1:]).all()
    assert (dc[:, 1:64] == old_c[:, 1:]).all() and (dc[:, 65:] == old_c[:, 1:]).all()
    assert (dl[:, 0] == old_l[:, 0]).all()                # (0, 0), no skip bit: unfiltered
    assert (dl[:, 64] != old_l[:, 0]).any()                # (0, 0) + skip: (19, 7)


def test_general_selection_matches_width_64_functions(ref):
    rng = np.random.default_rng(21)
    dl = rng.integers(0, 400, (5, 64)).astype(np.int64)
    dc = rng.integers(0, 400, (5, 64)).astype(np.int64)
    for lam, passes in [(0, 0), (7, 0), (3, 4), (50, 16)]:
        a = ref.select_presets_general(dl, dc, 64, None, lam, passes)
        b = ref.select_presets_refined(dl, dc, lam, passes)
        assert a["cost"] == b["cost"] and a["npresets"] == b["npresets"]
        assert list(a["presets"]) == list(b["presets"])
        assert np.array_equal(a["block_ids"], b["block_ids"])


def test_skipped_blocks_leave_the_selection(ref):
    """Blocks without coded residual signal no preset: their distortion is
    constant and they count neither in the sums nor in B."""
    rng = np.random.default_rng(22)
    dl = rng.integers(0, 400, (6, 128)).astype(np.int64)
    dc = rng.integers(0, 400, (6, 128)).astype(np.int64)
    sk = np.array([0, 1, 0, 0, 1, 0], np.uint8)
    full = ref.select_presets_general(dl, dc, 128, sk, 9, 2)
    sub = ref.select_presets_general(dl[sk == 0], dc[sk == 0], 128, None, 9, 2)
    assert full["cost"] == sub["cost"] and full["npresets"] == sub["npresets"]
    assert list(full["presets"]) == list(sub["presets"])
    assert list(full["block_ids"][sk == 0]) == list(sub["block_ids"])
    assert (full["block_ids"][sk == 1] == 0).all()


# --------------------------------------------------------------- section 5: low-complexity subset
def _mask(bits):
    m = 0
    for q in bits:
        m |= 1 << q
    return m


@pytest.mark.parametrize("seed", [40, 41, 42])
def test_subset_greedy_matches_brute_force(ref, seed):
    """R26: the greedy search over the allowed presets equals a brute-force
    greedy that only looks at presets whose two pairs are allowed; every
    chosen preset is allowed."""
    rng = np.random.default_rng(seed)
    B = int(rng.integers(1, 6))
    dl = rng.integers(0, 300, (B, 64)).astype(np.int64)
    dc = rng.integers(0, 300, (B, 64)).astype(np.int64)
    lq = sorted(set(rng.integers(0, 64, 9).tolist()))
    cq = sorted(set(rng.integers(0, 64, 5).tolist()))
    lam = int(rng.integers(0, 100))
    out = ref.select_presets_subset(dl, dc, 64, None, _mask(lq), _mask(cq), lam)
    full = (dl[:, :, None] + dc[:, None, :]).reshape(B, 4096)
    allowed = np.array([(t // 64 in lq) and (t % 64 in cq) for t in range(4096)])
    cur = np.full(B, np.iinfo(np.int64).max)
    chosen, totals = [], []
    for _ in range(8):
        tot = np.minimum(cur[:, None], full).sum(0)
        tot = np.where(allowed, tot, np.iinfo(np.int64).max)
        t = int(np.argmin(tot))
        chosen.append(t)
        totals.append(int(tot[t]))
        cur = np.minimum(cur, full[:, t])
    J = {n: totals[n - 1] + lam * B * int(math.log2(n)) for n in (1, 2, 4, 8)}
    best = min((1, 2, 4, 8), key=lambda n: (J[n], n))
    assert list(out["presets"]) == chosen
    assert out["npresets"] == best and out["cost"] == J[best]
    assert (out["block_ids"] == np.argmin(full[:, chosen[:best]], axis=1)).all()
    assert all(allowed[t] for t in out["presets"])


def test_subset_of_one_pair_and_full_masks(ref):
    rng = np.random.default_rng(43)
    dl = rng.integers(0, 500, (7, 64)).astype(np.int64)
    dc = rng.integers(0, 500, (7, 64)).astype(np.int64)
    one = ref.select_presets_subset(dl, dc, 64, None, 1 << 22, 1 << 5, 0, 3)
    assert list(one["presets"]) == [22 * 64 + 5] * 8
    assert one["npresets"] == 1 and one["cost"] == int((dl[:, 22] + dc[:, 5]).sum())
    assert (one["block_ids"] == 0).all()
    every = (1 << 64) - 1
    for lam, passes in [(0, 0), (30, 4)]:
        a = ref.select_presets_subset(dl, dc, 64, None, every, every, lam, passes)
        b = ref.select_presets_general(dl, dc, 64, None, lam, passes)
        assert list(a["presets"]) == list(b["presets"]) and a["cost"] == b["cost"]
        # a smaller subset never does better at N = 1
        c = ref.select_presets_subset(dl, dc, 64, None, every >> 32, every, lam, passes)
        assert c["cost"] >= b["cost"] or c["npresets"] != 1
    with pytest.raises(ValueError):
        ref.select_presets_subset(dl, dc, 64, None, 0, every, 0)


def test_subset_applies_to_both_skip_bit_halves(ref):
    """In the 128-combination tables the mask of pair q allows q and 64 + q:
    restricting the tables to those columns and searching them in full gives
    the same presets (mapped back)."""
    rng = np.random.default_rng(44)
    dl = rng.integers(0, 400, (5, 128)).astype(np.int64)
    dc = rng.integers(0, 400, (5, 128)).astype(np.int64)
    sk = np.array([0, 0, 1, 0, 0], np.uint8)
    lq, cq = [3, 17, 40], [0, 9]
    out = ref.select_presets_subset(dl, dc, 128, sk, _mask(lq), _mask(cq), 11, 2)
    lcols = lq + [64 + q for q in lq]
    ccols = cq + [64 + q for q in cq]
    # brute force over the allowed presets, restated with explicit columns
    full = dl[:, lcols][:, :, None] + dc[:, ccols][:, None, :]
    best1 = min(int(full[sk == 0, i, j].sum()) for i in range(len(lcols)) for j in range(len(ccols)))
    t0 = int(out["presets"][0])
    assert (t0 // 128) in lcols and (t0 % 128) in ccols
    assert int((dl[sk == 0, t0 // 128] + dc[sk == 0, t0 % 128]).sum()) == best1


# --------------------------------------------------------------- chroma formats (section 4)
def _format_frame(fmt, w=192, h=136, bd=8, seed=60):
    rng = np.random.default_rng(seed)
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(w, h, bd, 32, seed=seed)
    cw, ch = (w // 2, h) if fmt == 422 else (w, h)
    mx = (1 << bd) - 1
    u = np.clip(f.rec[0][:ch, :cw].astype(np.int64) // 2 + rng.integers(0, 40, (ch, cw)), 0, mx)
    v = np.clip(mx - f.rec[0][:ch, :cw].astype(np.int64) + rng.integers(0, 40, (ch, cw)), 0, mx)
    return f, u.astype(np.uint16), v.astype(np.uint16), synth.random_params(rng, w, h)


def test_422_chroma_is_not_filtered(ref):
    """Section 4: with different horizontal and vertical subsampling (4:2:2)
    the filter is disabled for chroma; luma is filtered as for 4:2:0."""
    f, u, v, params = _format_frame(422)
    oy, ou, ov = ref.filter_frame_format(f.rec[0], u, v, 8, params, 422)
    assert np.array_equal(ou, u) and np.array_equal(ov, v)
    assert np.array_equal(oy, ref.filter_frame(*f.rec, 8, params)[0])


def test_444_chroma_matches_luma_path_for_secondary_only(ref):
    """4:4:4 chroma is filtered like luma with the chroma parameters: with
    primary strengths 0 (no contrast adjustment involved) a chroma plane
    equal to the luma plane at chroma damping D + 1 gives the luma output
    at damping D (chroma uses D - 1, section 3.2)."""
    f, _, _, params = _format_frame(444, bd=10, seed=61)
    params[..., 0] = params[..., 2] = 0
    params[..., 4] = np.minimum(params[..., 4], 5)
    y = f.rec[0]
    luma = ref.filter_frame_format(y, y, y, 10, params, 444)[0]
    up = params.copy()
    up[..., 4] += 1
    up[..., 3] = up[..., 1]
    chroma = ref.filter_frame_format(y, y, y, 10, up, 444)
    assert np.array_equal(chroma[1], luma) and np.array_equal(chroma[2], luma)


def test_444_identities(ref):
    f, u, v, params = _format_frame(444, seed=62)
    params[..., 2] = params[..., 3] = 0                      # chroma strengths 0
    oy, ou, ov = ref.filter_frame_format(f.rec[0], u, v, 8, params, 444)
    assert np.array_equal(ou, u) and np.array_equal(ov, v)
    const = np.full_like(u, 77)
    params[..., 2], params[..., 3] = 9, 2
    _, cu, _ = ref.filter_frame_format(f.rec[0], const, const, 8, params, 444)
    assert np.array_equal(cu, const)


def _format_src(f, u, v, seed):
    """A source frame for the format tests: the luma source and chroma
    planes near the decoded ones (what a coder leaves)."""
    rng = np.random.default_rng(seed)
    mx = (1 << f.bitdepth) - 1
    su = np.clip(u.astype(np.int64) + rng.integers(-6, 7, u.shape), 0, mx).astype(np.uint16)
    sv = np.clip(v.astype(np.int64) + rng.integers(-6, 7, v.shape), 0, mx).astype(np.uint16)
    return (f.src[0], su, sv)


@pytest.mark.parametrize("fmt,bd", [(444, 8), (444, 10), (422, 8), (420, 12)])
def test_format_tables_are_sse_of_decoder_output(ref, fmt, bd):
    """Reading R25 in section 5's tables: each entry is the squared error of
    what the filter oracle outputs for that strength pair everywhere (4:2:2
    chroma: the unfiltered error for every pair)."""
    from paper_1602_05975_gb300 import synth
    if fmt == 420:
        f = synth.make_frame(136, 72, bd, 32, seed=75)
        planes, src = f.rec, f.src
    else:
        f, u, v, _ = _format_frame(fmt, w=136, h=72, bd=bd, seed=76)
        planes, src = (f.rec[0], u, v), _format_src(f, u, v, 77)
    dl, dc = ref.distortion_format(planes, src, bd, 5, fmt)
    params = np.zeros(f.params.shape, np.uint8)
    params[..., 4] = 5
    for q in (0, 6, 29, 63):
        p, s = q >> 2, (0, 1, 2, 4)[q & 3]
        params[..., 0] = params[..., 2] = p
        params[..., 1] = params[..., 3] = s
        out = ref.filter_frame_format(*planes, bd, params, fmt)
        for b in range(dl.shape[0]):
            by, bx = divmod(b, f.params.shape[1])
            ly = np.s_[by * 64:(by + 1) * 64, bx * 64:(bx + 1) * 64]
            el = int(((out[0][ly].astype(np.int64) - src[0][ly]) ** 2).sum())
            cy, cx = ((64, 64) if fmt == 444 else (64, 32) if fmt == 422 else (32, 32))
            cs = np.s_[by * cy:(by + 1) * cy, bx * cx:(bx + 1) * cx]
            ec = sum(int(((out[k][cs].astype(np.int64) - src[k][cs]) ** 2).sum()) for k in (1, 2))
            assert dl[b, q] == el and dc[b, q] == ec, (fmt, bd, q, b)
    if fmt == 422:
        assert (dc == dc[:, :1]).all()      # chroma is not filtered: one value per block


@pytest.mark.parametrize("fmt,bd", [(444, 8), (422, 10), (420, 12)])
def test_coded_format_tables_are_sse_of_decoder_output(ref, fmt, bd):
    """Readings R21 and R25 together: each of the 128 entries is the squared
    error of what the filter oracle outputs with that preset (skip-condition
    bit included) and the coded-residual map; blocks without residual are
    flagged and keep the unfiltered error."""
    from paper_1602_05975_gb300 import synth
    rng = np.random.default_rng(78)
    if fmt == 420:
        f = synth.make_frame(136, 72, bd, 32, seed=79)
        planes, src = f.rec, f.src
    else:
        f, u, v, _ = _format_frame(fmt, w=136, h=72, bd=bd, seed=80)
        planes, src = (f.rec[0], u, v), _format_src(f, u, v, 81)
    coded = (rng.random((9, 17)) < 0.5).astype(np.uint8)
    coded[:8, 8:16] = 0                                   # filter block 1: no residual
    dl, dc, sk = ref.distortion_coded_format(planes, src, bd, 5, fmt, coded)
    assert list(sk) == [0, 1, 0, 0, 0, 0]
    params = np.zeros(f.params.shape, np.uint8)
    params[..., 4] = 5
    for q in (0, 9, 63, 64, 77, 127):
        k, p, s = q >> 6, (q >> 2) & 15, (0, 1, 2, 4)[q & 3]
        params[..., 0] = params[..., 2] = p
        params[..., 1] = params[..., 3] = s
        params[..., 5] = 3 * k                            # the same bit for both groups
        out = ref.filter_frame_format(*planes, bd, params, fmt, coded)
        for b in range(dl.shape[0]):
            by, bx = divmod(b, f.params.shape[1])
            ly = np.s_[by * 64:(by + 1) * 64, bx * 64:(bx + 1) * 64]
            el = int(((out[0][ly].astype(np.int64) - src[0][ly]) ** 2).sum())
            cy, cx = ((64, 64) if fmt == 444 else (64, 32) if fmt == 422 else (32, 32))
            cs = np.s_[by * cy:(by + 1) * cy, bx * cx:(bx + 1) * cx]
            ec = sum(int(((out[c][cs].astype(np.int64) - src[c][cs]) ** 2).sum()) for c in (1, 2))
            assert dl[b, q] == el and dc[b, q] == ec, (fmt, bd, q, b)


def test_unknown_format_rejected(ref):
    f, u, v, params = _format_frame(444, seed=63)
    with pytest.raises(ValueError):
        ref.filter_frame_format(f.rec[0], u, v, 8, params, 411)


# --------------------------------------------------------------- section 5, eq. 14
def _sums(sv, dv):
    sv = sv.astype(np.int64).ravel()
    dv = dv.astype(np.int64).ravel()
    return (sv.size, int(sv.sum()), int((sv * sv).sum()), int(dv.sum()), int((dv * dv).sum()),
            int(((dv - sv) ** 2).sum()))


def test_eq14_term_invariances(ref):
    """The 8x8 function of eq. 14 is symmetric in source and decoded block,
    translation invariant (variances and errors do not change), and scales
    with the squared error when both variances vanish."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        s = rng.integers(0, 256, 64)
        d = np.clip(s + rng.integers(-20, 21, 64), 0, 255)
        t = ref.eq14_term(*_sums(s, d), 8)
        assert t == ref.eq14_term(*_sums(d, s), 8)
        assert t == ref.eq14_term(*_sums(s + 300, d + 300), 8)
        assert t >= 0
    # flat blocks: D = C1 / (2 sqrt(C2)) * sse with C1 = 6.25, C2 = 312.5
    s = np.full(64, 100)
    d = np.full(64, 103)
    assert ref.eq14_term(*_sums(s, d), 8) == round(256 * 6.25 / (2 * 312.5 ** 0.5) * 64 * 9)


def test_eq14_constants_scale_with_bit_depth(ref):
    """R23: at 10 bits samples x4 give exactly 16 times the 8-bit value
    (before the rounding to 1/256)."""
    rng = np.random.default_rng(4)
    for _ in range(100):
        s = rng.integers(0, 256, 64)
        d = np.clip(s + rng.integers(-30, 31, 64), 0, 255)
        t8 = ref.eq14_term(*_sums(s, d), 8)
        t10 = ref.eq14_term(*_sums(4 * s, 4 * d), 10)
        assert abs(t10 - 16 * t8) <= 8


def _eq14_exact_256(n, s1s, s2s, s1d, s2d, sse, bd):
    """256 * eq. 14 for one 8x8 block taken exactly: rational variances and
    constants, a 60-digit square root."""
    import decimal
    from fractions import Fraction
    ctx = decimal.Context(prec=60)
    c1 = Fraction(25, 4) * 4 ** (bd - 8)
    c2 = Fraction(625, 2) * 16 ** (bd - 8)
    vs = Fraction(n * s2s - s1s * s1s, n * n)
    vd = Fraction(n * s2d - s1d * s1d, n * n)
    rad = vs * vd + c2
    root = ctx.sqrt(ctx.divide(decimal.Decimal(rad.numerator), decimal.Decimal(rad.denominator)))
    num = vs + vd + c1
    num_d = ctx.divide(decimal.Decimal(num.numerator), decimal.Decimal(num.denominator))
    return ctx.multiply(ctx.divide(ctx.multiply(256 * num_d, decimal.Decimal(sse)), 2 * root), 1)


def test_eq14_term_is_exact_value_rounded(ref):
    """R24: each 8x8 value is round(256 * D) of eq. 14 taken exactly
    (rational variances, 60-digit square root), ties away from zero; only a
    value within a relative 2^-48 of a half-integer may round either way.
    Covers full and edge-cut blocks (n = 64, 32, 16), flat blocks and every
    bit depth."""
    import decimal
    rng = np.random.default_rng(5)
    near_ties = 0
    for bd in (8, 10, 12):
        for n in (64, 32, 16):
            for _ in range(150):
                s = rng.integers(0, 1 << bd, n)
                d = np.clip(s + rng.integers(-60, 61, n) * (1 << (bd - 8)), 0, (1 << bd) - 1)
                if rng.random() < 0.3:
                    d = np.full(n, int(d.mean()))
                sums = _sums(s, d)
                exact = _eq14_exact_256(*sums, bd)
                got = ref.eq14_term(*sums, bd)
                lo = int(exact.to_integral_value(rounding=decimal.ROUND_HALF_UP))
                frac = exact - int(exact)
                if abs(frac - decimal.Decimal("0.5")) <= exact * decimal.Decimal(2) ** -48:
                    near_ties += 1
                    assert got in (int(exact), int(exact) + 1)
                else:
                    assert got == lo, (bd, n, sums, exact, got)
    assert near_ties < 5


def test_eq14_term_catches_dropped_terms(ref):
    """Each part of eq. 14 moves the value: a dropped C1, C2, factor 2, or a
    variance taken as the sample variance (n - 1) would each change the
    term of one of these blocks."""
    rng = np.random.default_rng(51)
    s = rng.integers(0, 256, 64)
    d = np.clip(s + rng.integers(-9, 10, 64), 0, 255)
    sums = _sums(s, d)
    got = ref.eq14_term(*sums, 8)
    n, s1s, s2s, s1d, s2d, sse = sums
    vs = (n * s2s - s1s * s1s) / n ** 2
    vd = (n * s2d - s1d * s1d) / n ** 2
    variants = [
        (vs + vd) / (2 * (vs * vd + 312.5) ** 0.5) * sse,           # no C1
        (vs + vd + 6.25) / (2 * (vs * vd) ** 0.5) * sse,            # no C2
        (vs + vd + 6.25) / ((vs * vd + 312.5) ** 0.5) * sse,        # no factor 2
        (vs * n / (n - 1) + vd * n / (n - 1) + 6.25)
        / (2 * (vs * vd * (n / (n - 1)) ** 2 + 312.5) ** 0.5) * sse,  # sample variances
    ]
    for v in variants:
        assert abs(round(256 * v) - got) > 2


def test_eq14_large_variance_tends_to_sse(ref):
    s = np.tile(np.array([0, 255]), 32)
    d = s.copy()
    d[0] = 5
    t = ref.eq14_term(*_sums(s, d), 8)
    assert abs(t / 256 - 25) < 0.02 * 25


def test_eq14_tables_from_decoder_output(ref):
    """Each table entry is the sum over the 8x8 blocks of every plane of the
    eq. 14 value of the filter oracle's output for that strength pair
    (chroma 8x8 blocks cut by the frame edge included)."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(136, 72, 8, 32, seed=71)         # chroma 68x36: partial 8x8 blocks
    dl, dc = ref.distortion_eq14(f.rec, f.src, 8, 5)
    params = np.zeros(f.params.shape, np.uint8)
    params[..., 4] = 5
    for q in (0, 5, 22, 37, 63):
        p, s = q >> 2, (0, 1, 2, 4)[q & 3]
        params[..., 0] = params[..., 2] = p
        params[..., 1] = params[..., 3] = s
        out = ref.filter_frame(*f.rec, 8, params)
        for pl, tab in ((0, dl), (1, dc)):
            fb = 64 >> (pl > 0)
            planes = (0,) if pl == 0 else (1, 2)
            h, w = out[planes[0]].shape
            for b in range(tab.shape[0]):
                by, bx = divmod(b, f.params.shape[1])
                tot = 0
                for k in planes:
                    for y in range(by * fb, min((by + 1) * fb, h), 8):
                        for x in range(bx * fb, min((bx + 1) * fb, w), 8):
                            tot += ref.eq14_term(*_sums(f.src[k][y:y + 8, x:x + 8],
                                                        out[k][y:y + 8, x:x + 8]), 8)
                assert tab[b, q] == tot, (q, pl, b)


def test_periodic_frame_tables_by_class(ref):
    """The construction behind the large-frame search tests: the oracle's
    tables of frames that tile a 128x128 pattern equal the tables gathered
    by block class from the 4x4-block frame of the pattern, and so do the
    presets selected on them."""
    from periodic_frames import periodic_search_case
    for bd in (8, 10):
        for c in periodic_search_case(ref, [(512, 384), (384, 256)], bd, seed=6100 + bd):
            dl, dc = ref.distortion(c["rec"], c["src"], bd, c["damping"])
            assert np.array_equal(dl, c["dl"]) and np.array_equal(dc, c["dc"])
            o = ref.select_presets(dl, dc, c["lam"])
            assert list(o["presets"]) == list(c["exp"]["presets"])
            assert np.array_equal(o["block_ids"], c["exp"]["block_ids"])
        for c in periodic_search_case(ref, [(512, 384)], bd, seed=6200 + bd, coded=True):
            dl, dc, sk = ref.distortion_coded(c["rec"], c["src"], bd, c["damping"], c["coded"])
            assert np.array_equal(dl, c["dl"]) and np.array_equal(dc, c["dc"])
            assert np.array_equal(sk, c["skipped"]) and 0 < sk.sum() < sk.size
            o = ref.select_presets_general(dl, dc, 128, sk, c["lam"])
            assert list(o["presets"]) == list(c["exp"]["presets"])
            assert np.array_equal(o["block_ids"], c["exp"]["block_ids"])


def test_eq14_format_tables_for_420_equal_the_420_oracle(ref):
    """The format-aware eq. 14 tables reduce to the 4:2:0 ones (8 and 12
    bits, a chroma plane with edge-cut 8x8 blocks)."""
    from paper_1602_05975_gb300 import synth
    for bd, (w, h) in ((8, (136, 72)), (12, (72, 40))):
        f = synth.make_frame(w, h, bd, 32, seed=72 + bd)
        a = ref.distortion_eq14(f.rec, f.src, bd, 4)
        b = ref.distortion_eq14_format(f.rec, f.src, bd, 4, 420)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("fmt,bd", [(444, 8), (422, 10), (444, 12)])
def test_eq14_format_tables_from_decoder_output(ref, fmt, bd):
    """Each entry of the 4:2:2 / 4:4:4 eq. 14 tables is the sum over the 8x8
    blocks of each plane (the plane's own grid, edge-cut blocks included) of
    eq. 14 on the filter oracle's output for that pair (reading R25: 4:2:2
    chroma unfiltered, 4:4:4 chroma filtered in 8x8 blocks with the chroma
    strengths)."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(136, 72, bd, 32, seed=73, chroma=fmt)
    dl, dc = ref.distortion_eq14_format(f.rec, f.src, bd, 5, fmt)
    params = np.zeros(f.params.shape, np.uint8)
    params[..., 4] = 5
    fr, fc = f.params.shape[:2]
    for q in (0, 6, 37, 63):
        p, s = q >> 2, (0, 1, 2, 4)[q & 3]
        params[..., 0] = params[..., 2] = p
        params[..., 1] = params[..., 3] = s
        out = ref.filter_frame_format(*f.rec, bd, params, fmt)
        for pl, tab in ((0, dl), (1, dc)):
            planes = (0,) if pl == 0 else (1, 2)
            h, w = out[planes[0]].shape
            fh, fw = -(-h // fr), -(-w // fc)          # the filter block in this plane
            fh, fw = (64 if fh > 32 else 32), (64 if fw > 32 else 32)
            for b in range(tab.shape[0]):
                by, bx = divmod(b, fc)
                tot = 0
                for k in planes:
                    for y in range(by * fh, min((by + 1) * fh, h), 8):
                        for x in range(bx * fw, min((bx + 1) * fw, w), 8):
                            tot += ref.eq14_term(*_sums(f.src[k][y:y + 8, x:x + 8],
                                                        out[k][y:y + 8, x:x + 8]), bd)
                assert tab[b, q] == tot, (fmt, bd, q, pl, b)


@pytest.mark.parametrize("fmt,bd", [(420, 8), (444, 10), (422, 12)])
def test_eq14_coded_tables_from_decoder_output(ref, fmt, bd):
    """Each entry of the 128-combination eq. 14 tables (reading R21 with
    R22-R25) is the sum over the 8x8 blocks of each plane of eq. 14 on what
    the filter oracle outputs for that preset with the coded-residual map:
    skip bit clear leaves uncoded blocks unfiltered, (0, 0) with the bit set
    is (19, 7), a filter block without coded residual is never filtered."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(136, 72, bd, 32, seed=74, chroma=fmt)
    rng = np.random.default_rng(75)
    coded = (rng.random((9, 17)) < 0.5).astype(np.uint8)
    coded[:, 8:16] = 0                       # filter block (0, 1) without residual
    dl, dc, sk = ref.distortion_eq14_coded_format(f.rec, f.src, bd, 5, fmt, coded)
    assert sk.tolist() == [int(not coded[by * 8:by * 8 + 8, bx * 8:bx * 8 + 8].any())
                           for by in range(2) for bx in range(3)]
    assert sk[1] == 1 and sk[0] == 0
    fr, fc = f.params.shape[:2]
    params = np.zeros(f.params.shape, np.uint8)
    params[..., 4] = 5
    for q in (0, 64, 6, 70, 101):
        k, p, s = q >> 6, (q & 63) >> 2, (0, 1, 2, 4)[q & 3]
        params[..., 0] = params[..., 2] = p
        params[..., 1] = params[..., 3] = s
        params[..., 5] = 3 * k                 # the skip-condition bits of both groups
        out = ref.filter_frame_format(*f.rec, bd, params, fmt, coded=coded)
        for pl, tab in ((0, dl), (1, dc)):
            planes = (0,) if pl == 0 else (1, 2)
            h, w = out[planes[0]].shape
            fh = 64 if -(-h // fr) > 32 else 32
            fw = 64 if -(-w // fc) > 32 else 32
            for b in range(tab.shape[0]):
                by, bx = divmod(b, fc)
                tot = 0
                for kk in planes:
                    for y in range(by * fh, min((by + 1) * fh, h), 8):
                        for x in range(bx * fw, min((bx + 1) * fw, w), 8):
                            tot += ref.eq14_term(*_sums(f.src[kk][y:y + 8, x:x + 8],
                                                        out[kk][y:y + 8, x:x + 8]), bd)
                assert tab[b, q] == tot, (fmt, bd, q, pl, b)


def test_eq14_coded_tables_all_coded_reduce_to_64(ref):
    """With every 8x8 block coded, both skip-bit halves equal the 64-pair
    eq. 14 tables, except the (0, 0) slot with the bit set ((19, 7))."""
    from paper_1602_05975_gb300 import synth
    f = synth.make_frame(136, 72, 10, 32, seed=76)
    dl, dc, sk = ref.distortion_eq14_coded_format(f.rec, f.src, 10, 4, 420,
                                                  np.ones((9, 17), np.uint8))
    el, ec = ref.distortion_eq14_format(f.rec, f.src, 10, 4, 420)
    assert not sk.any()
    for t, e in ((dl, el), (dc, ec)):
        assert np.array_equal(t[:, :64], e)
        assert np.array_equal(t[:, 65:], e[:, 1:])
