"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them compares the oracle with
itself: expected values come from the paper's worked example, closed forms,
exact rational arithmetic, brute force on tiny inputs, or invariants.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import streamfmt
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Eq. 2 and the worked example of Sec. 4.1
# --------------------------------------------------------------------------

def test_worked_example_widths_on_lattice(oracle_mod):
    """Sec. 4.1 worked example: with eps = 0.005 the lattice step is 0.01, so the
    AABB corners and the centre particle have codes x (0,3000,1400), y (0,2,1),
    z (0,200,110); the bit box must have m = (12, 2, 8), 22 bits against 36."""
    g = golden("worked_example_sec4_1.json")
    step = 2 * g["eps"]
    pts = [g["aabb_lo"], g["aabb_hi"], g["centre"]]
    q = np.array([[round(v / step) for v in p] for p in pts], np.int64)
    assert q.tolist() == [[0, 0, 0], [3000, 2, 200], [1400, 1, 110]]
    c, lo, hi, qref, m = oracle_mod.bitbox(q)
    assert c == 2
    assert qref.tolist() == [1400, 1, 110]
    assert m.tolist() == g["m"]
    assert int(m.sum()) == g["bits_per_particle"]
    assert 3 * int(m.max()) == g["bits_per_particle_one_width"]


def test_worked_example_through_full_compressor(oracle_mod):
    """Same example run through error bound, quantization, partition and layout."""
    g = golden("worked_example_sec4_1.json")
    pos = np.array([g["aabb_lo"], g["aabb_hi"], g["centre"]], np.float64)
    stream, perm = oracle_mod.compress(pos, oracle_mod.ABS, g["eps"], leaf_size=4)
    st = streamfmt.parse(stream)
    assert st.num_leaves == 1
    assert list(st.leaves[0].m) == g["m"]


def test_hand_computed_stream(oracle_mod):
    """Fig. 4 layout of the worked example, every payload bit derived by hand."""
    g = golden("hand_stream_worked_example.json")
    pos = np.array(g["positions"], np.float64)
    stream, perm = oracle_mod.compress(pos, oracle_mod.ABS, g["eb"], leaf_size=g["leaf_size"])
    st = streamfmt.parse(stream)
    assert st.n == 3 and st.dtype == 1 and st.eb_mode == 0 and st.eb == g["eb"] and st.eps == g["eb"]
    assert st.num_leaves == g["num_leaves"]
    lf = st.leaves[0]
    assert lf.particle_offset == g["leaf"]["particle_offset"]
    assert lf.word_offset == g["leaf"]["word_offset"]
    assert list(lf.q_ref) == g["leaf"]["q_ref"]
    assert list(lf.m) == g["leaf"]["m"]
    assert [list(c) for c in lf.codes] == g["codes"]
    assert st.words.tolist() == g["payload_words"]
    assert perm.tolist() == g["decoded_order"]
    assert len(stream) == 96 + 32 * 1 + 4 * 2


def _eq2_exact(R: int) -> int:
    """Eq. 2 with D/(2 eps) = R evaluated exactly: m = ceil(log2(R + 1/2) + 1),
    i.e. the least integer m with 2^(m-1) >= R + 1/2."""
    x = Fraction(2 * R + 1, 2)
    m = -10
    while Fraction(2) ** (m - 1) < x:
        m += 1
    return max(m, 0) if R > 0 else 0


def test_eq2_closed_form_small_R_exact(oracle_mod):
    for R in list(range(0, 4100)) + [2 ** k + d for k in range(12, 30) for d in (-1, 0, 1)]:
        assert oracle_mod.num_bits(R) == _eq2_exact(R), R


def test_eq2_real_valued_formula_all_R_below_2_20(oracle_mod):
    """Eq. 2 as printed, in floating point, for every R < 2^20 (log2(R + 0.5) is
    never an integer for R >= 1, so the ceiling is unambiguous)."""
    R = np.arange(0, 1 << 20, dtype=np.float64)
    m_eq2 = np.ceil(np.log2(R + 0.5) + 1.0).astype(np.int64)
    nb = oracle_mod.lib().oracle_num_bits
    got = np.fromiter((nb(r) for r in range(1 << 20)), dtype=np.int64, count=1 << 20)
    assert np.array_equal(got, m_eq2)


def test_eq2_with_real_distances(oracle_mod):
    """Eq. 2 in real units: D = max(c - pos_min, pos_max - c) and eps from the
    problem statement; positions placed exactly on the 2*eps lattice."""
    rng = np.random.default_rng(7)
    eps = 0.25  # step 0.5 is exact in binary
    for _ in range(200):
        n = int(rng.integers(2, 40))
        q = rng.integers(0, 1 << int(rng.integers(1, 18)), (n, 3))
        q[rng.integers(0, n)] = q.min(axis=0)
        pos = (q * (2 * eps)).astype(np.float64)
        c, lo, hi, qref, m = oracle_mod.bitbox(q)
        cen = pos[c]
        for d in range(3):
            D = max(cen[d] - pos[:, d].min(), pos[:, d].max() - cen[d])
            expect = 0 if D == 0 else math.ceil(math.log2(D / (2 * eps) + 0.5) + 1)
            assert m[d] == expect


# --------------------------------------------------------------------------
# Eq. 1 predictable range and Fig. 2 code mapping
# --------------------------------------------------------------------------

def _leaf_stream(oracle_mod, q_rows, eps=0.25):
    pos = np.asarray(q_rows, np.float64) * (2 * eps)
    stream, perm = oracle_mod.compress(pos, oracle_mod.ABS, eps + 1e-9, leaf_size=len(q_rows))
    return streamfmt.parse(stream), perm


def test_fig2_code_one_interval_below_centre(oracle_mod):
    """Fig. 2 caption: one interval below the prediction -> code 2^(m-1) - 2."""
    g = golden("fig2_code_below_centre.json")
    for m in g["m_values"]:
        if m > 18:
            continue  # keep the lattice small enough for an exact float64 grid here
        R = (1 << (m - 1)) - 1  # widest offset that still needs exactly m bits
        rows = [[1000 + R, 0, 0], [1000 - R, 0, 0], [1000, 0, 0], [999, 0, 0]]
        st, perm = _leaf_stream(oracle_mod, rows)
        lf = st.leaves[0]
        assert lf.m[0] == m
        assert lf.q_ref[0] == R and perm[0] == 2  # origin is the minimum, 1000 - R
        below = [c for c, p in zip(lf.codes, perm[1:]) if p == 3][0]
        assert below[0] == (1 << (m - 1)) - 2


def test_eq1_predictable_range_boundary(oracle_mod):
    """Eq. 1: with m bits the predictable half-range is 2 eps (2^(m-1) - 0.5),
    i.e. offsets up to 2^(m-1) - 1 lattice steps; one step more needs m + 1
    bits.  Codes stay within [0, 2^m - 2]."""
    for m in range(2, 16):
        R = (1 << (m - 1)) - 1
        half_range = 2 * 0.25 * ((1 << (m - 1)) - 0.5)
        assert R * 0.5 <= half_range < (R + 1) * 0.5
        st, _ = _leaf_stream(oracle_mod, [[5000, 0, 0], [5000 + R, 0, 0], [5000 - R, 0, 0]])
        assert st.leaves[0].m[0] == m
        codes = [c[0] for c in st.leaves[0].codes]
        assert min(codes) >= 0 and max(codes) <= (1 << m) - 2
        st, _ = _leaf_stream(oracle_mod, [[5000, 0, 0], [5000 + R + 1, 0, 0], [5000 - R, 0, 0]])
        # the AABB centre moves by half a step; the centre particle stays the middle one
        assert st.leaves[0].m[0] == m + 1


# --------------------------------------------------------------------------
# Sec. 3 error bound: strict invariant, special cases, nearest lattice point
# --------------------------------------------------------------------------

CASES = [
    ("uniform", np.float32, "rel", 1e-3), ("uniform", np.float32, "rel", 1e-4), ("uniform", np.float32, "abs", 0.01),
    ("cosmology", np.float32, "rel", 1e-4), ("cosmology", np.float32, "rel", 1e-3),
    ("cosmology", np.float64, "rel", 1e-6), ("fluid", np.float64, "abs", 1e-4), ("fluid", np.float32, "abs", 1e-4),
    ("fluid", np.float64, "rel", 1e-2),
]


@pytest.mark.parametrize("gen,dtype,mode,eb", CASES)
def test_error_bound_invariant(oracle_mod, gen, dtype, mode, eb):
    """Sec. 3: |p - p_hat| <= eps for every particle and axis; NRMSE <= eps / Delta_max (Sec. 5.1)."""
    pos = synth.by_name(gen, 6000, seed=3, dtype=dtype)
    m = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    stream, perm = oracle_mod.compress(pos, m, eb, leaf_size=128)
    dec = oracle_mod.decompress(stream)
    b = oracle_mod.error_bound(pos, m, eb)
    eps = eb if mode == "abs" else eb * b.delta_max
    assert b.eps == eps
    assert np.array_equal(np.sort(perm), np.arange(len(pos)))
    err = np.abs(pos[perm].astype(np.float64) - dec.astype(np.float64))
    assert int((err > eps).sum()) == 0 and err.max() <= eps
    nr = oracle_mod.nrmse(pos, dec, perm, b.delta_max)
    assert nr <= eps / b.delta_max
    assert oracle_mod.psnr(nr) >= -20 * math.log10(eps / b.delta_max)
    # the PSNR formula itself
    manual = math.sqrt(np.mean(((pos[perm].astype(np.float64) - dec) / b.delta_max) ** 2))
    assert nr == pytest.approx(manual, rel=1e-12)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_requantization_round_trip(oracle_mod, dtype):
    """Dequantized values quantize back to the same codes (codes are lossless)."""
    pos = synth.cosmology(5000, seed=11, dtype=dtype)
    stream, perm = oracle_mod.compress(pos, oracle_mod.REL, 1e-4, leaf_size=256)
    st = streamfmt.parse(stream)
    codes = streamfmt.decoded_codes(st)
    q = oracle_mod.quantize(pos, oracle_mod.REL, 1e-4)
    assert np.array_equal(codes, q[perm])
    dec = oracle_mod.decompress(stream)
    o = np.array(st.o)
    requant = np.rint((dec.astype(np.float64) - o) / st.s).astype(np.int64)
    assert np.array_equal(requant, codes)


def test_quantize_is_nearest_lattice_point(oracle_mod):
    """Brute force with exact rationals: q minimises |p - (o + s q)| over the
    integers (round half to even); cases within 2^-40 of a tie are skipped,
    since there the double-precision rule decides."""
    rng = np.random.default_rng(5)
    for dtype in (np.float32, np.float64):
        pos = (rng.uniform(-3, 50, (300, 3))).astype(dtype)
        b = oracle_mod.error_bound(pos, oracle_mod.REL, 3e-3)
        q = oracle_mod.quantize(pos, oracle_mod.REL, 3e-3)
        s = Fraction(b.s)
        for i in range(len(pos)):
            for d in range(3):
                t = (Fraction(float(pos[i, d])) - Fraction(b.o[d])) / s
                fl = math.floor(t)
                frac = t - fl
                if abs(frac - Fraction(1, 2)) < Fraction(1, 2 ** 40):
                    continue
                best = fl if frac < Fraction(1, 2) else fl + 1
                assert q[i, d] == best


def test_margin_formula(oracle_mod):
    """Reading of Sec. 3: eb' = eps - ulp_T(M2) - 4 ulp_f64(M2), M2 = 2 max(max|p|, eps)."""
    pos = np.array([[1.0, 2.0, 3.0], [100.5, 7.0, -4.0]], np.float32)
    b = oracle_mod.error_bound(pos, oracle_mod.ABS, 0.01)
    M2 = 2 * 100.5
    ulp32 = 2.0 ** (math.floor(math.log2(M2)) - 23)
    ulp64 = 2.0 ** (math.floor(math.log2(M2)) - 52)
    assert b.eb_prime == 0.01 - ulp32 - 4 * ulp64
    assert b.s == 2 * b.eb_prime
    assert b.o == (1.0, 2.0, -4.0)
    assert b.delta_max == 99.5


def test_empty_input(oracle_mod):
    pos = np.zeros((0, 3), np.float32)
    stream, perm = oracle_mod.compress(pos, oracle_mod.REL, 1e-3)
    assert len(stream) == 96
    st = streamfmt.parse(stream)
    assert st.n == 0 and st.num_leaves == 0 and st.payload_words == 0
    assert oracle_mod.decompress(stream).shape == (0, 3)


def test_single_particle(oracle_mod):
    pos = np.array([[1.5, -2.25, 1e5]], np.float64)
    stream, perm = oracle_mod.compress(pos, oracle_mod.ABS, 1e-3)
    st = streamfmt.parse(stream)
    assert st.num_leaves == 1 and st.payload_words == 0 and st.leaves[0].q_ref == (0, 0, 0)
    assert np.array_equal(oracle_mod.decompress(stream), pos)


@pytest.mark.parametrize("mode", ["abs", "rel"])
def test_identical_particles(oracle_mod, mode):
    """Delta_max = 0: every code is 0, every width is 0, reconstruction exact."""
    pos = np.tile(np.array([[3.25, 3.25, -1.0]], np.float32), (1000, 1))
    m = oracle_mod.ABS if mode == "abs" else oracle_mod.REL
    stream, perm = oracle_mod.compress(pos, m, 1e-3, leaf_size=100)
    st = streamfmt.parse(stream)
    assert st.payload_words == 0 and all(lf.m == (0, 0, 0) for lf in st.leaves)
    assert np.array_equal(oracle_mod.decompress(stream), pos)
    assert perm.tolist() == list(range(1000)) or sorted(perm.tolist()) == list(range(1000))


def test_collinear(oracle_mod):
    """Particles on a line along x: m_y = m_z = 0 in every bit box."""
    x = np.random.default_rng(2).uniform(0, 10, 2000)
    pos = np.stack([x, np.full_like(x, 4.0), np.full_like(x, -7.5)], 1).astype(np.float32)
    stream, perm = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=64)
    st = streamfmt.parse(stream)
    assert all(lf.m[1] == 0 and lf.m[2] == 0 and lf.m[0] > 0 for lf in st.leaves)
    dec = oracle_mod.decompress(stream)
    assert np.abs(dec[:, 1:] - pos[perm][:, 1:]).max() == 0


def test_rejections(oracle_mod):
    good = np.ones((10, 3), np.float32)
    for eb in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(oracle_mod.OracleError) as e:
            oracle_mod.compress(good, oracle_mod.ABS, eb)
        assert e.value.code == oracle_mod.ERR_ARG
    bad = good.copy()
    bad[3, 1] = np.nan
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.compress(bad, oracle_mod.ABS, 0.1)
    assert e.value.code == oracle_mod.ERR_NONFINITE
    bad[3, 1] = np.inf
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.compress(bad, oracle_mod.ABS, 0.1)
    assert e.value.code == oracle_mod.ERR_NONFINITE
    # eps below the float32 spacing at the data's magnitude: no lattice keeps the
    # bound, every axis is stored losslessly (Sec. 4.1, m_d > M); the bit-box
    # reduction, which needs codes, still refuses with the cause
    far = np.array([[1e6, 0, 0], [1e6 + 64, 1, 1]], np.float32)
    assert oracle_mod.error_bound(far, oracle_mod.ABS, 1e-3).raw == 7
    stream, perm = oracle_mod.compress(far, oracle_mod.ABS, 1e-3)
    assert oracle_mod.decompress(stream).tobytes() == far[perm].tobytes()
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.compress_reduced(far, oracle_mod.ABS, 1e-3)
    assert e.value.code == oracle_mod.ERR_EB_TOO_SMALL
    # codes beyond 2^30 on x only: x losslessly, y and z as codes
    wide = np.array([[0, 0, 0], [1.0, 0, 0]], np.float64)
    assert oracle_mod.error_bound(wide, oracle_mod.ABS, 1e-10).raw == 1
    stream, perm = oracle_mod.compress(wide, oracle_mod.ABS, 1e-10)
    assert oracle_mod.decompress(stream)[:, 0].tobytes() == wide[perm][:, 0].tobytes()
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.compress_reduced(wide, oracle_mod.ABS, 1e-10)
    assert e.value.code == oracle_mod.ERR_RANGE


def test_corrupt_streams_rejected(oracle_mod):
    pos = synth.uniform(3000, seed=4)
    stream, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=200)
    bad = bytearray(stream)
    bad[0] = ord("X")
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.decompress(bytes(bad))
    bad = bytearray(stream)
    bad[96 + 32 + 28] = 40  # width field above 31 in the second leaf
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.decompress(bytes(bad))
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.decompress(stream[:-4])


# --------------------------------------------------------------------------
# Sec. 4.2 storage cost: the payload is exactly term (3), word-aligned per leaf
# --------------------------------------------------------------------------

@pytest.mark.parametrize("gen", ["uniform", "cosmology", "fluid"])
def test_bit_count_identity(oracle_mod, gen):
    pos = synth.by_name(gen, 7000, seed=9)
    stream, _ = oracle_mod.compress(pos, oracle_mod.REL, 1e-3, leaf_size=300)
    st = streamfmt.parse(stream)
    bits = [sum(lf.m) * (lf.count - 1) for lf in st.leaves]
    assert st.payload_words == sum((b + 31) // 32 for b in bits)
    off = 0
    for lf, b in zip(st.leaves, bits):
        assert lf.word_offset == off
        off += (b + 31) // 32
    assert sum(lf.count for lf in st.leaves) == st.n
    assert len(stream) == 96 + 32 * st.num_leaves + 4 * st.payload_words
    # codes never use the all-ones pattern and stay within m bits
    for lf in st.leaves:
        for c in lf.codes:
            for d in range(3):
                if lf.m[d]:
                    assert 0 <= c[d] <= (1 << lf.m[d]) - 2


def test_centre_brute_force(oracle_mod):
    """Sec. 4.1: the centre is the particle closest to the AABB centre (first on ties)."""
    rng = np.random.default_rng(13)
    for _ in range(300):
        n = int(rng.integers(1, 30))
        q = rng.integers(0, int(rng.integers(1, 50)), (n, 3))
        c, lo, hi, qref, m = oracle_mod.bitbox(q)
        mid = (q.min(0) + q.max(0)) / 2.0
        dist = ((q - mid) ** 2).sum(1)
        assert c == int(np.flatnonzero(dist == dist.min())[0])
        assert lo.tolist() == q.min(0).tolist() and hi.tolist() == q.max(0).tolist()


def test_signed_zero_extrema_do_not_depend_on_order(oracle_mod):
    """Reading of Sec. 3 (origin at the minimum): -0 and +0 compare equal, so a zero
    extremum is stored as +0 whichever sign was met first."""
    a = np.array([[0.0, 1.0, 2.0], [-0.0, 3.0, 5.0], [1.0, 2.0, 3.0]], np.float32)
    b = a[[1, 0, 2]]
    sa, _ = oracle_mod.compress(a, oracle_mod.ABS, 0.01)
    sb, _ = oracle_mod.compress(b, oracle_mod.ABS, 0.01)
    assert streamfmt.parse(sa).o == streamfmt.parse(sb).o
    assert np.signbit(streamfmt.parse(sa).o[0]) == False  # noqa: E712
