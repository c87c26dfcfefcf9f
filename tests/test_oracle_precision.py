"""Pins of the oracle's 16-bit storage rounding (oracle/precision.py).

Each check compares against something other than the function itself:
numpy's binary16 conversion, the round-half-even on binary32 bit patterns
for bfloat16, and hand-worked ties, subnormals and overflow.
"""
import numpy as np

from oracle.precision import (QuantisedTables, bits16, f16_exp2, quantise, round_bf16,
                              round_f16, table_exp2)


def _wide_sample(rng, n):
    """Values over many binades, both signs, plus subnormal-range and huge ones."""
    e = rng.uniform(-30, 20, n)
    return rng.choice([-1.0, 1.0], n) * rng.uniform(1.0, 2.0, n) * np.exp2(e)


def test_f16_matches_numpy_binary16():
    rng = np.random.default_rng(1)
    x = np.concatenate([_wide_sample(rng, 200000), rng.normal(size=50000),
                        np.array([0.0, -0.0, 65504.0, 65519.99, 65520.0, 1e6, 2.0**-24,
                                  2.0**-25, 3 * 2.0**-26, 2.0**-14 - 2.0**-25])])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    got = round_f16(x)
    assert np.array_equal(got, ref, equal_nan=True)


def test_bf16_matches_binary32_bit_rounding():
    rng = np.random.default_rng(2)
    f = _wide_sample(rng, 200000).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    ref = (((u + 0x7FFF + lsb) >> 16) << 16).astype(np.uint32).view(np.float32)
    got = round_bf16(f.astype(np.float64))
    assert np.array_equal(got, ref.astype(np.float64))


def test_hand_worked_ties_and_edges():
    # bfloat16 has 7 fraction bits: ulp(1) = 2^-7
    assert round_bf16(1 + 2.0**-8) == 1.0                       # tie -> even (1.0)
    assert round_bf16(1 + 3 * 2.0**-8) == 1 + 2.0**-6           # tie -> even (..10)
    assert round_bf16(1 + 2.0**-8 + 2.0**-30) == 1 + 2.0**-7    # above the tie
    assert round_bf16(-(1 + 2.0**-8)) == -1.0
    # float16: 10 fraction bits, subnormal quantum 2^-24, max 65504
    assert round_f16(1 + 2.0**-11) == 1.0
    assert round_f16(1 + 3 * 2.0**-11) == 1 + 2.0**-9
    assert round_f16(2.0**-25) == 0.0                           # tie between 0 and 2^-24 -> 0
    assert round_f16(3 * 2.0**-25) == 2.0**-23                  # tie -> even (2 quanta)
    assert round_f16(65519.0) == 65504.0
    assert np.isinf(round_f16(65520.0))                         # tie with 2^16 -> overflow
    assert round_f16(0.1) == np.float64(np.float16(0.1))


def test_f16_exponent_window():
    for peak in [0.2, 0.25, 0.3, 1.0, 1.5, 3e-3, 7.9]:
        e = f16_exp2(peak)
        assert 2.0**14 <= peak * 2.0**e < 2.0**15


def test_quantise_scales_exactly_and_bits_roundtrip():
    rng = np.random.default_rng(3)
    z = (rng.normal(size=1000) + 1j * rng.normal(size=1000)) * 1e-3
    for kind in ("bf16", "f16"):
        e = 0 if kind == "bf16" else f16_exp2(np.abs(z).max())
        q = quantise(z, kind, e)
        # scaled values are representable: rounding them again changes nothing
        rr = round_bf16 if kind == "bf16" else round_f16
        assert np.array_equal(rr(np.ldexp(q.real, e)), np.ldexp(q.real, e))
        assert np.array_equal(rr(np.ldexp(q.imag, e)), np.ldexp(q.imag, e))
        # relative error within half an ulp of the format
        u = 2.0**-8 if kind == "bf16" else 2.0**-11
        assert np.all(np.abs(q.real - z.real) <= u * np.abs(z.real) + 1e-300)
        b = bits16(np.ldexp(q.real, e), kind)
        if kind == "f16":
            assert np.array_equal(b.view(np.float16).astype(np.float64), np.ldexp(q.real, e))
        else:
            back = (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
            assert np.array_equal(back, np.ldexp(q.real, e))


def test_quantised_tables_keep_shape_and_peak_window():
    from oracle.wkernel import KernelTables, Params
    prm = Params(grid_n=64, cell_rad=2e-3, support_min=7, support_max=11, oversample=4,
                 n_wplanes=3, w_max_lambda=50.0, npol=1)
    kt = KernelTables(prm)
    for kind in ("bf16", "f16"):
        qt = QuantisedTables(kt, kind)
        assert [t.shape for t in qt.planes] == [t.shape for t in kt.planes]
        e = table_exp2(kt, kind)
        peak = max(np.abs(t).max() for t in kt.planes)
        if kind == "f16":
            assert 2.0**14 <= peak * 2.0**e < 2.0**15
        flat, offs = qt.flat()
        assert flat.shape[0] == offs[-1]
        rel = np.abs(flat - kt.flat()[0]).max() / peak
        assert rel <= (2.0**-8 if kind == "bf16" else 2.0**-11)
