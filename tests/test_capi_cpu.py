"""CPU-only checks of the C-ABI library: it builds and loads, exports every
function include/thr.h declares, and its host codec (encoder, validator)
agrees with the oracle's independent codec.  No GPU compute is called."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import oracle_pins
import paper_1402_4466_gb300 as thr
import synth
from golden import format_cases

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "thr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_library_loads_and_exports_every_declared_symbol():
    lib = thr.load()
    names = declared_functions()
    assert set(names) == set(thr.ABI_SYMBOLS), names
    for name in names:
        assert getattr(lib, name) is not None
        # also resolvable through the dynamic loader directly
        ctypes.cast(getattr(lib, name), ctypes.c_void_p)


def test_encoder_matches_format_cases():
    for r, w, s in format_cases():
        got = thr.thr_rle_encode(np.array(w, dtype=np.uint64), r)
        assert got.tolist() == s, (r, w)
        assert thr.thr_rle_validate(np.array(s, dtype=np.uint64), r) == thr.THR_OK


def test_validator_rejects_malformed():
    for r, s in oracle_pins.bad_streams():
        st = thr.thr_rle_validate(np.array(s, dtype=np.uint64), r)
        if r == 0:
            assert st in (thr.THR_E_FORMAT, thr.THR_OK) and st == thr.THR_E_FORMAT
        else:
            assert st == thr.THR_E_FORMAT, (r, s)


def test_encoder_matches_oracle_encoder_random():
    rng = np.random.default_rng(21)
    for _ in range(80):
        r = int(rng.choice([1, 63, 64, 65, 127, 1000, 4096, 4097, 70000]))
        x = oracle_pins.random_bitsets(rng, 1, r)[0]
        w = oracle_pins.int_to_words(x, r)
        a = thr.thr_rle_encode(w, r)
        b = oracle.encode(w, r)
        assert np.array_equal(a, b)
        assert thr.thr_rle_validate(a, r) == thr.THR_OK


def test_encoder_matches_oracle_on_generated_bitmaps():
    r = (1 << 18) + 37
    words, _ = synth.many_criteria(2, 12, r)
    for w in words:
        assert np.array_equal(thr.thr_rle_encode(w, r), oracle.encode(w, r))


def test_encode_rejects_bits_past_r():
    with pytest.raises(thr.ThrError) as e:
        thr.thr_rle_encode(np.array([1 << 20], dtype=np.uint64), 10)
    assert e.value.status == thr.THR_E_INVAL


def test_build_rejects_bad_input_before_gpu_work():
    lib = thr.load()
    h = ctypes.c_void_p(0)
    w = np.array([oracle_pins.marker(0, 1, 0), oracle_pins.marker(0, 1, 0)], dtype=np.uint64)
    offs = np.array([0, 2], dtype=np.uint64)
    st = lib.idx_build_rle(ctypes.c_void_p(w.ctypes.data), ctypes.c_void_p(offs.ctypes.data),
                           1, 128, None, ctypes.byref(h))
    assert st == thr.THR_E_FORMAT and h.value is None
    assert "fill run split" in thr.thr_last_error()
    st = lib.idx_build_rle(ctypes.c_void_p(w.ctypes.data), ctypes.c_void_p(offs.ctypes.data),
                           1, 0, None, ctypes.byref(h))
    assert st == thr.THR_E_INVAL
    st = lib.idx_build_rle(ctypes.c_void_p(w.ctypes.data), ctypes.c_void_p(offs.ctypes.data),
                           0, 128, None, ctypes.byref(h))
    assert st == thr.THR_E_INVAL


def test_query_rejects_null_index():
    lib = thr.load()
    ids = np.zeros(1, dtype=np.uint32)
    n = ctypes.c_uint64(0)
    st = lib.thr_query(None, ctypes.c_void_p(ids.ctypes.data), 1, 1, None, 0,
                       ctypes.byref(n), 0, None)
    assert st == thr.THR_E_INVAL


def test_encode_rows_matches_word_encoders():
    """The row-list encoder gives the same canonical stream as the library's
    and the oracle's word encoders (sparse, dense, runs with full words,
    ragged last word, empty and full bitmaps)."""
    import oracle
    rng = np.random.default_rng(40)
    cases = []
    for r in (1, 63, 64, 65, 1000, 4096 + 17, 200_003):
        cases.append((np.zeros(0, np.int64), r))
        cases.append((np.arange(r), r))
        for p in (1e-4, 0.01, 0.3, 0.9):
            cases.append((synth.bernoulli_rows(rng, r, p), r))
        w = synth.clustered(3, r % 97, r, 0.2)
        cases.append((np.nonzero(synth.words_to_bits(w, r))[0], r))
    for rows, r in cases:
        words = synth.rows_to_words(rows, r)
        got = thr.thr_rle_encode_rows(rows, r)
        assert np.array_equal(got, thr.thr_rle_encode(words, r)), r
        assert np.array_equal(got, oracle.encode(words, r)), r
    # repeated rows are one row; unsorted rows are rejected
    assert np.array_equal(thr.thr_rle_encode_rows([5, 5, 9], 100),
                          thr.thr_rle_encode_rows([5, 9], 100))
    with pytest.raises(thr.ThrError):
        thr.thr_rle_encode_rows([9, 5], 100)
    with pytest.raises(thr.ThrError):
        thr.thr_rle_encode_rows([100], 100)


def test_rule_model_coefficients_round_trip():
    """The rule chooser's 12 coefficients (host state): set, read back, and
    the shipped ones restored; no GPU involved."""
    from paper_1402_4466_gb300 import selector_weights
    shipped = selector_weights.load()["rule_coefficients"]
    before = thr.rule_model()
    try:
        c = np.arange(1, 13, dtype=np.float64) * 0.5
        assert np.array_equal(thr.rule_model(c), c)
        assert np.array_equal(thr.rule_model(), c)
        assert np.array_equal(thr.rule_model(shipped), np.asarray(shipped, np.float64))
    finally:
        thr.rule_model(before)


def test_shipped_selector_weights_fit_the_library():
    """The shipped model has the library's parameter count and a 12-term rule."""
    from paper_1402_4466_gb300 import selector_weights
    d = selector_weights.load()
    assert len(d["params"]) == thr.SEL_PARAMS
    assert len(d["mean"]) == 16 and len(d["istd"]) == 16
    assert len(d["rule_coefficients"]) == 12
    assert all(np.isfinite(d["params"])) and all(v > 0 for v in d["istd"])


def test_binding_constants_match_the_header():
    """Every flag, status and size constant of include/thr.h has the same
    value in the Python binding (the binding restates them for ctypes)."""
    text = open(HEADER).read()
    defines = {m.group(1): int(m.group(2), 0) for m in
               re.finditer(r"^#define (THR_[A-Z0-9_]+) (0x[0-9A-Fa-f]+|[0-9]+)u?", text, flags=re.M)}
    enums = {m.group(1): int(m.group(2)) for m in
             re.finditer(r"^\s*(THR_(?:OK|E_[A-Z]+)) = ([0-9]+)", text, flags=re.M)}
    assert len(defines) >= 18 and len(enums) == 8
    sel = {"THR_SEL_FEATURES": thr.SEL_FEATURES, "THR_SEL_VARIANTS": thr.SEL_VARIANTS,
           "THR_SEL_PARAMS": thr.SEL_PARAMS}
    for name, value in {**defines, **enums}.items():
        if name in sel:
            assert sel[name] == value, name
        else:
            assert getattr(thr, name) == value, name
