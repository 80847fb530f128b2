"""Plant plausible mistakes in copies of oracle.c (on the CPU) and check that
the pins catch every one of them: a wrong comparison, a wrong bit order, a
wrong marker field, a dropped multiplicity, a dropped input, a wrong fill
value, a dropped canonical rule, and so on."""
import os

import pytest

import oracle
import oracle_pins

MUTANTS = [
    ("threshold > instead of >=", "count[x] >= T", "count[x] > T"),
    ("bit order reversed", "words[x / 64] |= 1ull << (x % 64);",
     "words[x / 64] |= 1ull << (63 - x % 64);"),
    ("literal count field at bit 32", "L = mw >> 33;", "L = mw >> 32;"),
    ("fill length field at bit 2", "F = (mw >> 1) & 0xFFFFFFFFull;",
     "F = (mw >> 2) & 0xFFFFFFFFull;"),
    ("fill bit read from bit 63", "b = mw & 1;", "b = (mw >> 63) & 1;"),
    ("encoder packs L at bit 32", "return (b & 1) | (F << 1) | (L << 33);",
     "return (b & 1) | (F << 1) | (L << 32);"),
    ("encoder fill bit inverted", "b = (v == ~0ull);", "b = (v == 0);"),
    ("counter set instead of incremented", "count[rows[k]]++;",
     "count[rows[k]] = 1;"),
    ("wrong input id", "uint64_t b = ids[q], nr = 0;",
     "uint64_t b = ids[q > 0 ? q - 1 : 0], nr = 0;"),
    ("all-ones word treated as literal", "return v == 0 || v == ~0ull;",
     "return v == 0;"),
    ("ones fill one row short",
     "x < (covered + F) * 64; x++)", "x < (covered + F) * 64 - 1; x++)"),
    ("fill runs split early", "words[i] == v && F < ORC_FMAX",
     "words[i] == v && F < 2"),
    ("ragged-word rule dropped",
     "if (b && (r % 64) != 0 && covered + F == W)", "if (0)"),
    ("fill-maximality rule inverted", "prevb == b && prevF != ORC_FMAX",
     "prevb != b && prevF != ORC_FMAX"),
    ("last row dropped", "if (count[x] >= T) words",
     "if (count[x] >= T && x + 1 < r) words"),
    ("row range ends one word early",
     "w1 = W * (uint64_t)(p + 1) / parts;", "w1 = W * (uint64_t)(p + 1) / parts - 1;"),
    ("ones fill of a range stops one word short",
     "uint64_t e = covered + F < w1 ? covered + F : w1;",
     "uint64_t e = covered + F < w1 ? covered + F : w1 - 1;"),
    ("literals of a range's first word skipped",
     "if (covered >= w0 && covered < w1) {", "if (covered > w0 && covered < w1) {"),
    ("literal copied from the wrong slot",
     "if (n < cap && out) out[n] = words[lit0 + k];",
     "if (n < cap && out) out[n] = words[lit0];"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_kill_mutant(tmp_path, name, old, new):
    src = open(oracle.SRC).read()
    assert old in src, f"mutation site for '{name}' no longer in oracle.c"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(old, new))
    so = oracle.compile_c(str(c), str(tmp_path / "libmutant.so"))
    o = oracle.load(so)
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(o)
        except Exception:
            return  # killed
    pytest.fail(f"mutant '{name}' survived every pin")
