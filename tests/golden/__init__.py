"""Parsers for the golden fixture files in this folder.

Each fixture is a small text file holding values printed in Kaser & Lemire,
arXiv 1402.4466 (the file's header comment names the section), or the
hand-written stream-format cases of this project.
"""
from __future__ import annotations

import os

HERE = os.path.dirname(os.path.abspath(__file__))
ALL_ONES = (1 << 64) - 1


def read_kv(name: str) -> dict:
    """key = value lines; '#' starts a comment."""
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (t.strip() for t in line.split("=", 1))
            out[k] = v
    return out


def bits_row0_first(s: str) -> int:
    """'0011' (row 0 first) -> Python int bitset (bit x = row x)."""
    return sum(1 << i for i, ch in enumerate(s) if ch == "1")


def hex_words(s: str) -> list[int]:
    return [int(t, 16) for t in s.split()]


def marker(b: int, F: int, L: int) -> int:
    return (b & 1) | (F << 1) | (L << 33)


def format_cases() -> list[tuple[int, list[int], list[int]]]:
    """(r, uncompressed words, canonical stream) triples."""
    cases = []
    with open(os.path.join(HERE, "format_cases.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            r, words, stream = (t.strip() for t in line.split("|"))
            w = []
            for t in words.split():
                w.append(0 if t == "Z" else ALL_ONES if t == "O" else int(t, 16))
            s = []
            for t in stream.split():
                if t.startswith("m("):
                    b, F, L = (int(x) for x in t[2:-1].split(","))
                    s.append(marker(b, F, L))
                else:
                    s.append(int(t, 16))
            cases.append((int(r), w, s))
    return cases
