"""Loader of the fixtures under tests/golden/.

Each fixture holds values the paper prints, with its citation in the header
lines (starting with '#').  Data lines are whitespace-separated numbers; a
file of "key value" lines also reads as a dict.  Nothing here computes
anything.
"""
from __future__ import annotations

import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name: str) -> list[list[str]]:
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                out.append(line.split())
    return out


def _num(tok: str):
    for conv in (int, float):
        try:
            return conv(tok)
        except ValueError:
            pass
    return tok  # a key


def rows(name: str) -> list[list]:
    """Data lines as lists of numbers (int where the token is an integer;
    keys stay strings)."""
    return [[_num(t) for t in r] for r in _lines(name)]


def table(name: str) -> dict:
    """A fixture of "key value" lines as a dict."""
    return {r[0]: _num(r[1]) for r in _lines(name)}


def citation(name: str) -> str:
    """The header comment of a fixture (its source)."""
    with open(os.path.join(GOLDEN, name)) as f:
        return " ".join(line[1:].strip() for line in f if line.startswith("#"))
