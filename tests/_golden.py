"""Readers for the cited text fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for raw in f:
            s = raw.strip()
            if s and not s.startswith("#"):
                yield s


def fields(name):
    """Rows split on '|' into lists of whitespace-separated tokens."""
    for s in lines(name):
        yield [part.split() for part in s.split("|")]
