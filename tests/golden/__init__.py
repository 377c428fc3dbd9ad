"""Text fixtures of values printed in the paper, each file citing its passage."""

import os

HERE = os.path.dirname(os.path.abspath(__file__))


def read_fixture(name):
    """Parse ``key value...`` lines (``#`` comments) into a dict of lists of strings;
    repeated keys accumulate."""
    out = {}
    with open(os.path.join(HERE, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append(vals)
    return out
