"""Readers for the cited values in tests/golden/*.txt."""
import os
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))


def rows(name):
    out = []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                out.append(line.split())
    return out


def table1_coarse_sizes():
    return {(m, int(k)): int(v) for m, k, v in rows("table1_coarse_sizes.txt")}


def table1_iterations():
    return {(m, int(k)): int(v) for m, k, v in rows("table1_iterations.txt")}


def fig1():
    return {k: float(Fraction(v)) for k, v in rows("fig1_weight.txt")}
