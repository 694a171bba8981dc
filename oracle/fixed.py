"""ORACLE - test infrastructure, not part of the product.

Reference arithmetic of the 128-bit fixed-point BC form (units 2^-64, an
unsigned integer as (low, high) uint64 words) in plain Python integers, for
checking the library's exact reduction of partial BC vectors: conversion of
an FP64 value to the nearest multiple of 2^-64, exact sums, and the correctly
rounded FP64 value of a sum (CPython's int-to-float division rounds to
nearest, ties to even).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

MASK64 = (1 << 64) - 1


def to_int(f) -> list:
    """Python integers of an [n, 2] (or [2n]) uint64 fixed-point vector."""
    a = np.asarray(f).view(np.uint64).reshape(-1, 2)
    return [(int(h) << 64) | int(lo) for lo, h in a]


def from_int(values) -> np.ndarray:
    """[n, 2] uint64 words of non-negative integers below 2^128."""
    out = np.zeros((len(values), 2), np.uint64)
    for i, v in enumerate(values):
        if v < 0 or v >> 128:
            raise ValueError("value outside [0, 2^128)")
        out[i, 0] = v & MASK64
        out[i, 1] = v >> 64
    return out


def from_double(x) -> np.ndarray:
    """Each non-negative FP64 value as the nearest multiple of 2^-64 (ties
    to even); exact whenever the value's last bit is worth at least 2^-64."""
    vals = []
    for d in np.asarray(x, np.float64):
        q = Fraction(float(d)) * (1 << 64)
        fl = q.numerator // q.denominator
        rem = q - fl
        if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl & 1):
            fl += 1
        vals.append(fl)
    return from_int(vals)


def sum_parts(parts) -> list:
    """Exact sums (Python integers) of several fixed-point vectors."""
    ints = [to_int(p) for p in parts]
    return [sum(col) for col in zip(*ints)]


def to_double(values) -> np.ndarray:
    """Correctly rounded FP64 of integers in units of 2^-64."""
    return np.array([v / (1 << 64) for v in values], np.float64)
