"""Counts that the GPU parity tests report beside their pass/fail bars: rays
checked, rays in the degenerate band, band rays whose cell sequence differs
from the oracle's, and the largest image error inside and outside the band.
tests/conftest.py prints them at the end of the run."""

RECORDS = []


def record(name, **values):
    RECORDS.append((name, values))


def format_records():
    lines = []
    for name, v in RECORDS:
        parts = []
        for k, x in v.items():
            parts.append(f"{k}={x:.3g}" if isinstance(x, float) else f"{k}={x}")
        lines.append(f"{name}: " + ", ".join(parts))
    return lines
