"""Parity protocol between the CUDA path and the CPU oracle (test helper).

The protocol itself lives in ``oracle.parity`` so that the tests, ``smoke()`` and the
benchmark's oracle leg apply the same rules; this module re-exports it for the tests.
"""
from oracle.parity import (ADJ_FACTOR, CANCEL_CAP, EPS64, SEL_RTOL, VAL_RTOL,  # noqa: F401
                           cancellation_bound, check_location, check_sample, rel_err,
                           tally_summary)
