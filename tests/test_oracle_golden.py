"""Regression of the oracle against the digests written by tests/golden/make_golden.py."""
import json
import os

import golden_path  # noqa: F401  (adds tests/golden to sys.path)
import make_golden


def test_small_run_matches_golden_digests():
    with open(os.path.join(os.path.dirname(make_golden.__file__), "small_run.json")) as f:
        want = json.load(f)
    got = make_golden.small_run()
    assert got == want
