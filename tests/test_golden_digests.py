"""The oracle and the generator give the digests recorded by
tests/golden/make_golden.py on this host too (x86_64 and aarch64 alike)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_oracle_digests_match_recorded():
    with open(os.path.join(HERE, "golden", "oracle_digests.json")) as f:
        want = json.load(f)
    got = {name: make_golden.digest(a) for name, a in make_golden.cases()}
    assert got == want
