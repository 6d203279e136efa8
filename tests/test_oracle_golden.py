"""The oracle reproduces its stored outputs bit for bit on this machine."""
import json
import os

from tests.golden.make_oracle_golden import compute

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_stored_golden():
    with open(os.path.join(HERE, "golden", "oracle_8x8_seed1.json")) as f:
        want = json.load(f)
    got = compute()
    for key in want:
        assert got[key] == want[key], key
