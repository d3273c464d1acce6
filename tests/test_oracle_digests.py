"""The oracle's integer outputs on the `tiny` parameter set (keys, an
encryption, plain and hoisted rotations, a product with relinearisation, a
rescale) against the digests that tests/golden/make_oracle_digests.py wrote
from the oracle alone: any change to the oracle's arithmetic shows here, and
regenerating the digests takes a commit that names the passage behind it.
These guard the oracle against drift; the pins against the paper and the
mathematics are the other test_oracle_* files."""
import importlib.util
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_outputs_match_the_stored_digests():
    path = os.path.join(HERE, "golden", "make_oracle_digests.py")
    spec = importlib.util.spec_from_file_location("make_oracle_digests", path)
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(os.path.join(HERE, "golden", "oracle_tiny_digests.json")) as f:
        want = json.load(f)
    got = mk.compute()
    assert sorted(got) == sorted(want)
    assert [k for k in want if got[k] != want[k]] == []
