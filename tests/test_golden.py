"""The oracle's recorded result on the 1-ligand configuration is reproduced
on this host (portability of generator + oracle; the file is written by
tests/golden/make_golden.py, which calls only the generator and the oracle)."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tiny_oracle_golden():
    from tests.golden.make_golden import compute
    want = json.load(open(os.path.join(HERE, "golden", "tiny_oracle.json")))
    got = compute()
    assert got["top_starts"] == want["top_starts"]
    assert got["top_tors"] == want["top_tors"]
    np.testing.assert_allclose(got["top_scores"], want["top_scores"], rtol=1e-12)
    assert got["maps_sum"] == want["maps_sum"] and got["xyz_sum"] == want["xyz_sum"]
    np.testing.assert_allclose(got["sum_all_start_scores"], want["sum_all_start_scores"], rtol=1e-12)
