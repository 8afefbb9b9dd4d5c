"""The oracle's defaults are the constants the paper prints (tests/golden/paper_constants.json)."""
import json
import os

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_oracle_defaults_are_the_papers_constants():
    g = json.load(open(GOLDEN))
    o = oracle.Options()
    assert o.alpha_min == g["alpha_theta"]["value"] == 1.0 / 255.0
    assert [o.group_w, o.group_h] == g["pixel_group"]["value"]
    assert g["sigma_envelope_sq"]["value"] == 9.0
