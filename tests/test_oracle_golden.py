"""The oracle's compositor against hand-derived worked examples of Sec. 3.2
(tests/golden/entity_blend_examples.json; each example carries its citation
and derivation)."""
import json
import os

import numpy as np

from oracle import render as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "entity_blend_examples.json")
MODES = {"FULL": R.FULL, "DIRECT": R.DIRECT, "MSAA_ALL": R.MSAA_ALL, "ENTITY_ALL": R.ENTITY_ALL}


def _fragments(spec):
    out = []
    for i, f in enumerate(spec):
        if f["kind"] == "g":
            out.append(dict(kind="g", id=i, alpha=float(f["alpha"]), color=np.asarray(f["color"], np.float64)))
        else:
            out.append(dict(kind="t", id=i, alpha=float(f["alpha"]), color=np.asarray(f["color"], np.float64),
                            mask=int(f["mask"]), centre=True))
    return out


def test_golden_entity_examples():
    data = json.load(open(GOLDEN))
    assert len(data["examples"]) >= 5
    for ex in data["examples"]:
        assert ex["cite"].startswith("Sec. 3.2")
        r = R.composite(_fragments(ex["fragments"]), mode=MODES[ex["mode"]], t_eps=None,
                        t_product=bool(ex.get("t_product", False)), bg=tuple(ex.get("bg", (0.0, 0.0, 0.0))))
        exp = ex["expect"]
        assert np.allclose(r["color"], exp["color"], atol=1e-12), ex["name"]
        if "T" in exp:
            assert abs(r["T"] - exp["T"]) < 1e-12, ex["name"]
        assert np.allclose([w for _, w in r["weights"]], exp["weights"], atol=1e-12), ex["name"]
