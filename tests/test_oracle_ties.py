"""Pins of the oracle's tie alternatives (test reading of the fragment
threshold alpha >= 1/255 and the termination T < t_eps, Sec. 3.2 with the 3DGS
cut-offs it inherits): when a decision sits within rounding distance of its
threshold, composite_alternatives returns the composite with that decision
taken either way.  Checked against the blend of Eq. 1-2 written out for two-
and three-fragment pixels."""
import numpy as np

from oracle import render as R


def _g(i, alpha, color):
    return {"kind": "g", "id": i, "alpha": float(alpha), "color": np.asarray(color, np.float64), "z": 1.0 + i}


def _blend(frags):
    """Eq. 1-2 for Gaussians only: C = sum_i c_i a_i prod_{j<i} (1 - a_j)."""
    C, T = np.zeros(3), 1.0
    for f in frags:
        C += T * f["alpha"] * f["color"]
        T *= 1.0 - f["alpha"]
    return np.r_[C, T]


def _has(alts, v):
    return np.abs(alts - v).max(1).min() < 1e-15


def test_no_tie_gives_the_composite_only():
    frags = [_g(0, 0.3, (1, 0, 0)), _g(1, 0.6, (0, 1, 0))]
    alts = R.composite_alternatives(frags)
    r = R.composite(frags)
    assert alts.shape == (1, 4) and not r["tie"] and r["decisions"] == []
    assert np.allclose(alts[0], _blend(frags), rtol=0, atol=1e-15)


def test_alpha_tie_both_ways():
    a = R.ALPHA_MIN + 4e-7  # fp64 keeps it; fp32 may drop it
    frags = [_g(0, a, (0.9, 0.2, 0.1)), _g(1, 0.5, (0.1, 0.3, 0.8))]
    r = R.composite(frags)
    assert r["tie"] and r["decisions"] == [True]
    alts = R.composite_alternatives(frags)
    assert len(alts) == 2
    assert np.allclose(alts[0], _blend(frags), rtol=0, atol=1e-15)  # the fp64 outcome first
    assert _has(alts, _blend(frags[1:]))
    # just below the cut: dropped in fp64, blended in the alternative
    frags[0]["alpha"] = R.ALPHA_MIN - 4e-7
    alts = R.composite_alternatives(frags)
    assert np.allclose(alts[0], _blend(frags[1:]), rtol=0, atol=1e-15)
    assert _has(alts, _blend(frags))


def test_termination_tie_both_ways():
    # after the first fragment T = t_eps (1 + 5e-4): within 0.1% of the threshold
    t_eps = 1e-4
    a0 = 1.0 - t_eps * (1 + 5e-4)
    frags = [_g(0, a0, (0.5, 0.5, 0.5)), _g(1, 0.7, (1, 0, 1))]
    r = R.composite(frags, t_eps=t_eps)
    assert r["tie"] and r["decisions"] == [False] and r["n"] == 2
    alts = R.composite_alternatives(frags, t_eps=t_eps)
    assert len(alts) == 2
    assert _has(alts, _blend(frags))        # goes on to the second fragment
    assert _has(alts, _blend(frags[:1]))    # stops after the first


def test_two_ties_give_four_outcomes():
    a = R.ALPHA_MIN + 2e-7
    frags = [_g(0, a, (1, 0, 0)), _g(1, 0.4, (0, 1, 0)), _g(2, R.ALPHA_MIN - 3e-7, (0, 0, 1))]
    alts = R.composite_alternatives(frags)
    assert len(alts) == 4
    for keep0 in (True, False):
        for keep2 in (True, False):
            sub = [f for f, k in zip(frags, (keep0, True, keep2)) if k]
            assert _has(alts, _blend(sub))


def test_render_pixels_reports_the_alternatives():
    # one Gaussian, its opacity scaled so that its alpha at pixel (9, 8) sits
    # 3e-7 above 1/255 (alpha is linear in the opacity below the 0.99 clamp)
    from tests import helpers as H
    c = H.cam(16, 16)

    def scene(o):
        g = H.gaussians(np.array([[0.0, 0.0, 0.0]]), scales=np.full((1, 3), 0.05, np.float32),
                        opac=np.array([o], np.float32), colors=np.array([[0.3, 0.6, 0.9]]))
        return H.scene(g, [], c)

    a = R.Frame(scene(0.5), 0).fragments_at(9, 8)[0]["alpha"]
    o = np.float32(0.5 * (R.ALPHA_MIN + 3e-7) / a)
    sc = scene(o)
    a2 = R.Frame(sc, 0).fragments_at(9, 8)[0]["alpha"]
    assert 0 < a2 - R.ALPHA_MIN < 1e-6
    alts = {}
    pix = np.array([[x, y] for y in range(16) for x in range(16)])
    rgb, T, tie, _ = R.render_pixels(sc, pix, alts=alts)
    k = 8 * 16 + 9
    assert tie[k] and set(alts) == set(np.nonzero(tie)[0].tolist())
    for j, v in alts.items():
        assert np.allclose(v[0], np.r_[rgb[j], T[j]], rtol=0, atol=1e-15)
    assert _has(alts[k], np.r_[0.0, 0.0, 0.0, 1.0])  # the fragment dropped: nothing blends
    img = R.render_image(sc)
    assert set(img["alts"]) == set(np.nonzero(img["tie"].reshape(-1))[0].tolist())
    assert np.abs(img["alts"][k] - alts[k]).max() < 1e-15
