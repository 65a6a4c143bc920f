"""Textured meshes (c_i sampled from a texture at the perspective-correct uv)
on the GPU against the oracle."""
import numpy as np
import pytest
import torch

from oracle import render as R
from paper_2601_19233_gb300 import scenes as S
from tests import helpers as H
from tests.test_gpu_render import check_image, check_lists, ctx, gpu_render  # noqa: F401

pytestmark = pytest.mark.gpu


def _textured_scene(seed=41, null_vcolor=False):
    rng = np.random.default_rng(seed)
    sc = S.small_scene(seed, 75, 53, 400, mesh_subdiv=2, transparent_frac=0.4)
    m = sc.meshes[0]
    # spherical uv of the sphere's vertices, a random 37 x 23 texture
    d = m.verts / np.linalg.norm(m.verts, axis=1, keepdims=True)
    uv = np.stack([0.5 + np.arctan2(d[:, 0], d[:, 2]) / (2 * np.pi), 0.5 - np.arcsin(d[:, 1]) / np.pi], 1)
    tex = rng.uniform(0, 1, size=(23, 37, 3)).astype(np.float32)
    sc.meshes[0] = S.Mesh(m.verts, m.faces, None if null_vcolor else m.vcolor, m.valpha, m.falpha,
                          uv=uv.astype(np.float32), texture=tex)
    # plus an untextured quad behind, so both kinds share the lists
    sc.meshes.append(H.screen_quad(sc.cameras[0], 0.9, 0.7, (0.3, 0.6, 0.2)))
    return sc


@pytest.mark.parametrize("tile", [8, 16])
def test_textured_mesh_matches_oracle(ctx, tile):
    sc = _textured_scene(null_vcolor=(tile == 8))
    out, fr = gpu_render(ctx, sc, tile=tile)
    check_lists(sc, fr, tile)
    check_image(sc, out)


def test_textured_mesh_validation_and_no_backward(ctx):
    from paper_2601_19233_gb300 import umgs
    sc = _textured_scene(43)
    g = umgs.gaussians_to_device(sc.gaussians)
    ms = [umgs.mesh_to_device(m) for m in sc.meshes]
    bad = umgs.mesh_to_device(sc.meshes[0])
    bad.texture = None  # uv without a texture
    with pytest.raises(umgs.UmgsError):
        umgs.render(ctx, g, [bad], sc.cameras, umgs.render_opts(16))
    fr = umgs.Frame(ctx)
    out = umgs.render(ctx, g, ms, sc.cameras, umgs.render_opts(16, save=True), frame=fr)
    with pytest.raises(umgs.UmgsError) as e:
        umgs.render_backward(ctx, fr, g, ms, torch.ones_like(out))
    assert e.value.status == 6  # NOT_IMPLEMENTED
