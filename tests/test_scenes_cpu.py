"""The synthetic-input generators (CPU): determinism, mesh validity and the
batching concatenation the batched form relies on."""
import numpy as np
import pytest

import scenes


def _signed_volumes(P, tets):
    a, b, c, d = (P[tets[:, k]] for k in range(4))
    return np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) / 6.0


def test_tori_are_seeded_and_positively_oriented():
    s1 = scenes.tori_scene(nx=2, ny=1, nz=1, seed=3)
    s2 = scenes.tori_scene(nx=2, ny=1, nz=1, seed=3)
    s3 = scenes.tori_scene(nx=2, ny=1, nz=1, seed=4)
    assert np.array_equal(s1["rest_pos"], s2["rest_pos"]) and np.array_equal(s1["tets"], s2["tets"])
    assert not np.array_equal(s1["rest_pos"], s3["rest_pos"])  # the seed picks orientations / moduli
    vol = _signed_volumes(s1["rest_pos"], s1["tets"])
    assert np.all(vol > 0)
    assert np.all((s1["tet_E"] >= 1e4) & (s1["tet_E"] <= 1e6))  # log-uniform range


def test_surface_is_closed_and_consistent():
    s = scenes.tori_scene(nx=1, ny=1, nz=1)
    tris, edges = s["surf_tris"], s["surf_edges"]
    # a closed 2-manifold surface: every surface edge is shared by exactly two surface triangles
    e = np.sort(np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]]), axis=1)
    uniq, cnt = np.unique(e, axis=0, return_counts=True)
    assert np.all(cnt == 2)
    assert np.array_equal(np.unique(np.sort(edges, axis=1), axis=0), uniq)
    assert np.array_equal(np.unique(tris), np.sort(s["surf_verts"]))
    # Euler characteristic of a torus surface: V - E + F = 0
    assert len(s["surf_verts"]) - len(uniq) + len(tris) == 0


def test_concat_scenes_offsets_and_scene_ids():
    parts = [scenes.cubes_scene(n=2), scenes.gripper_scene(1200, np.random.default_rng(1)), scenes.cubes_scene(n=1)]
    b = scenes.concat_scenes(parts)
    offs = b["scene_vert_offsets"]
    assert b["n_scenes"] == 3 and len(offs) == 4 and offs[0] == 0
    assert offs[-1] == len(b["rest_pos"]) == sum(len(p["rest_pos"]) for p in parts)
    vs = b["vert_scene"]
    assert np.all(np.diff(vs) >= 0)  # non-decreasing, as the library requires
    for k, p in enumerate(parts):
        assert np.all(vs[offs[k]:offs[k + 1]] == k)
        assert np.array_equal(b["rest_pos"][offs[k]:offs[k + 1]], p["rest_pos"])
    # elements keep their own scene's vertices
    t = b["tets"]
    assert np.all(vs[t[:, 0]][:, None] == vs[t])


@pytest.mark.parametrize("name", ["cubes", "beam"])
def test_named_scenes_build(name):
    s = scenes.scene_by_name(name)
    assert len(s["rest_pos"]) > 0 and len(s["tets"]) > 0
    assert np.all(_signed_volumes(s["rest_pos"], s["tets"]) > 0)
