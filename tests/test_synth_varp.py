"""Input helpers of the variable-degree cases (``synth.meshes``): element
frames rotated by ``reorient`` describe the same elements and boundaries, and
``sponge_degrees`` / ``checker_degrees`` give the degrees asked for."""
import numpy as np
import pytest

from synth import meshes as M


def _face_centres(mesh):
    faces = M.face_corners(mesh.dim)
    X = mesh.xyz[mesh.elem_vert]
    return np.stack([X[:, list(f)].mean(axis=1) for f in faces], axis=1)   # (E, 2d, dim)


@pytest.mark.parametrize("dim", [2, 3])
def test_reorient_keeps_elements_orientation_and_boundaries(dim):
    n = (5, 4) if dim == 2 else (3, 3, 2)
    m = M.periodic_box(dim, n, (0.0,) * dim, (1.0,) * dim, jitter=0.2)
    m.face_tag = m.face_tag.copy()
    m.face_tag[m.face_tag == 1] = M.TAG_FARFIELD          # distinct tags to track
    m.face_tag[0, 0] = M.TAG_WALL
    r = M.reorient(m, seed=4)
    # same corner set per element
    assert all(set(a) == set(b) for a, b in zip(m.elem_vert, r.elem_vert))
    # a rotation, not a reflection: the signed volume keeps its sign
    def signed(mesh):
        X = mesh.xyz[mesh.elem_vert]
        a, b = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
        if dim == 2:
            return a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
        return np.einsum("ej,ej->e", np.cross(a, b), X[:, 4] - X[:, 0])
    assert np.all(np.sign(signed(r)) == np.sign(signed(m)))
    # every face keeps its tag: match faces by their centres
    cm, cr = _face_centres(m), _face_centres(r)
    for e in range(m.n_elem):
        for f in range(2 * dim):
            g = int(np.argmin(np.linalg.norm(cr[e] - cm[e, f], axis=1)))
            assert np.allclose(cr[e, g], cm[e, f]) and r.face_tag[e, g] == m.face_tag[e, f]
    # the rotations used are all the proper ones
    assert len(M._rotations(dim)) == (4 if dim == 2 else 24)
    assert all(round(np.linalg.det(R)) == 1 for R in M._rotations(dim))


def test_sponge_and_checker_degrees():
    m = M.naca_omesh(0.02, 0.4, 0.12, 2.0, 400)
    ep = M.sponge_degrees(m, (0.5, 0.0), (1.0, 3.0, 6.0), (3, 2, 1, 0))
    r = np.linalg.norm(M.element_centroids(m) - np.array([0.5, 0.0]), axis=1)
    order = np.argsort(r)
    assert np.all(np.diff(ep[order]) <= 0)                 # never higher further out
    assert ep[r < 1.0].min() == 3 and ep[r >= 6.0].max() == 0 and np.any(r >= 6.0)
    c = M.checker_degrees(m, (0, 1, 2, 3), seed=1)
    assert set(np.unique(c)) == {0, 1, 2, 3} and c.dtype == np.int32
    alt = M.checker_degrees(m, (2, 3))
    assert np.array_equal(alt[:4], [2, 3, 2, 3])
