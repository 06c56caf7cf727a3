"""CPU tests of the seeded scene generators' own properties (inputs, not the method)."""
import numpy as np

from paper_2208_10009_gb300 import scenes


def test_random_clutter_is_seeded_and_general():
    a = scenes.random_clutter(scenes.SEED_BASE + 10)
    b = scenes.random_clutter(scenes.SEED_BASE + 10)
    for x, y in zip((a[0].verts, a[0].tris, a[0].tri_face, a[1], a[2]), (b[0].verts, b[0].tris, b[0].tri_face, b[1], b[2])):
        assert np.array_equal(x, y)
    sc, tx, rx = a
    assert sc.nf == 6 + 20 * 6 and sc.nt == 6 * 2 * 4 + 20 * 6 * 2
    v = sc.verts[sc.tris]
    n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
    assert np.linalg.norm(n, axis=1).min() > 0.01
    # the box sides (faces 6..) lie on no coordinate plane
    nn = n / np.linalg.norm(n, axis=1)[:, None]
    boxes = sc.tri_face >= 6
    assert np.abs(nn[boxes]).max(axis=1).max() < 1 - 1e-6
    # Tx and Rx inside the room, outside every box: a point inside a box's side planes on all
    # three axes would sit between each pair of opposite sides
    pts = np.concatenate([tx, rx])
    assert np.all(pts > 0) and np.all(pts < [20.0, 16.0, 6.0])
    for f in range(6, sc.nf, 6):
        for p in pts:
            inside = True
            for side in range(3):
                # a box's sides come as (x-, y-, z-, x+, y+, z+)
                t1 = sc.tris[sc.tri_face == f + side][0]
                t2 = sc.tris[sc.tri_face == f + side + 3][0]
                n1 = np.cross(sc.verts[t1[1]] - sc.verts[t1[0]], sc.verts[t1[2]] - sc.verts[t1[0]])
                s1 = np.dot(p - sc.verts[t1[0]], n1)
                s2 = np.dot(p - sc.verts[t2[0]], n1)
                inside &= s1 * s2 < 0
            assert not inside
