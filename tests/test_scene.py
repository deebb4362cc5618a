"""Host checks of the seeded scene generator (inputs only)."""
import numpy as np

from paper_2501_17792_gb300 import scene as S


def test_template_shapes_and_ranges():
    t = S.make_template(1000, 4096, 3)
    assert t.means.shape == (4096, 3) and t.sh.shape == (4096, 16, 3)
    assert np.allclose(t.skin_w.sum(1), 1.0, atol=1e-6)
    assert (t.skin_w >= 0).all() and (t.skin_idx < 24).all()
    assert np.allclose(np.linalg.norm(t.quats, axis=1), 1.0, atol=1e-6)
    assert (t.opacity > 0).all() and (t.opacity < 1).all()
    assert abs(t.scales.mean() - 0.01) < 0.001
    # each Gaussian's top joint is the nearest segment owner: weights sorted
    assert (np.diff(t.skin_w, axis=1) <= 1e-7).all()
    assert 1.55 < t.means[:, 1].max() < 2.0 and t.means[:, 1].min() > -0.1


def test_seeded_and_prefix_lod():
    a = S.make_template(1001, 1024, 0)
    b = S.make_template(1001, 1024, 0)
    assert np.array_equal(a.means, b.means) and np.array_equal(a.sh, b.sh)


def test_crowd_layout_matches_the_paper_counts():
    inst = S.crowd_instances(14, 50, 70)
    assert inst.n == 3500
    assert set(np.unique(inst.template_id)) == set(range(14))
    z = inst.root[:, 2, 3]
    assert abs(z.min() - 3.0) <= 0.31
    R = inst.root[:, :, :3].astype(np.float64)
    assert np.abs(np.einsum("nij,nkj->nik", R, R) - np.eye(3)).max() < 1e-6


def test_camera_convention():
    cam = S.look_camera((0.0, 1.6, 0.0), 10.0, 1920, 1080)
    R = cam.R.astype(np.float64)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
    assert np.allclose(np.cross(R[0], R[1]), R[2], atol=1e-6)
    assert np.allclose(cam.center, [0, 1.6, 0], atol=1e-6)
    # ground points 17.7 and 9.1 degrees below the horizon: below and above
    # the optical axis of a camera pitched down 10 degrees
    for z, below in ((5.0, True), (10.0, False)):
        p = R @ (np.array([0.0, 0.0, z]) - cam.center)
        v = cam.fy * p[1] / p[2] + cam.cy
        assert (v > cam.cy) == below
