"""Pins of the RGB-D rendering oracle (oracle/render.py): poses whose result
is known without the oracle's arithmetic."""
import numpy as np

from oracle import render as RD


def frames(H=24, W=32, seed=0, holes=True):
    rng = np.random.default_rng(seed)
    depth = rng.integers(500, 4000, (H, W)).astype(np.uint16)
    if holes:
        depth[rng.random((H, W)) < 0.1] = 0
    rgb = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    return rgb, depth


def test_identity_pose_reproduces_the_frame():
    rgb, depth = frames()
    K = (500.0, 510.0, 15.5, 11.5)
    out_rgb, out_d = RD.render(rgb, depth, K, np.eye(3), (0, 0, 0), K, depth.shape)
    np.testing.assert_array_equal(out_d, depth)
    valid = depth > 0
    np.testing.assert_array_equal(out_rgb[valid], rgb[valid])
    assert not out_rgb[~valid].any()


def test_rotation_by_pi_about_the_axis_mirrors_the_frame():
    rgb, depth = frames(seed=1)
    H, W = depth.shape
    K = (400.0, 400.0, (W - 1) / 2, (H - 1) / 2)
    R = np.diag([-1.0, -1.0, 1.0])
    out_rgb, out_d = RD.render(rgb, depth, K, R, (0, 0, 0), K, depth.shape)
    np.testing.assert_array_equal(out_d, depth[::-1, ::-1])
    valid = depth[::-1, ::-1] > 0
    np.testing.assert_array_equal(out_rgb[valid], rgb[::-1, ::-1][valid])


def test_translation_along_the_axis_adds_depth_at_the_principal_point():
    rgb, depth = frames(holes=False, seed=2)
    H, W = depth.shape
    depth[:] = 1000
    K = (300.0, 300.0, 16.0, 12.0)
    _, out_d = RD.render(rgb, depth, K, np.eye(3), (0, 0, 250.0), K, depth.shape)
    assert out_d[12, 16] == 1250  # the principal ray keeps its pixel
    assert out_d.max() == 1250 and (out_d[out_d > 0] == 1250).all()
    # farther away the plane covers fewer pixels (perspective)
    assert 0 < (out_d > 0).sum() < H * W


def test_nearest_point_wins_and_ties_go_to_the_lower_index():
    depth = np.zeros((1, 4), np.uint16)
    depth[0, 1] = 2000
    depth[0, 2] = 1000
    rgb = np.zeros((1, 4, 3), np.uint8)
    rgb[0, 1] = (10, 20, 30)
    rgb[0, 2] = (40, 50, 60)
    K = (100.0, 100.0, 1.5, 0.0)
    # splat radius 1 around each point's own pixel: pixels 1 and 2 are covered by both
    out_rgb, out_d = RD.render(rgb, depth, K, np.eye(3), (0, 0, 0), K, (1, 4), splat=1)
    assert list(out_d[0]) == [2000, 1000, 1000, 1000]
    assert tuple(out_rgb[0, 1]) == (40, 50, 60)
    depth[0, 2] = 2000  # equal depth: the lower point index (pixel 1) wins where both land
    out_rgb, out_d = RD.render(rgb, depth, K, np.eye(3), (0, 0, 0), K, (1, 4), splat=1)
    assert tuple(out_rgb[0, 2]) == (10, 20, 30) and tuple(out_rgb[0, 3]) == (40, 50, 60)


def test_rgb_sampled_nearest_when_sizes_differ():
    rgb = np.zeros((4, 8, 3), np.uint8)
    rgb[..., 0] = np.arange(8)[None, :] * 10
    depth = np.full((2, 4), 1000, np.uint16)
    K = (100.0, 100.0, 1.5, 0.5)
    out_rgb, _ = RD.render(rgb, depth, K, np.eye(3), (0, 0, 0), K, (2, 4))
    assert list(out_rgb[0, :, 0]) == [0, 20, 40, 60]  # depth column i -> rgb column 2i
