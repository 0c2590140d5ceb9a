"""The plane-IoU helper of the evaluation: known polygon pairs."""
import bench


def test_convex_iou_known_cases():
    sq = [(0, 0), (1, 0), (1, 1), (0, 1)]
    assert abs(bench.convex_iou(sq, sq) - 1.0) < 1e-12
    assert abs(bench.convex_iou(sq, [(0.5, 0), (1.5, 0), (1.5, 1), (0.5, 1)]) - 1 / 3) < 1e-12
    assert bench.convex_iou(sq, [(2, 2), (3, 2), (3, 3), (2, 3)]) == 0.0
    assert abs(bench.convex_iou(sq[::-1], [(0, 0), (2, 0), (2, 2), (0, 2)]) - 0.25) < 1e-12  # orientation-free
    tri = [(0, 0), (1, 0), (0, 1)]
    assert abs(bench.convex_iou(tri, sq) - 0.5) < 1e-12
    assert abs(bench.polygon_area(sq) - 1.0) < 1e-12
