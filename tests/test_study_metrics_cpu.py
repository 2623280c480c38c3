"""The supervision study's metrics (bench.py) on hand-computable inputs: the
symmetric Chamfer distance and the pixel dilation that defines "within r
pixels of a thin part"."""
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_chamfer_is_the_average_of_the_two_directed_means():
    P = torch.tensor([[0.0, 0.0, 0.0]], dtype=torch.float64)
    Q = torch.tensor([[1.0, 0.0, 0.0], [3.0, 0.0, 0.0]], dtype=torch.float64)
    # P -> Q: 1; Q -> P: (1 + 3) / 2 = 2
    assert bench._chamfer(torch, P, Q) == 1.5
    assert bench._chamfer(torch, Q, P) == 1.5
    assert bench._chamfer(torch, Q, Q) == 0.0
    assert bench._chamfer(torch, P[:0], Q) != bench._chamfer(torch, P[:0], Q)   # NaN when a set is empty


def test_chamfer_of_a_translated_cloud():
    g = torch.Generator().manual_seed(3)
    P = torch.rand(500, 3, generator=g, dtype=torch.float64) * 10
    shift = torch.tensor([0.0, 0.0, 1e-3], dtype=torch.float64)
    # the points are far apart compared with the shift, so every nearest
    # neighbour is the translated copy
    assert abs(bench._chamfer(torch, P, P + shift) - 1e-3) < 1e-12


def test_dilation_marks_the_square_neighbourhood_per_view():
    V, W = 2, 7
    mask = torch.zeros(V * W * W, dtype=torch.bool)
    mask[1 * W * W + 3 * W + 3] = True                   # view 1, pixel (3, 3)
    for r, side in ((0, 1), (1, 3), (2, 5)):
        got = bench._dilate(torch, mask, V, W, r).view(V, W, W)
        assert not got[0].any()                           # views do not leak into each other
        assert int(got[1].sum()) == side * side
        assert got[1, 3 - r:4 + r, 3 - r:4 + r].all()
    edge = torch.zeros(V * W * W, dtype=torch.bool)
    edge[0] = True                                        # view 0, corner pixel
    assert int(bench._dilate(torch, edge, V, W, 1).sum()) == 4
