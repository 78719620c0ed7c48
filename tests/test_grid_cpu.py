"""Host logic of the grid evaluation of the winding-number field (no GPU):
node coordinates, their order and chunking, and the box around the cloud."""
import torch

from paper_2405_16634_b300 import wnf


def test_grid_points_order_and_chunks():
    lo = torch.tensor([-1.0, 0.0, 2.0])
    res, side = 5, 4.0
    full = wnf.grid_points(lo, side, res)
    assert full.shape == (res ** 3, 3) and full.dtype == torch.float32
    assert torch.equal(full[0], lo)
    assert torch.allclose(full[-1], lo + side)
    # z fastest, then y, then x
    assert torch.allclose(full[1] - full[0], torch.tensor([0.0, 0.0, 1.0]))
    assert torch.allclose(full[res] - full[0], torch.tensor([0.0, 1.0, 0.0]))
    assert torch.allclose(full[res * res] - full[0], torch.tensor([1.0, 0.0, 0.0]))
    parts = [wnf.grid_points(lo, side, res, k0, min(k0 + 17, res ** 3)) for k0 in range(0, res ** 3, 17)]
    assert torch.equal(torch.cat(parts), full)


def test_grid_box_covers_the_cloud_with_padding():
    pts = torch.tensor([[0.0, 0.0, 0.0], [2.0, 1.0, 0.5], [1.0, -1.0, 0.25]])
    lo, side = wnf.grid_box(pts, pad=0.1)
    assert abs(side - 2.0 * 1.2) < 1e-6          # largest extent 2 (x and y), padded by 0.1 on each side
    hi = lo + side
    assert torch.all(lo <= pts.min(0).values) and torch.all(hi >= pts.max(0).values)
    assert torch.allclose(0.5 * (lo + hi), 0.5 * (pts.min(0).values + pts.max(0).values))
