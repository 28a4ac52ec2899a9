"""Host logic of the reconstruction drivers, on CPU tensors: the per-instance
inner products and broadcasts that give CGLS its per-instance step lengths."""
import torch

from paper_2604_19176_gb300.recon import _Segments


class _FakePlan:
    """Just the layout of a plan with two uneven instances (3x3 and 2x2 images,
    data of 4 and 6 elements)."""

    device = torch.device("cpu")
    geoms = [object(), object()]

    def layout(self):
        return [0, 9, 13], [0, 4, 10]


def test_segment_dot_and_expand():
    seg = _Segments(_FakePlan())
    a = torch.arange(13, dtype=torch.float32)
    b = torch.ones(13)
    d = seg.dot(a, b, image=True)
    assert d.dtype == torch.float64
    assert d.tolist() == [float(sum(range(9))), float(sum(range(9, 13)))]
    g = torch.arange(10, dtype=torch.float32)
    assert seg.dot(g, g, image=False).tolist() == [float(sum(i * i for i in range(4))),
                                                   float(sum(i * i for i in range(4, 10)))]
    e = seg.expand(torch.tensor([2.0, -1.0], dtype=torch.float64), True, a)
    assert e.tolist() == [2.0] * 9 + [-1.0] * 4
    e = seg.expand(torch.tensor([2.0, -1.0]), False, g.reshape(2, 5))
    assert e.shape == (2, 5) and e.reshape(-1).tolist() == [2.0] * 4 + [-1.0] * 6
