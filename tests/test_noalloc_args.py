"""Host-side argument checks of the allocation-free residual-norm wrapper: the C entry
point has no context to check sizes against, so the binding refuses mismatched
shapes, short outputs and arrays on different devices before any launch."""

import pytest

torch = pytest.importorskip("torch")


def _binding():
    from paper_1710_09913_gb300 import build
    build.build()
    from paper_1710_09913_gb300 import binding as B
    return B


def test_refuses_mismatched_shapes():
    B = _binding()
    b = torch.zeros(10, 3, dtype=torch.float64)
    with pytest.raises(ValueError, match="Ky"):
        B.residual_norms_noalloc(b, torch.zeros(9, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="r must"):
        B.residual_norms_noalloc(b, torch.zeros_like(b), r=torch.zeros(10, 2, dtype=torch.float64))
    with pytest.raises(ValueError, match="b must"):
        B.residual_norms_noalloc(torch.zeros(2, 2, 2, dtype=torch.float64),
                                 torch.zeros(2, 2, 2, dtype=torch.float64))


def test_refuses_host_tensors():
    B = _binding()
    b = torch.zeros(10, 3, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        B.residual_norms_noalloc(b, torch.zeros_like(b))
