"""The backward rule used by the differentiable contraction (holomorphic derivatives in, PyTorch
conjugate-Wirtinger gradients out) checked by gradcheck on a small multilinear function with the
same structure: holomorphic in complex vectors, linear in a real matrix. CPU only."""
import torch

from paper_2107_13952_gb300 import vjp_from_holomorphic


class Bilinear(torch.autograd.Function):
    # a = psi1^T B psi2 with psi complex, B real: holomorphic derivatives
    # d a/d psi1 = B psi2, d a/d psi2 = B^T psi1, d a/d B = psi1 psi2^T
    @staticmethod
    def forward(ctx, p1, p2, B):
        ctx.save_for_backward(p1, p2, B)
        return (p1 @ B.to(p1.dtype) @ p2).reshape(())

    @staticmethod
    def backward(ctx, g):
        p1, p2, B = ctx.saved_tensors
        Bc = B.to(p1.dtype)
        return (vjp_from_holomorphic(g, Bc @ p2, False), vjp_from_holomorphic(g, Bc.T @ p1, False),
                vjp_from_holomorphic(g, torch.outer(p1, p2), True))


def test_backward_rule_matches_gradcheck():
    torch.manual_seed(0)
    p1 = torch.randn(4, dtype=torch.complex128, requires_grad=True)
    p2 = torch.randn(3, dtype=torch.complex128, requires_grad=True)
    B = torch.randn(4, 3, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(Bilinear.apply, (p1, p2, B))
