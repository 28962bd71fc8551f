"""The complex-gradient convention the force follows: for a real loss L and complex
z, PyTorch returns dL/dRe z + i dL/dIm z (checked on L = |z|^2, gradient 2z), the
same convention as G = dS/dRe U + i dS/dIm U of rhmc_force."""
import torch


def test_torch_complex_gradient_convention():
    z = torch.tensor([1.5 - 0.25j, -0.3 + 2.0j], dtype=torch.complex128, requires_grad=True)
    L = (z.abs() ** 2).sum()
    L.backward()
    assert torch.allclose(z.grad, 2 * z.detach())
    # a real linear functional Re <G, z> has gradient G
    G = torch.tensor([0.7 + 0.1j, -1.0 - 3.0j], dtype=torch.complex128)
    z2 = z.detach().clone().requires_grad_(True)
    (torch.vdot(G, z2).real).backward()
    assert torch.allclose(z2.grad, G)
