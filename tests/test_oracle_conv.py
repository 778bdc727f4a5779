"""Pins for the oracle's 3-D convolution of the learned initialiser and its
adjoints: equal to torch.nn.functional.conv3d (FP64, CPU) and its autograd
gradients, the library special case of the plain definition."""
import numpy as np
import torch

import oracle as O


def _torch_weight(w):
    # [Cout][27][Cin] with tap t = (kz*3+ky)*3+kx  ->  [Cout][Cin][kz][ky][kx]
    cout, _, cin = w.shape
    return torch.tensor(w.reshape(cout, 3, 3, 3, cin).transpose(0, 4, 1, 2, 3).copy())


def test_conv_forward_and_adjoints_equal_torch(rng):
    nz, ny, nx, cin, cout = 5, 6, 7, 3, 4
    x = rng.standard_normal((nz, ny, nx, cin))
    w = rng.standard_normal((cout, 27, cin))
    b = rng.standard_normal(cout)
    out = O.conv3d(x, w, b)
    xt = torch.tensor(x.transpose(3, 0, 1, 2)[None].copy(), requires_grad=True)
    wt = _torch_weight(w).requires_grad_(True)
    ref = torch.nn.functional.conv3d(xt, wt, torch.tensor(b), padding=1)
    np.testing.assert_allclose(out, ref[0].detach().numpy().transpose(1, 2, 3, 0), atol=1e-12)
    g = rng.standard_normal(out.shape)
    (ref * torch.tensor(g.transpose(3, 0, 1, 2)[None].copy())).sum().backward()
    din = O.conv3d_dgrad(g, w)
    np.testing.assert_allclose(din, xt.grad[0].numpy().transpose(1, 2, 3, 0), atol=1e-11)
    dw = O.conv3d_wgrad(x, g)
    np.testing.assert_allclose(_torch_weight(dw).numpy(), wt.grad.numpy(), atol=1e-10)


def test_adjoint_dot_product(rng):
    nz, ny, nx, cin, cout = 4, 5, 3, 2, 3
    x = rng.standard_normal((nz, ny, nx, cin))
    w = rng.standard_normal((cout, 27, cin))
    g = rng.standard_normal((nz, ny, nx, cout))
    lhs = np.sum(O.conv3d(x, w) * g)
    assert abs(lhs - np.sum(x * O.conv3d_dgrad(g, w))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(w * O.conv3d_wgrad(x, g))) < 1e-10 * abs(lhs)
