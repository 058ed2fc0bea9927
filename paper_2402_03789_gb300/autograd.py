"""torch.autograd.Function over the hand-written convolution kernels.

Forward: the fused convolution of one interaction block (Eq. 3, Figure 2b):
radial MLP of the edge lengths, CG tensor product with the edge harmonics and
the sum into receivers.  Backward: the adjoint kernel (Eqs. 5 and 8) giving
dL/dx and dL/dd (through the tensor product, the radial MLP and the edge
embedding).  No PyTorch arithmetic runs on either pass.
"""

import torch


class ConvFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, d, model, layer, row_ptr, src, precision):
        x = x.contiguous()
        d = d.contiguous()
        m = model.conv_forward(layer, row_ptr, src, d, x, precision)
        ctx.save_for_backward(x, d, row_ptr, src)
        ctx.model = model
        ctx.layer = layer
        ctx.precision = precision
        return m

    @staticmethod
    def backward(ctx, g_m):
        x, d, row_ptr, src = ctx.saved_tensors
        g_x, g_d = ctx.model.conv_backward(ctx.layer, row_ptr, src, d, x, g_m.contiguous(), ctx.precision)
        return g_x, g_d, None, None, None, None, None


def conv(model, layer, x, d, row_ptr, src, precision="fp32"):
    """Messages m [n_atoms, m_dim] of block `layer`; differentiable in x and d.

    x: [n_atoms, x_dim] float32 (irreps as [l][m][channel] blocks), d: [E, 3]
    float32 edge vectors r_src - r_recv, row_ptr/src: int32 CSR by receiver.
    """
    return ConvFunction.apply(x, d, model, layer, row_ptr, src, precision)
