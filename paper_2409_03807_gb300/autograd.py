"""torch.autograd.Function around the training kernels of liblsn.

``LipschitzTrainingLoss.apply(theta, q, ctx, lambda_ls)`` returns the scalar
L = L_C + lambda_ls L_LS (Eq. 10) for the flat float64 parameter tensor
``theta`` and snapshot positions ``q`` (B x n, float64); its backward pass
is the library's hand-written backward kernels (lsn_train_eval), which
recompute the per-tet quantities instead of storing them.  Argument
marshalling only: every step runs in the CUDA kernels.
"""
import torch


class LipschitzTrainingLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, q, lctx, lambda_ls):
        lctx.train_set_params(theta.detach().to(torch.float64).contiguous())
        grad = torch.empty(theta.shape, dtype=torch.float64, device=theta.device)
        losses, _ = lctx.train_eval(q.detach().contiguous(), lambda_ls, grad=grad)
        fctx.save_for_backward(grad)
        fctx.theta_dtype = theta.dtype
        return theta.new_tensor(losses[2], dtype=torch.float64)

    @staticmethod
    def backward(fctx, grad_out):
        (grad,) = fctx.saved_tensors
        return (grad_out.to(grad.dtype) * grad).to(fctx.theta_dtype), None, None, None
