"""torch.autograd.Function over the CRN particle filter.

forward  = one fused launch of the filter forward pass and its reverse-time
           adjoint (pf_loglik_grad): log p-hat(y|theta_i) for every row i and the
           gradient d log p-hat / d theta_i, kept for backward;
backward = grad_out[:, None] * gradient (no further device work).
The gradient is the one of App. A/B (common random numbers and ancestors held
fixed), so it is exact for the estimator, as the paper's autograd gradient is.

Stream order: the handle enqueues on its own stream.  forward makes that stream
wait for torch's current stream (so theta is ready) and makes the current stream
wait for the handle's work (so the outputs are ready for the ops that follow).
theta's contiguous copy and the outputs are allocated on the current stream, and
torch's caching allocator hands a freed block only to later allocations on that
same stream, whose work is queued behind the wait: no memory the kernels touch can
be reused while they run.  (The tensors are not marked as used on the handle's
stream: that stream may be destroyed with the handle before they are freed.)
"""
import torch

from . import binding


class CRNPFLogLik(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, handle, iteration=1):
        if not theta.is_cuda or theta.dtype != torch.float64:
            raise TypeError("theta must be a float64 CUDA tensor")
        th = theta.detach().contiguous()
        n = th.shape[0]
        ll = torch.empty(n, dtype=torch.float64, device=th.device)
        grad = torch.empty_like(th) if theta.requires_grad else None
        with torch.cuda.device(th.device):
            cur = torch.cuda.current_stream(th.device)
            hs_ptr = handle.stream_ptr()
            if hs_ptr == cur.cuda_stream:
                handle.pf_loglik_grad(th, iteration, ll, grad)
            else:
                hs = torch.cuda.ExternalStream(hs_ptr, device=th.device)
                hs.wait_stream(cur)  # theta (and its contiguous copy) written first
                handle.pf_loglik_grad(th, iteration, ll, grad)
                cur.wait_stream(hs)  # later ops on the current stream see ll and grad
        ctx.save_for_backward(grad if grad is not None else th.new_zeros(0))
        return ll

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        return grad_out[:, None] * grad, None, None


def loglik(theta, handle, iteration=1):
    """log p-hat for each row of theta (differentiable w.r.t. theta)."""
    return CRNPFLogLik.apply(theta, handle, iteration)
