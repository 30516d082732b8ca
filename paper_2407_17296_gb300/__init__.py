"""GB300-native CRN particle filter and gradient-enhanced SMC^2 (arXiv 2407.17296).

The compute path is the CUDA library ``libsmc2.so`` (C ABI in include/smc2.h);
``binding`` marshals arguments to it, ``autograd`` wraps the filter as a
torch.autograd.Function, ``workloads`` generates seeded synthetic inputs.
Submodules are imported lazily so that input generation needs no GPU.
"""
__all__ = ["binding", "autograd", "workloads", "build"]
