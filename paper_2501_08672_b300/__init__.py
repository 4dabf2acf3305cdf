"""B300-native differentiable Gaussian-splatting path of GS-LIVO (arXiv 2501.08672).

The compute path is the C-ABI library `libgs_b300.so` (hand-written sm_103a
CUDA, see include/gs.h); `binding` marshals arguments to it and `render`
wraps it as a torch.autograd.Function.  `scenes` draws seeded synthetic
inputs.
"""
