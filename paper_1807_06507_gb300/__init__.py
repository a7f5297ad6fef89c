"""GB300-native sliding-window inter-channel Pearson correlation.

From-scratch implementation of the hot path of Poyda & Zhizhin,
"Optimization of the n-dimensional sliding window inter-channel correlation
algorithm for multi-core architecture" (arXiv:1807.06507): Pearson c of
every sliding window of two equal-size grids, computed from separable sliding
sums of x, y, xy, x^2 and y^2 in fused CUDA kernels for sm_103a, behind the C
ABI of include/swcorr.h.

    from paper_1807_06507_gb300 import swcorr
    plan = swcorr.Plan((3000, 4000), k=7, dtype="u16")
    c = plan.run(x_cuda, y_cuda)

The binding loads the in-tree libswcorr.so (built by ``build.build()``) and
raises if it is missing.
"""
__all__ = ["swcorr", "build", "workloads"]
