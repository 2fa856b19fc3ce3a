"""CPU FP64 oracle for the APLICUR preconditioned-LSQR path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or execute anything in this package: only the tests, the smoke check and the
CPU-baseline leg of the benchmark use it.  It shares no code with the CUDA
library; the one thing both sides take from a common place is the seeded input
data (the workloads module), which holds none of the method's arithmetic.

Every function restates a step of the paper in plain numpy/scipy, in the
paper's order and notation, without blocking or fusion.
"""
