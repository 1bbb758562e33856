"""FP64 CPU oracle of the semilinear full multigrid method (arXiv 1611.05677).

Test infrastructure only: the tests, the smoke check and the benchmark's CPU
baseline leg import it; the CUDA solver never does.
"""
