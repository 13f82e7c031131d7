"""CPU oracle (FP64, plain numpy/scipy) for the restarted PDHG path.

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the CPU
baseline leg of the benchmark.  The CUDA product path never imports it.
"""
