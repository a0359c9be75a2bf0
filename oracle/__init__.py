"""CPU FP64 oracle (test infrastructure only).

Plain NumPy/SciPy restatement of the paper's scheme and solver, plus a plain C
ILU(0).  Only the tests, the smoke check and the benchmark's CPU-baseline /
reference leg may import it; the CUDA library never does.
"""
