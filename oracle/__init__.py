"""FP64 CPU oracle for the stencil iteration spaces: test infrastructure only.

Only the test suite, the smoke check and the benchmark's CPU baseline may
import this package; the CUDA library never does.
"""
