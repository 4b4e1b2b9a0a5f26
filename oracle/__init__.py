"""ORACLE (test infrastructure only): plain CPU restatement of the UGKWP-LTS step, used to check the CUDA
library. Only tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import it."""
