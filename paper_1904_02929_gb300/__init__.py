"""GB300-native (sm_103a) sheared-suspension step of arXiv:1904.02929.

The compute path is the CUDA library ``libsusp.so`` behind the C ABI of
``include/susp.h``; ``paper_1904_02929_gb300.susp`` is its Python binding and
``paper_1904_02929_gb300.inputs`` holds the seeded synthetic workloads.
"""
__all__ = ["susp", "inputs", "build"]
