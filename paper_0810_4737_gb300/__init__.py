"""GB300-native REED-MD track stepper.

``paper_0810_4737_gb300.reed`` is the Python binding of the CUDA library
(``include/reed.h``); ``paper_0810_4737_gb300.workloads`` holds the synthetic
workload definitions; ``paper_0810_4737_gb300.build`` compiles the library.
Submodules are imported on first use so that importing the package needs
neither the GPU nor the compiled library.
"""
import importlib

__all__ = ["reed", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
