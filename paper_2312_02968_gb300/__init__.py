"""GB300-native MOND particle-mesh force pipeline (Visser, Eijt & de Nijs 2023).

The compute path lives in the CUDA library ``libmondpm.so`` behind the C ABI of
``include/mond_pm.h``; ``binding`` marshals arguments into it and nothing else.
Importing this package does not load the library; ``binding.lib()`` does, and
raises if it has not been built.
"""
__all__ = ["binding", "workloads"]
