"""GB300-native dense 3-D deformable registration hot path (arXiv 2509.25044).

The compute runs in hand-written CUDA kernels for sm_103a behind a C ABI
(``include/reg.h``); ``paper_2509_25044_gb300.capi`` binds it with ctypes.
Submodules are imported lazily so that the synthetic-data generators can be
used without loading the CUDA library.
"""
__all__ = ["capi", "synth", "torch_ops"]


def __getattr__(name):
    import importlib
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
