"""GB300-native polyphase filter bank (arXiv 1411.3656).

The compute path is the C-ABI library ``libppf.so`` (hand-written sm_103a CUDA,
declared in ``include/ppf.h``).  ``paper_1411_3656_gb300.ppf`` is a thin ctypes
binding with the same entry-point names; it is imported lazily so that the
input generators in ``paper_1411_3656_gb300.synth`` work without a GPU.
"""
__version__ = "0.1.0"


def __getattr__(name):
    if name == "ppf":
        import importlib
        return importlib.import_module(".ppf", __name__)
    raise AttributeError(name)
