"""GB300-native TopoSZp: topology-aware error-bounded compression of float32
scientific fields (arXiv 2602.17552), as hand-written CUDA kernels for sm_103a
behind a C ABI (include/toposzp.h).

Submodules are imported lazily so that ``paper_2602_17552_gb300.synth`` (input
generators) can be used without loading the CUDA library.
"""
import importlib

__all__ = ["codec", "synth", "batch", "serve", "build"]

_EXPORTS = {
    "compress": "codec", "decompress": "codec", "compress_async": "codec", "decompress_async": "codec",
    "critical_points": "codec", "topo_errors": "codec", "inspect": "codec", "unpack_labels": "codec",
    "compress_bound": "codec", "TopoSZpError": "_lib",
}


def __getattr__(name):
    if name in _EXPORTS:
        return getattr(importlib.import_module(f".{_EXPORTS[name]}", __name__), name)
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
