"""GB300 batched pose evaluator for the geometric docking kernel of GeoDock-MA.

A thin Python binding over the C ABI of ``libgeodock.so`` (declared in
``include/geodock.h``): the functions keep the C names and only marshal
arguments. Every step of the path (field, initial poses, fragment rotation,
bump check, score, argmax, best pose) runs in the library's CUDA kernels;
there is no CPU fallback. The library is loaded on first use of any name
below and a missing library raises ImportError; build it with
``python -m paper_1901_06363_gb300.build``.
"""
_EXPORTS = ("Docker", "DockError", "dock_knobs", "knobs_struct", "lib", "library_path", "RESULT_DTYPE", "DOCK_OK",
            "DOCK_ERR_INVALID_ARG", "DOCK_ERR_TOPOLOGY", "DOCK_ERR_OUT_OF_MEMORY", "DOCK_ERR_CUDA",
            "DOCK_ERR_TIMEOUT", "DOCK_ERR_UNSUPPORTED")

__all__ = list(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        from . import binding
        return getattr(binding, name)
    raise AttributeError(name)
