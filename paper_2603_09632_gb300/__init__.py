"""GB300 (sm_103a) differentiable Gaussian-splatting rasterizer of the X-GS Perceiver.

The compute path is the CUDA library ``libgs.so`` behind the C ABI in ``include/gs.h``;
``_lib`` is its ctypes binding (argument marshalling only), ``render`` a convenience
layer, ``autograd`` the ``torch.autograd.Function``; the serving loop is ``_lib.Server``.
The library is loaded on first use of any of these names and loading raises if it has
not been built (``python -m paper_2603_09632_gb300._build``); there is no fallback.
"""
import importlib

_EXPORTS = {
    "GSError": "_lib", "Scene": "_lib", "Workspace": "_lib", "make_camera": "_lib",
    "Rasterizer": "render", "as_camera": "render",
}

__all__ = sorted(_EXPORTS)


def __getattr__(name):
    if name in _EXPORTS:
        mod = importlib.import_module(f".{_EXPORTS[name]}", __name__)
        return getattr(mod, name)
    raise AttributeError(name)
