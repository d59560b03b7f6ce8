"""GB300-native WD WENO 2x image zoom (arXiv 2312.00229).

The compute path is the CUDA library ``libwdweno.so`` (sources in ``csrc/``,
C ABI in ``include/wdweno.h``); this package is a thin ctypes binding around
it plus a ``torch.autograd.Function``.  Submodules load lazily so that the
seeded scene generators can be imported on a machine without the library.
"""
from __future__ import annotations

import importlib

__all__ = ["zoom2x", "zoom2x_fwd", "zoom2x_bwd", "zoom2x_batched", "Params", "lib", "scenes",
           "WenoZoom2x", "BatchedPlan", "HostPipeline", "cascade_zoom", "resample", "zoom_to"]


def __getattr__(name):
    if name in ("zoom2x", "zoom2x_fwd", "zoom2x_bwd", "zoom2x_batched", "Params", "lib",
                "WenoZoom2x", "BatchedPlan", "HostPipeline", "cascade_zoom", "resample",
                "zoom_to"):
        mod = importlib.import_module(".api", __name__)
        return getattr(mod, name)
    if name in ("scenes", "binding", "api", "autotune"):
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
