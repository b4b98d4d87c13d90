"""GB300-native open-boundary SPH: the arbitrary-positioned in-/outflow buffer of arXiv 2406.16786.

The compute path is the CUDA library ``libsphbuf.so`` (sources in ``csrc/``, C ABI in
``include/sphbuf.h``); ``domain.Domain`` is its Python binding.  ``workloads`` builds seeded
synthetic channel and pipe problems.  There is no CPU fallback: without the built library
every call raises.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "Domain", "Batch", "SphbufError", "rotation_from_normal", "cell_list_build"]


def __getattr__(name):
    if name in ("Domain", "Batch", "SphbufError", "rotation_from_normal", "cell_list_build"):
        from . import domain

        return getattr(domain, name)
    raise AttributeError(name)
