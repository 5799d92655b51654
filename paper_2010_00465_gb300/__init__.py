"""GB300 (sm_103a) library computing cos(A) and sin(A) of a dense matrix together,
by the factorised Taylor method of arXiv:2010.00465.

The compute path lives in ``libcossin.so`` (C ABI in ``include/cossin.h``);
``api`` wraps it for PyTorch tensors.  Importing this package loads nothing:
the library is opened on first use and a missing build raises.
"""
from . import build  # noqa: F401  (module: build.build() compiles the library)


def __getattr__(name):
    if name in ("cossin", "norm1", "select", "workspace_size", "prof_enable", "prof_reset",
                "prof_read", "PRECISIONS"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
