"""GB300 (sm_103a) hot path of Language Embedded 3D Gaussians (arXiv 2311.18482).

The CUDA library libleg.so (C ABI in include/leg.h) is built in place by
`paper_2311_18482_gb300.build`; `binding` marshals torch tensors into it.
`synth` draws the seeded synthetic workloads.  Attributes of `binding` are
re-exported lazily so importing `synth` does not load torch or the library.
"""
import importlib

_SUBMODULES = ("binding", "build", "synth", "training")


def __getattr__(name):
    if name.startswith("__"):
        raise AttributeError(name)
    if name in _SUBMODULES:
        return importlib.import_module(f"{__name__}.{name}")
    binding = importlib.import_module(f"{__name__}.binding")
    try:
        return getattr(binding, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
