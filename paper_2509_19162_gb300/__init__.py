"""GB300-native (sm_103a) growth of permutation Cayley graphs.

The hot path of CayleyPy's growth computation (arxiv 2509.19162): breadth-first growth of a
Cayley graph from the identity, returning the sphere sizes |S_r| (Section 2.1, Def. "Growth").
Kernels and driver live in ``csrc/`` behind the C ABI of ``include/cg_growth.h``; this
package is the thin Python binding.  ``build()`` compiles the library for sm_103a.
"""



def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library for sm_103a (no-op when up to date); returns its path."""
    from .builder import build as _build
    return _build(force=force, verbose=verbose)


_API = ("Growth", "GrowthResult", "growth", "Batch", "use_torch_allocator", "STRATEGIES", "shard",
        "unshard")


def __getattr__(name):
    if name in _API:
        from . import api as _g
        return getattr(_g, name)
    if name == "serve":
        from . import serve as _s
        return _s
    raise AttributeError(name)
