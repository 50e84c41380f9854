"""GB300-native best-first graph search (Speed-ANN, arXiv 2201.13007).

The product is libann.so (C ABI in include/ann.h, kernels in csrc/). This
package is its Python binding: ``_abi`` holds the ctypes declarations with the
C names, ``index.Index`` wraps them for torch tensors, ``synth`` builds seeded
inputs. Nothing here computes any part of the search.
"""
from ._abi import (AnnError, ann_index_create, ann_index_destroy, ann_index_get_info,  # noqa: F401
                   ann_last_error, ann_search, ann_search_ex, ann_search_host)


def __getattr__(name):
    if name in ("Index", "stats_dict"):
        from . import index
        return getattr(index, name)
    raise AttributeError(name)
