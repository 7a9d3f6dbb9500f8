"""zd-tree exact k-NN in low dimensions on one GB300 (sm_103a).

The compute path lives in the CUDA library ``libzd`` (``csrc/``); the module
``zd`` is a thin ctypes binding with the C ABI's names.  Importing this
package loads nothing: the library is opened on first use, and every entry
point raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["zd", "datagen"]
