"""GB300-native coalesced-ghost Vlasov translation (sm_103a CUDA behind a C ABI).

The compute path lives in the shared library built from ``csrc/`` (see ``vlasov.py``
for the Python binding of the C ABI declared in ``include/vlasov.h``).  Importing this
package does not load the library; ``vlasov.load()`` does, and fails loudly when the
CUDA library has not been built.
"""
__all__ = ["inputs", "vlasov"]
