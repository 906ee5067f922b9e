"""GB300-native upper hood (Wagener's merge schedule) behind a C ABI.

The compute path is the CUDA library ``libwagener.so`` (built from ``csrc/``
for sm_103a); this package only marshals arguments to it. Importing the
package is cheap: the library is loaded on first use by ``_lib``.
"""
__all__ = ["inputs"]
