"""gbfft: batched one-dimensional complex-to-complex FFTs on GB300 (sm_103a).

The compute path is the C-ABI library ``libgbfft.so`` built from ``csrc/``;
:mod:`paper_2207_06803_gb300.gbfft` is its thin ctypes binding.  Importing this
package loads nothing: the library is opened on first use and a missing or
unbuilt library raises instead of falling back to any other implementation.
"""
