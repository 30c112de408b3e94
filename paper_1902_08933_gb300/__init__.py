"""GB300 (sm_103a) phase-field lattice Boltzmann library, arXiv:1902.08933.

The compute path is the C-ABI library ``liblbm.so`` built from ``csrc/``;
``paper_1902_08933_gb300.lbm`` is its thin ctypes binding. Importing this
package loads nothing: the library is loaded, and its absence reported, on
first use.
"""
__all__ = ["lbm", "workloads"]
