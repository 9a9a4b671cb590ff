"""B300-native componentwise ADMM for linearized multi-phase OPF.

The compute path is the C-ABI library ``libopf_admm.so`` (sm_103a CUDA and
host C++), reached through :mod:`paper_2501_08293_b300.opf`.  Importing this
package does not load the library; ``feeders`` (synthetic input data) can be
used on machines without a GPU.
"""
__version__ = "0.1.0"
