"""GB300-native Schwarz waveform relaxation (SWR) for i u_t + u_xx + V u = 0 (Besse & Xing).

The compute path is the C-ABI library ``libswr.so`` (hand-written sm_103a CUDA);
``paper_1503_02564_gb300.swr`` is its thin ctypes binding.  Importing the package
does not load the library; the first call into the binding does, and fails
loudly if it is missing.
"""
__all__ = ["swr", "workloads"]
