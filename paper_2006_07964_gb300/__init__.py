"""GB300-native high-order curvilinear Navier-Stokes RK-stage residual (HiResX hot path).

The compute path lives in the CUDA library ``libhx.so`` built from ``csrc/``;
``hx`` is its thin ctypes binding (argument marshalling only) and
``workloads`` builds the synthetic inputs.
"""
