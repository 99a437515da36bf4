"""Standalone GB300 microbenchmarks behind design choices of the scan kernels.

    python -m paper_2201_10956_gb300.microbench mma_b1      # binary tensor-core rate
    python -m paper_2201_10956_gb300.microbench mma_issue   # tcgen05.mma issue cost by form
    python -m paper_2201_10956_gb300.microbench mufu_lg2    # lg2.approx throughput (K2 bound)

Each is one CUDA source beside this file, compiled with nvcc for sm_103a into the package's
build folder and run; it prints its measurements.  They are not part of the library."""
